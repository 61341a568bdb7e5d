// fsp_learned.cu -- kernels of the learned pair order in the search: the
// generic parent features and top-K (network shapes without the fused
// inference kernel), phase 1 (each child's predicted pairs: cut or list) and
// phase 2 (the full bound of the listed children).
#include "fsp_solve.cuh"

// ---------------------------------------------------------- learned order --

// Features of the popped parents (parent t = stack[S - 1 - t]).
__global__ void k_parent_features(DevInst I, SolveWs ws, float T)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const SolveCtl *ctl = ws.ctl;
    if (t >= ctl->n_parents) return;
    const long long S = ctl->s_pop + ctl->n_parents;
    int32_t C[FSP_MAX_MACHINES], Sr[FSP_MAX_MACHINES], Q[FSP_MAX_MACHINES];
    uint32_t U[8];
    fsp_features(I, ws.stack + (S - 1 - t) * I.stride, T, ws.px + t * (2 * I.m + 1), U, C, Sr, Q);
}

// The K best-scored pairs of each parent, best first (ties: lower pair index).
__global__ void k_topk(SolveWs ws, int P, int K)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ws.ctl->n_parents) return;
    const float *sc = ws.pscore + t * P;
    int16_t *out = ws.topk + t * K;
    uint32_t taken[FSP_MAX_MACHINES * (FSP_MAX_MACHINES - 1) / 2 / 32 + 1];
    for (int w = 0; w < (P + 31) / 32; ++w) taken[w] = 0u;
    for (int j = 0; j < K; ++j) {
        int best = -1;
        float bv = 0.f;
        for (int q = 0; q < P; ++q) {
            if (taken[q >> 5] & (1u << (q & 31))) continue;
            const float v = sc[q];
            if (best < 0 || v > bv) { best = q; bv = v; }
        }
        if (best < 0) best = 0;
        taken[best >> 5] |= 1u << (best & 31);
        out[j] = (int16_t)best;
    }
}

// Phase 1: branch, then evaluate each child's K predicted pairs; a child
// whose partial bound reaches the iteration's UB is cut (its full bound is
// at least as large), the others go to the list for the full bound.
template <int MT, int NV, int NW>
__global__ void __launch_bounds__(256) k_branch_learned(DevInst I, SolveWs ws, Bound2Smem L, int K)
{
    const SolveCtl *ctl = ws.ctl;
    const long long nch = ctl->n_children;
    const int B = blockDim.x, tid = threadIdx.x;
    if ((long long)blockIdx.x * B >= nch) return;
    extern __shared__ __align__(16) unsigned char smem[];
    FspEntry *ent_s = reinterpret_cast<FspEntry *>(smem + L.ent_off);
    int2 *pq_s = reinterpret_cast<int2 *>(smem + L.pq_off);
    int32_t *cs = reinterpret_cast<int32_t *>(smem + L.cs_off);
    int32_t *sq = reinterpret_cast<int32_t *>(smem + L.sq_off);
    fsp_stage_pq(I, ent_s, pq_s);
    const int n = I.n, stride = I.stride;
    const int np = (int)ctl->n_parents;
    const long long S = ctl->s_pop + np;
    const int ub_iter = ctl->ub_iter;
    const long long c = (long long)blockIdx.x * B + tid;
    bool listed = false, cut = false;
    if (c < nch) {
        const int pi = solve_parent_of(ws.poff, np, c);
        const int ci = (int)(c - __ldg(ws.poff + pi));
        FspRec<NV> par, ch;
        fsp_load_rec(par, ws.stack + (S - 1 - pi) * stride);
        fsp_make_child(par, n, ci, ch);
        fsp_store_rec(ch, ws.children + c * stride);
        uint32_t Um[NW];
        int32_t C[MT], SQ[MT], lb;
        bool bad;
        fsp_prologue<MT, NV, NW>(ch, n, pq_s, I.mp, Um, C, SQ, lb, bad, I.var);
#pragma unroll
        for (int k = 0; k < MT; ++k) {
            cs[k * B + tid] = C[k];
            sq[k * B + tid] = SQ[k];
        }
        for (int j = 0; j < K; ++j) {
            const int kl = __ldg(ws.topk + (long long)pi * K + j);
            int k = 0, rem = kl;  // pair index -> (k, l), k-major
            while (rem >= MT - 1 - k) { rem -= MT - 1 - k; ++k; }
            const int l = k + 1 + rem;
            const int4 *e = reinterpret_cast<const int4 *>(ent_s + (size_t)kl * n);
            int32_t E = 0, M = FSP_NEG;
            for (int pos = 0; pos < n; ++pos) {
                const int4 t = e[pos];
                if (fsp_member<NW>(Um, t)) {
                    M = __viaddmax_s32(E, t.x, M);
                    E += t.y;
                }
            }
            lb = __viaddmax_s32(sq[l * B + tid], __viaddmax_s32(cs[k * B + tid], M, cs[l * B + tid]), lb);
        }
        if (lb >= ub_iter) {
            ws.lbs[c] = lb;
            cut = true;
        } else {
            listed = true;
        }
    }
    // warp-aggregated append to the list, and the count of cuts
    const unsigned lm = __ballot_sync(0xffffffffu, listed);
    const unsigned cm = __ballot_sync(0xffffffffu, cut);
    const int lane = tid & 31;
    int base = 0;
    if (lane == 0 && lm) base = (int)atomicAdd((unsigned long long *)&ws.ctl->n_list, (unsigned long long)__popc(lm));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (listed) ws.list[base + __popc(lm & ((1u << lane) - 1u))] = (int)c;
    if (lane == 0 && cm) atomicAdd((unsigned long long *)&ws.ctl->early, (unsigned long long)__popc(cm));
}

// Phase 2: the full bound of the listed children (persistent grid).
template <int MT, int NV, int NW>
__global__ void __launch_bounds__(FSP_B2) k_bound_list(DevInst I, SolveWs ws, Bound2Smem L)
{
    constexpr int NPT = FSP_NPT;
    const SolveCtl *ctl = ws.ctl;
    const long long cnt = ctl->n_list;
    const int B = blockDim.x, tid = threadIdx.x, SB = B * NPT;
    if ((long long)blockIdx.x * SB >= cnt) return;
    extern __shared__ __align__(16) unsigned char smem[];
    FspEntry *ent_s = reinterpret_cast<FspEntry *>(smem + L.ent_off);
    int2 *pq_s = reinterpret_cast<int2 *>(smem + L.pq_off);
    int32_t *cs = reinterpret_cast<int32_t *>(smem + L.cs_off);
    int32_t *sq = reinterpret_cast<int32_t *>(smem + L.sq_off);
    fsp_stage_pq(I, ent_s, pq_s);
    const int n = I.n, stride = I.stride;
    const int ub_iter = ctl->ub_iter;
    int slot[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) slot[j] = tid + j * B;
    for (long long base = (long long)blockIdx.x * SB; base < cnt; base += (long long)gridDim.x * SB) {
        uint32_t Um[NPT][NW];
        int32_t lb[NPT];
        int dch[NPT];
        long long cc[NPT];
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            const long long s2 = base + slot[j];
            cc[j] = s2 < cnt ? (long long)ws.list[s2] : -1;
            FspRec<NV> r;
            if (cc[j] >= 0) {
                fsp_load_rec(r, ws.children + cc[j] * stride);
            } else {
#pragma unroll
                for (int q = 0; q < 4 * NV; ++q) r.w[q] = 0u;
            }
            dch[j] = (int)fsp_rec_byte_dyn(r, n);
            int32_t C[MT], SQ[MT];
            bool bad;
            fsp_prologue<MT, NV, NW>(r, n, pq_s, I.mp, Um[j], C, SQ, lb[j], bad, I.var);
#pragma unroll
            for (int k = 0; k < MT; ++k) {
                cs[k * SB + slot[j]] = C[k];
                sq[k * SB + slot[j]] = SQ[k];
            }
        }
        fsp_pair_scan<MT, NPT, NW>(n, ent_s, cs, sq, SB, slot, Um, lb);
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            if (cc[j] < 0) continue;
            ws.lbs[cc[j]] = lb[j];
            if (dch[j] == n - 1 && lb[j] < ub_iter)
                atomicMin(&ws.ctl->best_key, ((unsigned long long)(uint32_t)lb[j] << 32) | (unsigned long long)cc[j]);
        }
    }
}

BranchLearnedFn pick_branch_learned(int mt, int nv, int nw)
{
#define FSP_CASE2(MT_, NV_, NW_) \
    if (mt == MT_ && nv == NV_ && nw == NW_) return &k_branch_learned<MT_, NV_, NW_>;
    FSP_SHAPES2(FSP_CASE2)
#undef FSP_CASE2
    return nullptr;
}

BoundListFn pick_bound_list(int mt, int nv, int nw)
{
#define FSP_CASE2(MT_, NV_, NW_) \
    if (mt == MT_ && nv == NV_ && nw == NW_) return &k_bound_list<MT_, NV_, NW_>;
    FSP_SHAPES2(FSP_CASE2)
#undef FSP_CASE2
    return nullptr;
}


void launch_parent_features(const DevInst &D, const SolveWs &ws, float T, long long npar, cudaStream_t st)
{
    k_parent_features<<<(unsigned)((npar + 127) / 128), 128, 0, st>>>(D, ws, T);
}

void launch_topk(const SolveWs &ws, int P, int K, long long npar, cudaStream_t st)
{
    k_topk<<<(unsigned)((npar + 127) / 128), 128, 0, st>>>(ws, P, K);
}
