// fsp_family.cu -- branching and bounding a parent's children together
// (steps a1-a6 of one search iteration, sm_103a).
//
// The children of one parent share its prefix and its remaining set U; the
// child that appends job c keeps U \ {c}.  For machine pair (k,l) the
// max-plus term of the two-machine bound (fsp_common.cuh)
//     M = max_{i in U'} (E_{<i} + w_i),  U' the child's remaining set,
// splits around c's position in the pair's Johnson order:
//     X_c = max( max_{i in U, i before c} (E_{<i} + w_i),
//                max_{i in U, i after c}  (E_{<i} + w_i) - e_c ),
// with E_{<i} summed over the parent's U (removing c lowers the sums of every
// later member by e_c and leaves the earlier ones alone).  One forward scan
// (prefix maxima) and one backward scan (suffix maxima) of a pair's order
// give X_c for every child at once.  The one-machine quantities of a child
// follow from the parent's in O(m): the release times advance by job c, the
// remaining sums drop by p[c], and the smallest tail over U \ {c} is the
// parent's smallest unless c attains it, in which case it is the second
// smallest.
//
// Most pairs cannot raise any child's bound above its one-machine bound
// LB1, and those are skipped without changing a single bound: the pair's
// value for child c is SQ_l + max(C_l, C_k + X_c), where SQ_l + C_l <= LB1(c)
// always, and X_c <= M_U + max(0, -e_c) with M_U the full-set term.  So after
// the forward scan alone, pair (k,l) is certified for the whole family when
//     M_U + max(0, -e_c) + SQ_l(c) + C_k(c) <= LB1(c)   for every child c,
// first tested in O(1) with per-machine extremes over the children, then
// child by child for the pairs that fail.  Only the uncertified pairs get
// the backward scan and the per-child lookups.  Every bound is the same
// integer as the per-child evaluation of all pairs (max-plus is associative,
// the sums are exact, and a certified pair's value is <= LB1).  Children at
// depth n-1 need no pair at all: with one job left, LB1 is the makespan and
// no pair exceeds it.
//
// Work split: one warp per parent (a "family").  Lanes own machines for the
// parent state, children for the child state and the lookups, and pairs for
// the scans and the certification.  The CTA is persistent and stages the
// instance tables once.
#include "fsp_family.cuh"

// Asynchronous copy of family f's record (lanes 0..NV-1, 16 bytes each) and
// of the running children count below it (lane NV; its first child is the
// count at the stack top minus this) into this warp's buffers.
template <int NV>
__device__ __forceinline__ void fam_fetch(const SolveWs &ws, long long S, int stride, int f, int lane,
                                          uint8_t *rec_dst, long long *cum_dst)
{
    if (lane < NV) {
        const unsigned d = (unsigned)__cvta_generic_to_shared(rec_dst + lane * 16);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d),
                     "l"(ws.stack + (S - 1 - f) * stride + lane * 16));
    } else if (lane == NV) {
        const unsigned d = (unsigned)__cvta_generic_to_shared(cum_dst);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(ws.cum + (S - 1 - f)));
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int MT, int NV, bool LRN, bool HEADS, bool BIDIR>
__global__ void __launch_bounds__(FAM_MAX_WARPS * 32, 1) k_branch_family(DevInst I, SolveWs ws, FamSmem L)
{
    constexpr int P = MT * (MT - 1) / 2;
    const SolveCtl *ctl = ws.ctl;
    const int W = blockDim.x >> 5;
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = I.n, stride = I.stride, mp = I.mp;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const FamView V = fam_view(smem, L, warp);

    // stage the instance tables (read-only: this may run while the selection
    // ahead of this kernel is still running)
    for (int i = threadIdx.x; i < n * P; i += blockDim.x) V.we[i] = __ldg(I.we + i);
    for (int i = threadIdx.x; i < P * V.rks8; i += blockDim.x) {
        const int kl = i / V.rks8, j = i - kl * V.rks8;
        V.rk8[i] = j < n ? __ldg(I.rank + kl * n + j) : (uint8_t)0;
    }
    for (int i = threadIdx.x; i < n * MT; i += blockDim.x) {
        const int j = i / MT, k = i - j * MT;
        V.pq[j * mp + k] = make_int2(__ldg(I.p + i), __ldg(I.q + i));
    }
    fam_tables_finish<MT>(V, n, mp);
    pdl_wait();  // the selection's control block and stack from here on
    const int np = (int)ctl->n_parents;
    if (blockIdx.x * W >= np) return;

    const long long S = ctl->s_pop + np;  // the stack before the pops (np >= 1 here)
    const long long top = ws.cum[S - 1];  // children of the whole stack
    const int ub_iter = ctl->ub_iter;
    // parents are taken from a shared counter one ahead: the next one's
    // record is copied into the other buffer while this one is processed
    unsigned long long *next_f = reinterpret_cast<unsigned long long *>(&ws.ctl->fam_next);
    int f = 0, buf = 0;
    int fc[4] = {0, 0, 0, 0};  // this warp's family counts (SolveCtl::fam) and early cuts
    if (lane == 0) f = (int)atomicAdd(next_f, 1ull);
    f = __shfl_sync(0xffffffffu, f, 0);
    if (f < np) fam_fetch<NV>(ws, S, stride, f, lane, V.recb, V.pofs);
    // learned order: lane j < K loads the family's j-th predicted pair one family
    // ahead, so the load completes while the previous family is bounded
    int pair = (LRN && f < np && lane < L.K) ? __ldg(ws.topk + (long long)f * L.K + lane) : 0;
    while (f < np) {
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        __syncwarp();
        const uint8_t *rec_s = V.recb + buf * 16 * NV;
        const long long c0 = top - V.pofs[buf];  // children of the parents above this one
        int fn = 0;
        if (lane == 0) fn = (int)atomicAdd(next_f, 1ull);
        fn = __shfl_sync(0xffffffffu, fn, 0);
        if (fn < np) fam_fetch<NV>(ws, S, stride, fn, lane, V.recb + (buf ^ 1) * 16 * NV, V.pofs + (buf ^ 1));
        const int pair_next = (LRN && fn < np && lane < L.K) ? __ldg(ws.topk + (long long)fn * L.K + lane) : 0;
        fam_bound<MT, NV, LRN, HEADS, BIDIR>(V, rec_s, c0, n, mp, stride, ub_iter, ws.children, ws.lbs,
                                             &ws.ctl->best_key, pair, L.K, nullptr, fc);
        __syncwarp();
        f = fn;
        pair = pair_next;
        buf ^= 1;
    }
    pdl_launch_dependents();  // no parent left: the elimination may be scheduled
    if (lane == 0) {
        for (int q = 0; q < 3; ++q)
            if (fc[q]) atomicAdd(reinterpret_cast<unsigned long long *>(&ws.ctl->fam[q]), (unsigned long long)fc[q]);
        if (fc[3]) atomicAdd(reinterpret_cast<unsigned long long *>(&ws.ctl->early), (unsigned long long)fc[3]);
    }
}

BranchFamilyFn pick_branch_family(int mt, int nv, bool learned, bool heads, bool bidir)
{
#define FSP_CASEF(MT_, NV_)                                                                                  \
    if (mt == MT_ && nv == NV_) {                                                                            \
        if (bidir) return (learned || heads) ? nullptr : &k_branch_family<MT_, NV_, false, false, true>;    \
        return learned ? (heads ? &k_branch_family<MT_, NV_, true, true, false>                              \
                                : &k_branch_family<MT_, NV_, true, false, false>)                            \
                       : (heads ? &k_branch_family<MT_, NV_, false, true, false>                             \
                                : &k_branch_family<MT_, NV_, false, false, false>);                          \
    }
    FSP_SHAPES_FAMILY(FSP_CASEF)
#undef FSP_CASEF
    return nullptr;
}

// Small pools of arbitrary nodes (fsp_bound_pool): one warp per node, so a
// pool too small to fill the GPU with one node per thread is not paced by
// one thread's serial work.  Lanes own machines for the node's release
// times (the diagonal recurrence), remaining sums and smallest tails, and
// machine pairs for the forward scans; the node bound is the warp's maximum.
// The same integers as the per-node kernels; a malformed record gives
// FSP_LB_INVALID and sets the instance's status bit 1.
template <int MT, int NV>
__global__ void __launch_bounds__(FAM_MAX_WARPS * 32, 1) k_bound_pool_warp(DevInst I, const uint8_t *__restrict__ nodes,
                                                                            long long count, int32_t *__restrict__ lb_out,
                                                                            FamSmem L)
{
    constexpr int P = MT * (MT - 1) / 2;
    constexpr int NS = (P + 31) / 32;
    typedef typename FamMask<NV>::type Mask;
    const int W = blockDim.x >> 5;
    if ((long long)blockIdx.x * W >= count) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = I.n, stride = I.stride, mp = I.mp;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const FamView V = fam_view(smem, L, warp);
    for (int i = threadIdx.x; i < n * P; i += blockDim.x) V.we[i] = __ldg(I.we + i);
    for (int i = threadIdx.x; i < P * V.rks8; i += blockDim.x) {
        const int kl = i / V.rks8, j = i - kl * V.rks8;
        V.rk8[i] = j < n ? __ldg(I.rank + kl * n + j) : (uint8_t)0;
    }
    for (int i = threadIdx.x; i < n * MT; i += blockDim.x) {
        const int j = i / MT, k = i - j * MT;
        V.pq[j * mp + k] = make_int2(__ldg(I.p + i), __ldg(I.q + i));
    }
    fam_tables_finish<MT>(V, n, mp);
    uint8_t *rec_s = V.recb;
    int32_t *Cs = V.cc, *SQs = V.sq;  // the node's release times and S + qmin per machine
    for (long long t = (long long)blockIdx.x * W + warp; t < count; t += (long long)gridDim.x * W) {
        if (lane < NV)
            reinterpret_cast<uint4 *>(rec_s)[lane] = __ldg(reinterpret_cast<const uint4 *>(nodes + t * stride) + lane);
        __syncwarp();
        int bad = 0;
        if (lane == 0) {  // a permutation of 0..n-1 and a depth <= n
            unsigned long long seen = 0ull;
            bad = rec_s[n] > n;
            for (int i = 0; i < n; ++i) {
                const int j = rec_s[i];
                if (j >= n || ((seen >> j) & 1ull)) bad = 1;
                else seen |= 1ull << j;
            }
        }
        bad = __shfl_sync(0xffffffffu, bad, 0);
        if (bad) {
            if (lane == 0) {
                lb_out[t] = FSP_LB_INVALID;
                atomicOr(I.status, 1);
            }
            __syncwarp();
            continue;
        }
        const int d = rec_s[n];
        const int k = lane < MT ? lane : MT - 1;
        int32_t Sk = 0, Qk = 0x7fffffff, Pk = 0x7fffffff;
        for (int i = d; i < n; ++i) {
            const int2 v = V.pq[rec_s[i] * mp + k];
            Sk += v.x;
            Qk = min(Qk, v.y);
            Pk = min(Pk, v.x);
        }
        int32_t Ck = 0;
        if (d > 0) {
            int32_t p0 = fam_prefix_p(0, lane, d, k, mp, rec_s, V.pq);
            int32_t p1 = fam_prefix_p(1, lane, d, k, mp, rec_s, V.pq);
            for (int s = 0; s < d + MT - 1; ++s) {
                const int32_t p2 = fam_prefix_p(s + 2, lane, d, k, mp, rec_s, V.pq);
                int32_t up = __shfl_up_sync(0xffffffffu, Ck, 1);
                if (lane == 0) up = 0;
                const int i = s - lane;
                if (lane < MT && i >= 0 && i < d) Ck = max(Ck, up) + p0;
                p0 = p1;
                p1 = p2;
            }
        }
        if (I.var == FSP_BOUND_HEADS && d < n) {
            // R_k = max(C_k, R_{k-1} + min over the remaining set of p[j][k-1])
            for (int kk = 1; kk < MT; ++kk) {
                const int32_t r_prev = __shfl_sync(0xffffffffu, Ck, kk - 1);
                const int32_t p_prev = __shfl_sync(0xffffffffu, Pk, kk - 1);
                if (lane == kk) Ck = max(Ck, r_prev + p_prev);
            }
        }
        const int32_t SQk = Sk + (Qk == 0x7fffffff ? 0 : Qk);
        if (lane < MT) {
            Cs[lane] = Ck;
            SQs[lane] = SQk;
        }
        __syncwarp();
        int32_t best = lane < MT ? Ck + SQk : 0;
        // the pairs: forward scans over the remaining set
        int klc[NS];
        Mask pm[NS];
        int32_t M[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            klc[s] = min(lane + 32 * s, P - 1);
            pm[s] = 0;
            M[s] = FSP_NEG;
        }
        for (int i = d; i < n; ++i) {
            const int j = rec_s[i];
#pragma unroll
            for (int s = 0; s < NS; ++s) pm[s] |= (Mask)1 << V.rk8[klc[s] * V.rks8 + j];
        }
        // each order from the back, one add-max per member: M <- max(M + e, w)
        Mask bit = (Mask)1 << (n - 1);
#pragma unroll 2
        for (int pos = n - 1; pos >= 0; --pos, bit >>= 1) {
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const int2 v = V.we[pos * P + klc[s]];
                if (pm[s] & bit) M[s] = __viaddmax_s32(M[s], v.y, v.x);
            }
        }
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const int km = V.klm[klc[s]];
            const int kk = km & 255, l = km >> 8;
            const int32_t v = __viaddmax_s32(SQs[l], __viaddmax_s32(Cs[kk], M[s], Cs[l]), best);
            if (lane + 32 * s < P) best = v;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
        if (lane == 0) lb_out[t] = best;
        __syncwarp();
    }
}

// Launch the warp-per-node bound on a pool of count nodes, if this shape has
// the kernel and its tables fit; returns FSP_ERR_ARG otherwise (the caller
// then uses the per-node kernels).
int fam_bound_pool(fsp_instance *I, int mt, int nv, const uint8_t *nodes, long long count, int32_t *lb_out,
                   cudaStream_t st)
{
    typedef void (*Fn)(DevInst, const uint8_t *, long long, int32_t *, FamSmem);
    Fn fn = nullptr;
#define FSP_CASEP(MT_, NV_) \
    if (mt == MT_ && nv == NV_) fn = &k_bound_pool_warp<MT_, NV_>;
    FSP_SHAPES_FAMILY(FSP_CASEP)
#undef FSP_CASEP
    const int w = fn ? family_warps(I, mt, nv) : 0;
    if (!fn || w == 0) return FSP_ERR_ARG;
    const FamSmem L = family_smem_layout(I, mt, nv, w);
    int rc = fsp_allow_smem(I, (const void *)fn, L.bytes);
    if (rc != FSP_OK) return rc;
    long long grid = (count + w - 1) / w;
    if (grid > I->sm_count) grid = I->sm_count;
    fn<<<(unsigned)grid, w * 32, L.bytes, st>>>(dev_view(I), nodes, count, lb_out, L);
    FSP_CUDA(cudaGetLastError());
    return FSP_OK;
}

// Warps per CTA that fit (the most up to FAM_MAX_WARPS); 0 if fewer than
// FAM_MIN_WARPS fit, and the per-child kernel is used instead.
int family_warps(const fsp_instance *I, int MT, int NV)
{
    for (int w = FAM_MAX_WARPS; w >= FAM_MIN_WARPS; --w)
        if ((long long)family_smem_layout(I, MT, NV, w).bytes <= I->smem_optin) return w;
    return 0;
}
