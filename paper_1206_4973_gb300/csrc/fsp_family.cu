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
// of its first child's index (lane NV) into this warp's buffers.
template <int NV>
__device__ __forceinline__ void fam_fetch(const SolveWs &ws, long long S, int stride, int f, int lane,
                                          uint8_t *rec_dst, int *poff_dst)
{
    if (lane < NV) {
        const unsigned d = (unsigned)__cvta_generic_to_shared(rec_dst + lane * 16);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d),
                     "l"(ws.stack + (S - 1 - f) * stride + lane * 16));
    } else if (lane == NV) {
        const unsigned d = (unsigned)__cvta_generic_to_shared(poff_dst);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(ws.poff + f));
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int MT, int NV, bool LRN, bool HEADS>
__global__ void __launch_bounds__(FAM_MAX_WARPS * 32, 1) k_branch_family(DevInst I, SolveWs ws, FamSmem L)
{
    constexpr int P = MT * (MT - 1) / 2;
    const SolveCtl *ctl = ws.ctl;
    const int np = (int)ctl->n_parents;
    const int W = blockDim.x >> 5;
    if (blockIdx.x * W >= np) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = I.n, stride = I.stride, mp = I.mp;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const FamView V = fam_view(smem, L, warp);

    // stage the instance tables
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

    const long long S = ctl->s_pop + np;
    const int ub_iter = ctl->ub_iter;
    // parents are taken from a shared counter one ahead: the next one's
    // record is copied into the other buffer while this one is processed
    unsigned long long *next_f = reinterpret_cast<unsigned long long *>(&ws.ctl->fam_next);
    int f = 0, buf = 0;
    if (lane == 0) f = (int)atomicAdd(next_f, 1ull);
    f = __shfl_sync(0xffffffffu, f, 0);
    if (f < np) fam_fetch<NV>(ws, S, stride, f, lane, V.recb, V.pofs);
    while (f < np) {
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        __syncwarp();
        const uint8_t *rec_s = V.recb + buf * 16 * NV;
        const long long c0 = V.pofs[buf];
        int fn = 0;
        if (lane == 0) fn = (int)atomicAdd(next_f, 1ull);
        fn = __shfl_sync(0xffffffffu, fn, 0);
        if (fn < np) fam_fetch<NV>(ws, S, stride, fn, lane, V.recb + (buf ^ 1) * 16 * NV, V.pofs + (buf ^ 1));
        fam_bound<MT, NV, LRN, HEADS>(V, rec_s, c0, n, mp, stride, ub_iter, ws.children, ws.lbs,
                                      &ws.ctl->best_key, LRN ? ws.topk + (long long)f * L.K : nullptr, L.K,
                                      reinterpret_cast<unsigned long long *>(&ws.ctl->early));
        __syncwarp();
        f = fn;
        buf ^= 1;
    }
}

BranchFamilyFn pick_branch_family(int mt, int nv, bool learned, bool heads)
{
#define FSP_CASEF(MT_, NV_)                                                                          \
    if (mt == MT_ && nv == NV_)                                                                      \
        return learned ? (heads ? &k_branch_family<MT_, NV_, true, true> : &k_branch_family<MT_, NV_, true, false>) \
                       : (heads ? &k_branch_family<MT_, NV_, false, true> : &k_branch_family<MT_, NV_, false, false>);
    FSP_SHAPES_FAMILY(FSP_CASEF)
#undef FSP_CASEF
    return nullptr;
}

// Warps per CTA that fit (the most up to FAM_MAX_WARPS); 0 if fewer than
// FAM_MIN_WARPS fit, and the per-child kernel is used instead.
int family_warps(const fsp_instance *I, int MT, int NV)
{
    for (int w = FAM_MAX_WARPS; w >= FAM_MIN_WARPS; --w)
        if ((long long)family_smem_layout(I, MT, NV, w).bytes <= I->smem_optin) return w;
    return 0;
}
