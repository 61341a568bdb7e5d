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

// Row stride (elements) of a byte table covering n columns, with an odd
// number of 32-bit words so that rows read by consecutive lanes fall in
// distinct banks.
static int odd_word_stride(int n, int per_word)
{
    int w = (n + per_word - 1) / per_word;
    if ((w & 1) == 0) ++w;
    return w * per_word;
}

FamSmem family_smem_layout(const fsp_instance *I, int MT, int NV, int warps)
{
    FamSmem L;
    const int n = I->n, P = I->P;
    L.rks8 = odd_word_stride(n, 4);
    L.mtp = MT | 1;
    size_t o = 0;
    L.we_off = o; o += fsp_align16((size_t)n * P * 8);
    L.rk8_off = o; o += fsp_align16((size_t)P * L.rks8);
    L.en_off = o; o += fsp_align16((size_t)n * P * 2);
    L.gam_off = o; o += fsp_align16((size_t)P * 4);
    L.klm_off = o; o += fsp_align16((size_t)P * 2);
    L.pq_off = o; o += fsp_align16((size_t)n * I->mp * 8);
    L.warp_off = o;
    size_t w = 0;
    L.w_ps = w; w += (size_t)MT * 16;
    L.w_psa = w; w += fsp_align16((size_t)MT * 4);
    L.w_ab = w; w += fsp_align16((size_t)MT * 8);
    L.w_rec = w; w += 32 * (size_t)NV;
    L.w_pofs = w; w += 16;
    L.w_cc = w; w += fsp_align16((size_t)n * L.mtp * 4);  // a family has at most n children
    L.w_sq = w; w += fsp_align16((size_t)n * L.mtp * 4);
    L.w_lb = w; w += fsp_align16((size_t)n * 4);
    L.w_T = w; w += fsp_align16((size_t)n * FAM_TS * 4);
    L.w_lkl = w; w += fsp_align16((size_t)P * 2);
    L.w_lm = w; w += fsp_align16((size_t)P * 4);
    L.warp_bytes = w;
    L.warps = warps;
    L.K = 0;
    L.bytes = o + w * warps;
    return L;
}

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

// Record of the child of parent `par` (depth d) that appends its remaining
// job of rank ci, c: the bytes in (d, d + ci] are the parent's shifted up by
// one, byte d is c and the depth byte n grows by one; word by word with
// funnel shifts, so no byte of the record is indexed at run time.
template <int NV>
__device__ __forceinline__ void fam_make_child(const FspRec<NV> &par, int n, int d, int ci, int c, FspRec<NV> &ch)
{
#pragma unroll
    for (int q = 0; q < 4 * NV; ++q) {
        const uint32_t w = par.w[q];
        const uint32_t sh = __funnelshift_l(q > 0 ? par.w[q - 1] : 0u, w, 8);
        const int lo = min(max(d + 1 - 4 * q, 0), 4), hi = min(max(d + ci + 1 - 4 * q, 0), 4);
        const uint32_t mlo = lo >= 4 ? 0xFFFFFFFFu : (1u << (8 * lo)) - 1u;
        const uint32_t mhi = hi >= 4 ? 0xFFFFFFFFu : (1u << (8 * hi)) - 1u;
        const uint32_t m = mhi & ~mlo;
        uint32_t x = (w & ~m) | (sh & m);
        const int bd = d - 4 * q;
        if (bd >= 0 && bd < 4) x = (x & ~(0xFFu << (8 * bd))) | ((uint32_t)c << (8 * bd));
        if ((n >> 2) == q) x += 1u << (8 * (n & 3));
        ch.w[q] = x;
    }
}

// p[job at prefix position t - lane][k], or 0 outside the prefix
__device__ __forceinline__ int32_t fam_prefix_p(int t, int lane, int d, int k, int mp,
                                                const uint8_t *__restrict__ rec_s, const int2 *__restrict__ pq_s)
{
    const int i = t - lane;
    const bool on = i >= 0 && i < d;
    return on ? pq_s[rec_s[on ? i : 0] * mp + k].x : 0;
}

// LRN: the learned order.  Children whose LB1 reaches the iteration's UB are
// cut at once; the parent's K predicted pairs (ws.topk) then give each open
// child a lower bound from their forward scans and cut more; only if a
// child is left do the certification and the remaining pairs run, for the
// children left.  A cut child keeps its partial bound (>= the UB); the
// others get the exact bound, so the search is the plain one.
template <int MT, int NV, bool LRN>
__global__ void __launch_bounds__(FAM_MAX_WARPS * 32, 1) k_branch_family(DevInst I, SolveWs ws, FamSmem L)
{
    constexpr int P = MT * (MT - 1) / 2;
    constexpr int NS = (P + 31) / 32;
    typedef typename FamMask<NV>::type Mask;
    const SolveCtl *ctl = ws.ctl;
    const int np = (int)ctl->n_parents;
    const int W = blockDim.x >> 5;
    if (blockIdx.x * W >= np) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = I.n, stride = I.stride, mp = I.mp;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int rks8 = L.rks8, mtp = L.mtp;
    int2 *we_s = reinterpret_cast<int2 *>(smem + L.we_off);
    uint8_t *rk8 = smem + L.rk8_off;
    uint16_t *en_s = reinterpret_cast<uint16_t *>(smem + L.en_off);
    int32_t *gam_s = reinterpret_cast<int32_t *>(smem + L.gam_off);
    uint16_t *klm_s = reinterpret_cast<uint16_t *>(smem + L.klm_off);
    int2 *pq_s = reinterpret_cast<int2 *>(smem + L.pq_off);
    unsigned char *wb = smem + L.warp_off + warp * L.warp_bytes;
    int4 *ps = reinterpret_cast<int4 *>(wb + L.w_ps);
    int32_t *psa = reinterpret_cast<int32_t *>(wb + L.w_psa);
    int32_t *ab = reinterpret_cast<int32_t *>(wb + L.w_ab);  // alpha[MT], beta[MT]
    uint8_t *recb = wb + L.w_rec;
    int *pofs = reinterpret_cast<int *>(wb + L.w_pofs);
    int32_t *cc = reinterpret_cast<int32_t *>(wb + L.w_cc);
    int32_t *sq = reinterpret_cast<int32_t *>(wb + L.w_sq);
    int32_t *lbv = reinterpret_cast<int32_t *>(wb + L.w_lb);
    int32_t *T = reinterpret_cast<int32_t *>(wb + L.w_T);
    uint16_t *lkl = reinterpret_cast<uint16_t *>(wb + L.w_lkl);
    int32_t *lm = reinterpret_cast<int32_t *>(wb + L.w_lm);

    // stage the instance tables
    for (int i = threadIdx.x; i < n * P; i += blockDim.x) we_s[i] = __ldg(I.we + i);
    for (int i = threadIdx.x; i < P * rks8; i += blockDim.x) {
        const int kl = i / rks8, j = i - kl * rks8;
        rk8[i] = j < n ? __ldg(I.rank + kl * n + j) : (uint8_t)0;
    }
    for (int kl = threadIdx.x; kl < P; kl += blockDim.x) {
        int k = 0, rem = kl;
        while (rem >= MT - 1 - k) { rem -= MT - 1 - k; ++k; }
        klm_s[kl] = (uint16_t)(k | ((k + 1 + rem) << 8));
    }
    for (int i = threadIdx.x; i < n * MT; i += blockDim.x) {
        const int j = i / MT, k = i - j * MT;
        pq_s[j * mp + k] = make_int2(__ldg(I.p + i), __ldg(I.q + i));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n * P; i += blockDim.x) {  // max(0, -e) = max(0, b - a)
        const int j = i / P, kl = i - j * P;
        const int km = klm_s[kl];
        en_s[i] = (uint16_t)max(0, pq_s[j * mp + (km >> 8)].x - pq_s[j * mp + (km & 255)].x);
    }
    __syncthreads();
    for (int kl = threadIdx.x; kl < P; kl += blockDim.x) {
        int g = 0;
        for (int j = 0; j < n; ++j) g = max(g, (int)en_s[j * P + kl]);
        gam_s[kl] = g;
    }
    __syncthreads();

    const long long S = ctl->s_pop + np;
    const int ub_iter = ctl->ub_iter;
    // parents are taken from a shared counter one ahead: the next one's
    // record is copied into the other buffer while this one is processed
    unsigned long long *next_f = reinterpret_cast<unsigned long long *>(&ws.ctl->fam_next);
    int f = 0, buf = 0;
    if (lane == 0) f = (int)atomicAdd(next_f, 1ull);
    f = __shfl_sync(0xffffffffu, f, 0);
    if (f < np) fam_fetch<NV>(ws, S, stride, f, lane, recb, pofs);
    while (f < np) {
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        __syncwarp();
        const uint8_t *rec_s = recb + buf * 16 * NV;
        FspRec<NV> par;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const uint4 x = reinterpret_cast<const uint4 *>(rec_s)[v];
            par.w[4 * v + 0] = x.x;
            par.w[4 * v + 1] = x.y;
            par.w[4 * v + 2] = x.z;
            par.w[4 * v + 3] = x.w;
        }
        const long long c0 = pofs[buf];
        int fn = 0;
        if (lane == 0) fn = (int)atomicAdd(next_f, 1ull);
        fn = __shfl_sync(0xffffffffu, fn, 0);
        if (fn < np) fam_fetch<NV>(ws, S, stride, fn, lane, recb + (buf ^ 1) * 16 * NV, pofs + (buf ^ 1));
        const int d = rec_s[n];
        const int r = n - d;

        // -- parent state on machine k = lane: remaining sum, smallest and
        // second smallest tail (and a job attaining the smallest), release time
        {
            const int k = lane < MT ? lane : MT - 1;
            int32_t Sk = 0, Q1 = 0x7fffffff, Q2 = 0x7fffffff, A = 0;
            for (int i = d; i < n; ++i) {
                const int j = rec_s[i];
                const int2 v = pq_s[j * mp + k];
                Sk += v.x;
                if (v.y < Q1) { Q2 = Q1; Q1 = v.y; A = j; }
                else Q2 = min(Q2, v.y);
            }
            // release times: lane k takes prefix position t - k at step t,
            // after lane k-1 has finished that position on machine k-1 (the
            // p values are read two steps ahead of their use)
            int32_t Ck = 0;
            if (d > 0) {
                int32_t p0 = fam_prefix_p(0, lane, d, k, mp, rec_s, pq_s);
                int32_t p1 = fam_prefix_p(1, lane, d, k, mp, rec_s, pq_s);
                for (int t = 0; t < d + MT - 1; ++t) {
                    const int32_t p2 = fam_prefix_p(t + 2, lane, d, k, mp, rec_s, pq_s);
                    int32_t up = __shfl_up_sync(0xffffffffu, Ck, 1);
                    if (lane == 0) up = 0;
                    const int i = t - lane;
                    if (lane < MT && i >= 0 && i < d) Ck = max(Ck, up) + p0;
                    p0 = p1;
                    p1 = p2;
                }
            }
            if (lane < MT) {
                ps[lane] = make_int4(Ck, Sk, Q1, Q2);
                psa[lane] = A;
            }
        }
        __syncwarp();

        // -- each lane a child: its record, release times, S + qmin, LB1
        for (int ci = lane; ci < r; ci += 32) {
            const int c = rec_s[d + ci];
            const int2 *prow = pq_s + c * mp;
            int32_t lb = 0, prev = 0;
#pragma unroll
            for (int k = 0; k < MT; ++k) {
                const int4 st = ps[k];
                const int2 v = prow[k];
                const int32_t ck = max(st.x, prev) + v.x;
                const int32_t sqk = st.y - v.x + (psa[k] == c ? st.w : st.z);
                prev = ck;
                cc[ci * mtp + k] = ck;
                sq[ci * mtp + k] = sqk;
                lb = max(lb, ck + sqk);
            }
            lbv[ci] = lb;
            FspRec<NV> ch;
            fam_make_child<NV>(par, n, d, ci, c, ch);
            fsp_store_rec(ch, ws.children + (c0 + ci) * stride);
        }
        __syncwarp();

        // exact terms of the listed pairs, 32 at a time: forward and backward
        // scans into T (one column per pair), then the lookups of the
        // children still open
        auto exact_pairs = [&](int cnt_all) {
            for (int b0 = 0; b0 < cnt_all; b0 += 32) {
                const int cnt = min(32, cnt_all - b0);
                if (lane < cnt) {
                    const int kl = lkl[b0 + lane];
                    Mask pm = 0;
#pragma unroll 4
                    for (int i = d; i < n; ++i) pm |= (Mask)1 << rk8[kl * rks8 + rec_s[i]];
                    int32_t E = 0, M = FSP_NEG;
                    Mask pf = pm;
#pragma unroll 2
                    for (int pos = 0; pos < n; ++pos) {
                        const int2 v = we_s[pos * P + kl];
                        const bool b = pf & 1u;
                        pf >>= 1;
                        T[pos * FAM_TS + lane] = M;
                        M = __viaddmax_s32(E, b ? v.x : FSP_NEG, M);
                        E += b ? v.y : 0;
                    }
                    int32_t R = E, Ms = FSP_NEG;
#pragma unroll 2
                    for (int pos = n - 1; pos >= 0; --pos) {
                        const int2 v = we_s[pos * P + kl];
                        const bool b = (pm >> pos) & 1u;
                        int32_t *t = T + pos * FAM_TS + lane;
                        *t = max(*t, Ms - v.y);
                        R -= b ? v.y : 0;
                        Ms = __viaddmax_s32(R, b ? v.x : FSP_NEG, Ms);
                    }
                }
                __syncwarp();
                for (int ci = lane; ci < r; ci += 32) {
                    int32_t lb = lbv[ci];
                    if (LRN && lb >= ub_iter) continue;
                    const int c = rec_s[d + ci];
                    const int32_t *cr = cc + ci * mtp, *sr = sq + ci * mtp;
#pragma unroll 4
                    for (int s = 0; s < cnt; ++s) {
                        const int kl = lkl[b0 + s];
                        const int km = klm_s[kl];
                        const int k = km & 255, l = km >> 8;
                        const int32_t X = T[rk8[kl * rks8 + c] * FAM_TS + s];
                        lb = __viaddmax_s32(sr[l], __viaddmax_s32(cr[k], X, cr[l]), lb);
                    }
                    lbv[ci] = lb;
                }
                __syncwarp();
            }
        };
        // lower bounds from the forward scan alone of the listed pairs (at most
        // 32): X_c >= the prefix maximum before c, so SQ_l + max(C_l, C_k +
        // prefix max) is a bound no larger than the pair's value
        auto forward_pairs = [&](int cnt) {
            if (lane < cnt) {
                const int kl = lkl[lane];
                Mask pm = 0;
#pragma unroll 4
                for (int i = d; i < n; ++i) pm |= (Mask)1 << rk8[kl * rks8 + rec_s[i]];
                int32_t E = 0, M = FSP_NEG;
#pragma unroll 2
                for (int pos = 0; pos < n; ++pos) {
                    const int2 v = we_s[pos * P + kl];
                    const bool b = pm & 1u;
                    pm >>= 1;
                    T[pos * FAM_TS + lane] = M;
                    M = __viaddmax_s32(E, b ? v.x : FSP_NEG, M);
                    E += b ? v.y : 0;
                }
            }
            __syncwarp();
            for (int ci = lane; ci < r; ci += 32) {
                int32_t lb = lbv[ci];
                if (lb >= ub_iter) continue;
                const int c = rec_s[d + ci];
                const int32_t *cr = cc + ci * mtp, *sr = sq + ci * mtp;
                for (int s = 0; s < cnt; ++s) {
                    const int kl = lkl[s];
                    const int km = klm_s[kl];
                    const int k = km & 255, l = km >> 8;
                    const int32_t X = T[rk8[kl * rks8 + c] * FAM_TS + s];
                    lb = __viaddmax_s32(sr[l], __viaddmax_s32(cr[k], X, cr[l]), lb);
                }
                lbv[ci] = lb;
            }
            __syncwarp();
        };
        // children still open (all of them in the plain order)
        auto open_any = [&]() {
            bool any = false;
            for (int ci = lane; ci < r; ci += 32) any |= lbv[ci] < ub_iter;
            return __any_sync(0xffffffffu, any);
        };

        const bool leaves = d + 1 == n - 1;
        bool open = !leaves;
        if (LRN) {
            if (open) open = open_any();
            if (open) {  // the parent's predicted pairs
                if (lane < L.K) lkl[lane] = (uint16_t)ws.topk[(long long)f * L.K + lane];
                __syncwarp();
                forward_pairs(L.K);
                open = open_any();
            }
            int cut = 0;
            for (int ci = lane; ci < r; ci += 32) cut += lbv[ci] >= ub_iter;
            cut = __reduce_add_sync(0xffffffffu, cut);
            if (lane == 0 && cut) atomicAdd(reinterpret_cast<unsigned long long *>(&ws.ctl->early), (unsigned long long)cut);
        }
        if (open) {
            // -- per machine: alpha_k = min_c (LB1 - C_k), beta_l = max_c SQ_l
            if (lane < MT) {
                int32_t a = 0x7fffffff, b = -0x7fffffff;
#pragma unroll 4
                for (int ci = 0; ci < r; ++ci) {
                    if (LRN && lbv[ci] >= ub_iter) continue;  // cut already
                    a = min(a, lbv[ci] - cc[ci * mtp + lane]);
                    b = max(b, sq[ci * mtp + lane]);
                }
                ab[lane] = a;
                ab[MT + lane] = b;
            }
            __syncwarp();

            // -- forward scan of every pair over U (its full-set term M_U);
            // pairs failing the O(1) test M_U + gam <= alpha_k - beta_l are listed
            int n1 = 0;
            {
                int klc[NS];
                Mask pm[NS];
                int32_t E[NS], M[NS];
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    klc[s] = min(lane + 32 * s, P - 1);
                    pm[s] = 0;
                    E[s] = 0;
                    M[s] = FSP_NEG;
                }
#pragma unroll 4
                for (int i = d; i < n; ++i) {
                    const int j = rec_s[i];
#pragma unroll
                    for (int s = 0; s < NS; ++s) pm[s] |= (Mask)1 << rk8[klc[s] * rks8 + j];
                }
                const int2 *wrow = we_s;
#pragma unroll 2
                for (int pos = 0; pos < n; ++pos, wrow += P) {
#pragma unroll
                    for (int s = 0; s < NS; ++s) {
                        const int2 v = wrow[klc[s]];
                        const bool b = pm[s] & 1u;
                        pm[s] >>= 1;
                        M[s] = __viaddmax_s32(E[s], b ? v.x : FSP_NEG, M[s]);
                        E[s] += b ? v.y : 0;
                    }
                }
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    const int kl = lane + 32 * s;
                    const int km = klm_s[klc[s]];
                    const bool fail = kl < P && M[s] > ab[km & 255] - ab[MT + (km >> 8)] - gam_s[klc[s]];
                    const unsigned msk = __ballot_sync(0xffffffffu, fail);
                    if (fail) {
                        const int at = n1 + __popc(msk & lt_mask);
                        lkl[at] = (uint16_t)kl;
                        lm[at] = M[s];
                    }
                    n1 += __popc(msk);
                }
            }
            __syncwarp();

            // -- the listed pairs child by child: M_U + max(0, -e_c) + SQ_l(c)
            // + C_k(c) <= LB1(c); the pairs that fail stay listed (in place)
            int n2 = 0;
            for (int b0 = 0; b0 < n1; b0 += 32) {
                const int e = b0 + lane;
                const bool valid = e < n1;
                const int kl = valid ? lkl[e] : 0;
                const int32_t Mu = valid ? lm[e] : 0;
                const int km = klm_s[kl];
                const int k = km & 255, l = km >> 8;
                bool ok = true;
                if (valid) {
#pragma unroll 4
                    for (int ci = 0; ci < r; ++ci) {
                        const int c = rec_s[d + ci];
                        const int32_t lbc = lbv[ci];
                        ok &= (LRN && lbc >= ub_iter) ||
                              Mu + (int)en_s[c * P + kl] + sq[ci * mtp + l] <= lbc - cc[ci * mtp + k];
                    }
                }
                const bool fail = valid && !ok;
                __syncwarp();
                const unsigned msk = __ballot_sync(0xffffffffu, fail);
                if (fail) lkl[n2 + __popc(msk & lt_mask)] = (uint16_t)kl;
                n2 += __popc(msk);
            }
            __syncwarp();

            exact_pairs(n2);
        }

        // -- the bounds; a depth n-1 child is a complete schedule
        for (int ci = lane; ci < r; ci += 32) {
            const long long cidx = c0 + ci;
            const int32_t lb = lbv[ci];
            ws.lbs[cidx] = lb;
            if (leaves && lb < ub_iter)
                atomicMin(&ws.ctl->best_key, ((unsigned long long)(uint32_t)lb << 32) | (unsigned long long)cidx);
        }
        __syncwarp();
        f = fn;
        buf ^= 1;
    }
}

BranchFamilyFn pick_branch_family(int mt, int nv, bool learned)
{
#define FSP_CASEF(MT_, NV_) \
    if (mt == MT_ && nv == NV_) return learned ? &k_branch_family<MT_, NV_, true> : &k_branch_family<MT_, NV_, false>;
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
