// fsp_family.cuh -- bounding a parent's children together (the "family"
// bound, fsp_family.cu): layout, the per-warp view of the shared memory and
// the per-family device code shared by the search kernel and the batch
// solver (fsp_batch.cu).
#pragma once

#include <type_traits>

#include "fsp_solve.cuh"

#define FAM_MAX_WARPS 20  // warps per CTA at most (one parent per warp at a time)
#define FAM_MIN_WARPS 4   // below this the per-child kernel is used
#define FAM_TS 33         // row stride of the per-warp scan table (32 pairs + 1)

// Compiled shapes: machines MT x record vectors NV (n <= 16 NV - 1).
#define FSP_SHAPES_FAMILY(X) \
    X(5, 1) X(5, 2) X(5, 3) X(5, 4) X(10, 1) X(10, 2) X(10, 3) X(10, 4) X(20, 1) X(20, 2) X(20, 3) X(20, 4)

// Position masks: n <= 31 jobs fit 32 bits (records of up to 32 bytes).
template <int NV>
struct FamMask {
    typedef unsigned long long type;
};
template <>
struct FamMask<1> {
    typedef uint32_t type;
};
template <>
struct FamMask<2> {
    typedef uint32_t type;
};

// Shared memory of a family CTA.  Instance tables: the Johnson entries
// position-major (we), each job's position per pair (rk8), max(0, -e) per
// job and pair (en) and its maximum over the jobs (gam), each pair's
// machines (klm), the {p, q} rows (pq).  Then per warp (offsets w_*): the
// parent state, the record buffers, the children's release times, S + qmin
// and running bounds (rows of mtp words), the scan table T [n][FAM_TS] and
// the list of pairs still to evaluate.
struct FamSmem {
    size_t we_off, rk8_off, en_off, gam_off, klm_off, pq_off, warp_off, warp_bytes, bytes;
    size_t w_ps, w_psa, w_pp, w_ab, w_pd, w_rec, w_pofs, w_cc, w_sq, w_lb, w_T, w_lkl, w_lm;
    int rks8, mtp, warps;
    int K;  // learned order: predicted pairs per parent
};

// Row stride (elements) of a byte table covering n columns, with an odd
// number of 32-bit words so that rows read by consecutive lanes fall in
// distinct banks.
__host__ __device__ inline int odd_word_stride(int n, int per_word)
{
    int w = (n + per_word - 1) / per_word;
    if ((w & 1) == 0) ++w;
    return w * per_word;
}

__host__ __device__ inline FamSmem family_smem_layout_nm(int n, int m, int mp, int MT, int NV, int warps)
{
    FamSmem L;
    const int P = m * (m - 1) / 2;
    L.rks8 = odd_word_stride(n, 4);
    L.mtp = MT | 1;
    size_t o = 0;
    L.we_off = o; o += fsp_align16((size_t)n * P * 8);
    L.rk8_off = o; o += fsp_align16((size_t)P * L.rks8);
    L.en_off = o; o += fsp_align16((size_t)n * P * 2);
    L.gam_off = o; o += fsp_align16((size_t)P * 4);
    L.klm_off = o; o += fsp_align16((size_t)P * 2);
    L.pq_off = o; o += fsp_align16((size_t)n * mp * 8);
    L.warp_off = o;
    size_t w = 0;
    L.w_ps = w; w += (size_t)MT * 16;
    L.w_psa = w; w += fsp_align16((size_t)MT * 4);
    L.w_pp = w; w += (size_t)MT * 16;
    L.w_ab = w; w += fsp_align16((size_t)MT * 8);
    L.w_pd = w; w += fsp_align16((size_t)MT * 4);
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

static inline FamSmem family_smem_layout(const fsp_instance *I, int MT, int NV, int warps)
{
    return family_smem_layout_nm(I->n, I->m, I->mp, MT, NV, warps);
}

int family_warps(const fsp_instance *I, int MT, int NV);
int fam_bound_pool(fsp_instance *I, int mt, int nv, const uint8_t *nodes, long long count, int32_t *lb_out,
                   cudaStream_t st);
#define FAM_POOL_SMALL 16384  // fsp_bound_pool uses one warp per node up to this many nodes

typedef void (*BranchFamilyFn)(DevInst, SolveWs, FamSmem);
BranchFamilyFn pick_branch_family(int mt, int nv, bool learned, bool heads, bool bidir = false);

// One warp's view of the family shared memory.
struct FamView {
    int2 *we;
    uint8_t *rk8;
    uint16_t *en;
    int32_t *gam;
    uint16_t *klm;
    int2 *pq;
    int4 *ps, *pp;
    int32_t *psa, *ab, *pd, *cc, *sq, *lbv, *T, *lm;
    uint16_t *lkl;
    uint8_t *recb;
    long long *pofs;
    int rks8, mtp;
};

__device__ __forceinline__ FamView fam_view(unsigned char *smem, const FamSmem &L, int warp)
{
    FamView V;
    V.we = reinterpret_cast<int2 *>(smem + L.we_off);
    V.rk8 = smem + L.rk8_off;
    V.en = reinterpret_cast<uint16_t *>(smem + L.en_off);
    V.gam = reinterpret_cast<int32_t *>(smem + L.gam_off);
    V.klm = reinterpret_cast<uint16_t *>(smem + L.klm_off);
    V.pq = reinterpret_cast<int2 *>(smem + L.pq_off);
    unsigned char *wb = smem + L.warp_off + warp * L.warp_bytes;
    V.ps = reinterpret_cast<int4 *>(wb + L.w_ps);
    V.psa = reinterpret_cast<int32_t *>(wb + L.w_psa);
    V.pp = reinterpret_cast<int4 *>(wb + L.w_pp);  // heads variant: smallest p per machine
    V.ab = reinterpret_cast<int32_t *>(wb + L.w_ab);  // alpha[MT], beta[MT]
    V.pd = reinterpret_cast<int32_t *>(wb + L.w_pd);  // bidirectional: the suffix's delivery times
    V.recb = wb + L.w_rec;                            // two record buffers
    V.pofs = reinterpret_cast<long long *>(wb + L.w_pofs);  // and the running counts below them
    V.cc = reinterpret_cast<int32_t *>(wb + L.w_cc);
    V.sq = reinterpret_cast<int32_t *>(wb + L.w_sq);
    V.lbv = reinterpret_cast<int32_t *>(wb + L.w_lb);
    V.T = reinterpret_cast<int32_t *>(wb + L.w_T);
    V.lkl = reinterpret_cast<uint16_t *>(wb + L.w_lkl);
    V.lm = reinterpret_cast<int32_t *>(wb + L.w_lm);
    V.rks8 = L.rks8;
    V.mtp = L.mtp;
    return V;
}

// The tables derived from staged {p, q} rows: each pair's machines, max(0, -e)
// per job and pair and its maximum per pair.  All threads of the CTA call it.
template <int MT>
__device__ __forceinline__ void fam_tables_finish(const FamView &V, int n, int mp)
{
    constexpr int P = MT * (MT - 1) / 2;
    for (int kl = threadIdx.x; kl < P; kl += blockDim.x) {
        int k = 0, rem = kl;
        while (rem >= MT - 1 - k) { rem -= MT - 1 - k; ++k; }
        V.klm[kl] = (uint16_t)(k | ((k + 1 + rem) << 8));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n * P; i += blockDim.x) {  // max(0, -e) = max(0, b - a)
        const int j = i / P, kl = i - j * P;
        const int km = V.klm[kl];
        V.en[i] = (uint16_t)max(0, V.pq[j * mp + (km >> 8)].x - V.pq[j * mp + (km & 255)].x);
    }
    __syncthreads();
    for (int kl = threadIdx.x; kl < P; kl += blockDim.x) {
        int g = 0;
        for (int j = 0; j < n; ++j) g = max(g, (int)V.en[j * P + kl]);
        V.gam[kl] = g;
    }
    __syncthreads();
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

// Record of the child of a bidirectional parent (prefix d1, suffix starting
// at byte e = n - d2) that puts its remaining job of rank ci, c, in front of
// the suffix: the bytes in [d1 + ci, e - 1) are the parent's shifted down by
// one, byte e - 1 is c and the suffix length byte n + 1 grows by one.
template <int NV>
__device__ __forceinline__ void fam_make_child_back(const FspRec<NV> &par, int n, int d1, int e, int ci, int c,
                                                    FspRec<NV> &ch)
{
#pragma unroll
    for (int q = 0; q < 4 * NV; ++q) {
        const uint32_t w = par.w[q];
        const uint32_t sh = __funnelshift_r(w, q + 1 < 4 * NV ? par.w[q + 1] : 0u, 8);
        const int lo = min(max(d1 + ci - 4 * q, 0), 4), hi = min(max(e - 1 - 4 * q, 0), 4);
        const uint32_t mlo = lo >= 4 ? 0xFFFFFFFFu : (1u << (8 * lo)) - 1u;
        const uint32_t mhi = hi >= 4 ? 0xFFFFFFFFu : (1u << (8 * hi)) - 1u;
        const uint32_t m = mhi & ~mlo;
        uint32_t x = (w & ~m) | (sh & m);
        const int be = e - 1 - 4 * q;
        if (be >= 0 && be < 4) x = (x & ~(0xFFu << (8 * be))) | ((uint32_t)c << (8 * be));
        if (((n + 1) >> 2) == q) x += 1u << (8 * ((n + 1) & 3));
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

// The children of one parent, bounded by one warp.  rec_s: the parent record
// in this warp's shared memory; c0: the index of its first child; the child
// records go to children, their bounds to lbs, and a depth n-1 child below
// ub_iter to the atomic minimum *best_key = (bound << 32) | child index.
// LRN: the learned order (lane j < K holds the parent's j-th predicted pair
// in my_pair).  Children whose LB1 reaches the iteration's UB are
// cut at once; the parent's K predicted pairs (topk_row) then give each open
// child a lower bound from their forward scans and cut more; only if a
// child is left do the certification and the remaining pairs run, for the
// children left.  A cut child keeps its partial bound (>= the UB); the
// others get the exact bound, so the search is the plain one.
// BIDIR: bidirectional records (prefix d1 at byte n, suffix d2 at byte n+1,
// the remaining set between them); the family's direction is forward when
// d1 <= d2, else backward (its children put a job in front of the suffix).
// Both directions remove the same job c from the remaining set, so the pair
// terms X_c and the certification are those of the forward family; only the
// one-machine quantities differ: a forward child's release times advance by c
// and its tail after machine k is max(D_k, qmin_k) with the parent's delivery
// times D; a backward child keeps the parent's release times and its delivery
// times advance by c.  A child with one job left gets its completion's
// makespan, max_k (C''_k + D'_k) with C'' its release times after that job.
template <int MT, int NV, bool LRN, bool HEADS, bool BIDIR = false>
__device__ __forceinline__ void fam_bound(const FamView &V, const uint8_t *rec_s, long long c0, int n, int mp,
                                          int stride, int ub_iter, uint8_t *children, int32_t *lbs,
                                          unsigned long long *best_key, int my_pair, int K,
                                          unsigned long long *early, int (&fc)[4])
{
    constexpr int P = MT * (MT - 1) / 2;
    constexpr int NS = (P + 31) / 32;
    typedef typename FamMask<NV>::type Mask;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int rks8 = V.rks8, mtp = V.mtp;
    const int2 *we_s = V.we;
    const uint8_t *rk8 = V.rk8;
    const uint16_t *en_s = V.en;
    const int32_t *gam_s = V.gam;
    const uint16_t *klm_s = V.klm;
    const int2 *pq_s = V.pq;
    int4 *ps = V.ps, *pp = V.pp;
    constexpr bool heads = HEADS;  // FSP_BOUND_HEADS
    int32_t *psa = V.psa, *ab = V.ab, *cc = V.cc, *sq = V.sq, *lbv = V.lbv, *T = V.T, *lm = V.lm;
    uint16_t *lkl = V.lkl;
    FspRec<NV> par;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const uint4 x = reinterpret_cast<const uint4 *>(rec_s)[v];
        par.w[4 * v + 0] = x.x;
        par.w[4 * v + 1] = x.y;
        par.w[4 * v + 2] = x.z;
        par.w[4 * v + 3] = x.w;
    }
    const int d = rec_s[n];
    const int d2 = BIDIR ? rec_s[n + 1] : 0;
    const int e = n - d2;  // the remaining set: positions [d, e)
    const int r = e - d;
    const bool fwd = !BIDIR || d <= d2;
    int32_t *pd = V.pd;

        // -- parent state on machine k = lane: remaining sum, smallest and
        // second smallest tail (and a job attaining the smallest), release time
        {
            const int k = lane < MT ? lane : MT - 1;
            int32_t Sk = 0, Q1 = 0x7fffffff, Q2 = 0x7fffffff, A = 0;
            for (int i = d; i < e; ++i) {
                const int j = rec_s[i];
                const int2 v = pq_s[j * mp + k];
                Sk += v.x;
                if (v.y < Q1) { Q2 = Q1; Q1 = v.y; A = j; }
                else Q2 = min(Q2, v.y);
            }
            // release times: lane k takes prefix position t - k at step t,
            // after lane k-1 has finished that position on machine k-1.  With
            // 10 machines or more its p values are staged first in its own
            // column of the scan table (free until the pair scans; row i =
            // prefix position i, stride 32, so the lanes' reads of different
            // rows fall in distinct banks); with 5, where the prefix is long
            // against the wavefront's width, each step reads its own p value,
            // two steps ahead of its use (measured faster there)
            int32_t Ck = 0;
            if (MT < 10 && d > 0) {
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
            } else if (d > 0) {
                // four prefix jobs per round (one word of the record), all four
                // loads issued before the stores (the stores may alias them)
                for (int i0 = 0; i0 < d; i0 += 4) {
                    const uint32_t wj = *reinterpret_cast<const uint32_t *>(rec_s + i0);
                    int32_t v[4];
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int j = i0 + b < d ? (int)((wj >> (8 * b)) & 0xFFu) : 0;
                        v[b] = pq_s[j * mp + k].x;
                    }
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        if (i0 + b < d) T[32 * (i0 + b) + lane] = v[b];
                }
#pragma unroll 4
                for (int t = 0; t < d + MT - 1; ++t) {
                    int32_t up = __shfl_up_sync(0xffffffffu, Ck, 1);
                    if (lane == 0) up = 0;
                    const int i = t - lane;
                    if (lane < MT && i >= 0 && i < d) Ck = max(Ck, up) + T[32 * i + lane];
                }
            }
            if (lane < MT) {
                ps[lane] = make_int4(Ck, Sk, Q1, Q2);
                psa[lane] = A;
            }
            if (BIDIR) {
                // delivery times of the suffix: lane k takes the suffix job t - (MT-1-k)
                // from the last at step t, after lane k+1 has finished it on machine k+1
                // (the suffix's p values staged in the lane's column like the prefix's)
                int32_t Dk = 0;
                if (MT < 10) {
                    for (int t = 0; t < d2 + MT - 1; ++t) {
                        int32_t down = __shfl_down_sync(0xffffffffu, Dk, 1);
                        if (lane == MT - 1) down = 0;
                        const int si = t - (MT - 1 - lane);
                        if (lane < MT && si >= 0 && si < d2)
                            Dk = max(Dk, down) + pq_s[rec_s[n - 1 - si] * mp + k].x;
                    }
                } else {
                    for (int s0 = 0; s0 < d2; s0 += 4) {
                        int32_t v[4];
#pragma unroll
                        for (int b = 0; b < 4; ++b) v[b] = s0 + b < d2 ? pq_s[rec_s[n - 1 - s0 - b] * mp + k].x : 0;
#pragma unroll
                        for (int b = 0; b < 4; ++b)
                            if (s0 + b < d2) T[32 * (s0 + b) + lane] = v[b];
                    }
#pragma unroll 4
                    for (int t = 0; t < d2 + MT - 1; ++t) {
                        int32_t down = __shfl_down_sync(0xffffffffu, Dk, 1);
                        if (lane == MT - 1) down = 0;
                        const int si = t - (MT - 1 - lane);
                        if (lane < MT && si >= 0 && si < d2) Dk = max(Dk, down) + T[32 * si + lane];
                    }
                }
                if (lane < MT) pd[lane] = Dk;
            }
            if (heads) {  // smallest and second smallest p on machine k, and a job attaining it
                int32_t P1 = 0x7fffffff, P2 = 0x7fffffff, AP = 0;
                for (int i = d; i < e; ++i) {
                    const int j = rec_s[i];
                    const int32_t v = pq_s[j * mp + k].x;
                    if (v < P1) { P2 = P1; P1 = v; AP = j; }
                    else P2 = min(P2, v);
                }
                if (lane < MT) pp[lane] = make_int4(P1, P2, AP, 0);
            }
        }
        __syncwarp();

        // -- each lane a child: its record, release times, S + qmin, LB1
        for (int ci = lane; ci < r; ci += 32) {
            const int c = rec_s[d + ci];
            const int2 *prow = pq_s + c * mp;
            if (BIDIR) {
                int32_t lb = 0;
                // the child's delivery times: the parent's (forward), or advanced by
                // c from machine m-1 down (backward; parked in the child's sq row)
                int32_t *dc = fwd ? pd : sq + ci * mtp;
                if (!fwd) {
                    int32_t nxt = 0;
#pragma unroll
                    for (int k = MT - 1; k >= 0; --k) {
                        nxt = max(pd[k], nxt) + prow[k].x;
                        dc[k] = nxt;
                    }
                }
                int32_t prev = 0, cm = 0, best = 0;
                const int2 *jrow = pq_s + rec_s[d + (r == 2 ? 1 - ci : 0)] * mp;  // the last job (r == 2)
#pragma unroll
                for (int k = 0; k < MT; ++k) {
                    const int4 st = ps[k];
                    const int32_t px = prow[k].x;
                    const int32_t ck = fwd ? max(st.x, prev) + px : st.x;
                    prev = ck;
                    const int32_t dk = dc[k];
                    const int32_t qm = psa[k] == c ? st.w : st.z;  // smallest tail over U \ {c}
                    const int32_t sqk = st.y - px + max(dk, qm == 0x7fffffff ? 0 : qm);
                    cm = max(ck, cm) + jrow[k].x;  // one job left: its completion's release times
                    best = max(best, cm + dk);
                    cc[ci * mtp + k] = ck;
                    sq[ci * mtp + k] = sqk;
                    lb = max(lb, ck + sqk);
                }
                if (r == 2) lb = best;  // one job left: the makespan of the child's completion
                lbv[ci] = lb;
                FspRec<NV> ch;
                if (fwd) fam_make_child<NV>(par, n, d, ci, c, ch);
                else fam_make_child_back<NV>(par, n, d, e, ci, c, ch);
                fsp_store_rec(ch, children + (c0 + ci) * stride);
                continue;
            }
            int32_t lb = 0, prev = 0, rprev = 0;
#pragma unroll
            for (int k = 0; k < MT; ++k) {
                const int4 st = ps[k];
                const int2 v = prow[k];
                const int32_t ck = max(st.x, prev) + v.x;
                const int32_t sqk = st.y - v.x + (psa[k] == c ? st.w : st.z);
                prev = ck;
                // heads variant: the earliest start of a job of U \ {c} on machine k
                int32_t rk = ck;
                if (heads && k > 0) {
                    const int4 pk = pp[k - 1];
                    rk = max(ck, rprev + (pk.z == c ? pk.y : pk.x));
                }
                rprev = rk;
                cc[ci * mtp + k] = rk;
                sq[ci * mtp + k] = sqk;
                lb = max(lb, rk + sqk);
            }
            lbv[ci] = lb;
            FspRec<NV> ch;
            fam_make_child<NV>(par, n, d, ci, c, ch);
            fsp_store_rec(ch, children + (c0 + ci) * stride);
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
                    for (int i = d; i < e; ++i) pm |= (Mask)1 << rk8[kl * rks8 + rec_s[i]];
                    // every lane at the same position (position-major rows and
                    // the lane's own T column: no bank conflicts); a member
                    // updates the running values, T is read at members only.
                    // Forward: the prefix maximum before each position
                    int32_t E = 0, M = FSP_NEG;
                    Mask bit = 1;
#pragma unroll 2
                    for (int pos = 0; pos < n; ++pos, bit <<= 1) {
                        const int2 v = we_s[pos * P + kl];
                        T[pos * FAM_TS + lane] = M;
                        if (pm & bit) {
                            M = __viaddmax_s32(E, v.x, M);
                            E += v.y;
                        }
                    }
                    // backward: the suffix maximum after each position, less its e
                    int32_t R = E, Ms = FSP_NEG;
#pragma unroll 2
                    for (int pos = n - 1; pos >= 0; --pos) {
                        const int2 v = we_s[pos * P + kl];
                        int32_t *tp = T + pos * FAM_TS + lane;
                        *tp = max(*tp, Ms - v.y);
                        if ((pm >> pos) & 1u) {
                            R -= v.y;
                            Ms = __viaddmax_s32(R, v.x, Ms);
                        }
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
                for (int i = d; i < e; ++i) pm |= (Mask)1 << rk8[kl * rks8 + rec_s[i]];
                int32_t E = 0, M = FSP_NEG;
                Mask bit = 1;
#pragma unroll 2
                for (int pos = 0; pos < n; ++pos, bit <<= 1) {  // lanes in step: no bank conflicts
                    const int2 v = we_s[pos * P + kl];
                    T[pos * FAM_TS + lane] = M;
                    if (pm & bit) {
                        M = __viaddmax_s32(E, v.x, M);
                        E += v.y;
                    }
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

        const bool leaves = r == 2;  // the children have one job left: complete schedules
        bool open = !leaves;
        if (!leaves) {  // counted in every order: children all cut by their one-machine bounds
            const bool any = open_any();
            fc[0] += !any;
            if (LRN) open = any;
        }
        if (LRN) {
            if (open) {  // the parent's predicted pairs
                if (lane < K) lkl[lane] = (uint16_t)my_pair;
                __syncwarp();
                forward_pairs(K);
                open = open_any();
                fc[1] += !open;
            }
            int cut = 0;
            for (int ci = lane; ci < r; ci += 32) cut += lbv[ci] >= ub_iter;
            cut = __reduce_add_sync(0xffffffffu, cut);
            if (early) {
                if (lane == 0 && cut) atomicAdd(early, (unsigned long long)cut);
            } else {
                fc[3] += cut;  // added once per warp by the caller (one address for every family)
            }
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
                int32_t M[NS];
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    klc[s] = min(lane + 32 * s, P - 1);
                    pm[s] = 0;
                    M[s] = FSP_NEG;
                }
#pragma unroll 4
                for (int i = d; i < e; ++i) {
                    const int j = rec_s[i];
#pragma unroll
                    for (int s = 0; s < NS; ++s) pm[s] |= (Mask)1 << rk8[klc[s] * rks8 + j];
                }
                // M_U from the back of each order, one add-max per member:
                // G <- max(G + e_i, w_i) gives max_i (E_{<i} + w_i) at the
                // first; all lanes read the same position row (no bank conflicts)
                Mask bit = (Mask)1 << (n - 1);
                const int2 *wrow = we_s + (n - 1) * P;
#pragma unroll 2
                for (int pos = n - 1; pos >= 0; --pos, wrow -= P, bit >>= 1) {
#pragma unroll
                    for (int s = 0; s < NS; ++s) {
                        const int2 v = wrow[klc[s]];
                        if (pm[s] & bit) M[s] = __viaddmax_s32(M[s], v.y, v.x);
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

            fc[2] += n2;
            exact_pairs(n2);
        }

        // -- the bounds; a depth n-1 child is a complete schedule
        for (int ci = lane; ci < r; ci += 32) {
            const long long cidx = c0 + ci;
            const int32_t lb = lbv[ci];
            lbs[cidx] = lb;
            if (leaves && lb < ub_iter)
                atomicMin(best_key, ((unsigned long long)(uint32_t)lb << 32) | (unsigned long long)cidx);
        }
}
