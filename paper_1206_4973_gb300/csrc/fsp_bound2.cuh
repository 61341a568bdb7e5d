// fsp_bound2.cuh -- the node bound for the common shapes (n <= 63 jobs,
// m in {5, 10, 20} machines): registers instead of shared-memory columns
// wherever the index is static, two nodes per thread, and one fused
// add-max instruction per scan step.
//
// Per node the work is the same as fsp_node_bound (fsp_common.cuh): the
// prefix's release times, the remaining sums and smallest tails, the
// one-machine bounds, then for every machine pair the max-plus scan over the
// pair's Johnson order.  Differences that make it faster on sm_103a:
//   * the record is read straight into registers (16 * NV bytes);
//   * p and the tails sit in shared memory as {p, q} pairs with an odd row
//     stride, so lanes reading different jobs' rows hit different banks;
//   * the Johnson entries are staged in shared memory (every lane reads the
//     same entry: a broadcast; reading them through L1 instead stalled on
//     the longer load latency and was slower on sm_103a);
//   * NPT nodes per thread share every entry load;
//   * a scan step is LOP3 (membership) + VIADDMNMX (M = max(E + w, M)) +
//     IADD (E += e): the DPX add-max runs the add and the max as one op.
#pragma once

#include "fsp_common.cuh"

template <int NV>
struct FspRec {
    uint32_t w[4 * NV];
};

template <int NV>
__device__ __forceinline__ void fsp_load_rec(FspRec<NV> &r, const uint8_t *src)
{
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const uint4 x = __ldg(s + v);
        r.w[4 * v + 0] = x.x;
        r.w[4 * v + 1] = x.y;
        r.w[4 * v + 2] = x.z;
        r.w[4 * v + 3] = x.w;
    }
}

template <int NV>
__device__ __forceinline__ void fsp_store_rec(const FspRec<NV> &r, uint8_t *dst)
{
    uint4 *s = reinterpret_cast<uint4 *>(dst);
#pragma unroll
    for (int v = 0; v < NV; ++v)
        s[v] = make_uint4(r.w[4 * v + 0], r.w[4 * v + 1], r.w[4 * v + 2], r.w[4 * v + 3]);
}

// Byte i of the record, i a runtime value (select over the words).
template <int NV>
__device__ __forceinline__ uint32_t fsp_rec_byte_dyn(const FspRec<NV> &r, int i)
{
    uint32_t x = r.w[0];
#pragma unroll
    for (int q = 1; q < 4 * NV; ++q) x = ((i >> 2) == q) ? r.w[q] : x;
    return (x >> ((i & 3) * 8)) & 0xFFu;
}

// Child of rank ci of the parent record: prefix, then the parent's remaining
// job ci, then the other remaining jobs in the same (increasing) order.
template <int NV>
__device__ __forceinline__ void fsp_make_child(const FspRec<NV> &par, int n, int ci, FspRec<NV> &ch)
{
    const int d = (int)fsp_rec_byte_dyn(par, n);
    const uint32_t x = fsp_rec_byte_dyn(par, d + ci);
#pragma unroll
    for (int q = 0; q < 4 * NV; ++q) ch.w[q] = 0u;
#pragma unroll
    for (int i = 0; i < 16 * NV; ++i) {
        const uint32_t cur = (par.w[i >> 2] >> ((i & 3) * 8)) & 0xFFu;
        const uint32_t prv = i > 0 ? (par.w[(i - 1) >> 2] >> (((i - 1) & 3) * 8)) & 0xFFu : 0u;
        uint32_t v;
        if (i < d) v = cur;
        else if (i == d) v = x;
        else if (i <= d + ci) v = prv;
        else if (i < n) v = cur;
        else if (i == n) v = (uint32_t)(d + 1);
        else v = 0u;
        ch.w[i >> 2] |= v << ((i & 3) * 8);
    }
}

// a1-a3 for one node: release times C, S + qmin per machine, the remaining
// set Um, the one-machine bound, and the validity of the record.  var =
// FSP_BOUND_HEADS raises C_k to the earliest start of any remaining job,
// max(C_k, C_{k-1} + min over the remaining set of p[j][k-1]).
template <int MT, int NV, int NW>
__device__ __forceinline__ void fsp_prologue(const FspRec<NV> &r, int n, const int2 *__restrict__ pq, int mp,
                                             uint32_t (&Um)[NW], int32_t (&C)[MT], int32_t (&SQ)[MT],
                                             int32_t &lb1, bool &bad, int var)
{
    const int d = (int)fsp_rec_byte_dyn(r, n);
    bad = d > n;
    uint32_t Am[NW];
    int32_t S[MT], Q[MT];
#pragma unroll
    for (int w = 0; w < NW; ++w) { Um[w] = 0u; Am[w] = 0u; }
#pragma unroll
    for (int k = 0; k < MT; ++k) { C[k] = 0; S[k] = 0; Q[k] = 0x7fffffff; }
#pragma unroll
    for (int i = 0; i < 16 * NV; ++i) {
        if (i < n) {
            uint32_t j = (r.w[i >> 2] >> ((i & 3) * 8)) & 0xFFu;
            if (j >= (uint32_t)n) { bad = true; j = 0; }
            const uint32_t bit = 1u << (j & 31u);
            const bool pre = i < d;
            if (NW == 1) {
                if (Am[0] & bit) bad = true;
                Am[0] |= bit;
                if (!pre) Um[0] |= bit;
            } else {
                const int wj = (int)(j >> 5);
#pragma unroll
                for (int w = 0; w < NW; ++w)
                    if (w == wj) {
                        if (Am[w] & bit) bad = true;
                        Am[w] |= bit;
                        if (!pre) Um[w] |= bit;
                    }
            }
            const int2 *row = pq + j * mp;
            int2 v[MT];
#pragma unroll
            for (int k = 0; k < MT; ++k) v[k] = row[k];
            if (pre) {
                C[0] += v[0].x;
#pragma unroll
                for (int k = 1; k < MT; ++k) C[k] = max(C[k], C[k - 1]) + v[k].x;
            } else {
#pragma unroll
                for (int k = 0; k < MT; ++k) {
                    S[k] += v[k].x;
                    Q[k] = min(Q[k], v[k].y);
                }
            }
        }
    }
    if (var == FSP_BOUND_HEADS && d < n && !bad) {
        int32_t Pm[MT];
#pragma unroll
        for (int k = 0; k < MT; ++k) Pm[k] = 0x7fffffff;
#pragma unroll
        for (int i = 0; i < 16 * NV; ++i) {
            if (i >= d && i < n) {
                const uint32_t j = (r.w[i >> 2] >> ((i & 3) * 8)) & 0xFFu;
                const int2 *row = pq + j * mp;
#pragma unroll
                for (int k = 0; k < MT; ++k) Pm[k] = min(Pm[k], row[k].x);
            }
        }
#pragma unroll
        for (int k = 1; k < MT; ++k) C[k] = max(C[k], C[k - 1] + Pm[k - 1]);
    }
    lb1 = 0;
#pragma unroll
    for (int k = 0; k < MT; ++k) {
        SQ[k] = S[k] + (Q[k] == 0x7fffffff ? 0 : Q[k]);
        lb1 = max(lb1, C[k] + SQ[k]);
    }
}

template <int NW>
__device__ __forceinline__ bool fsp_member(const uint32_t (&Um)[NW], const int4 &t)
{
    if (NW == 1) return (Um[0] & (uint32_t)t.z) != 0u;
    return (((t.w == 0) ? Um[0] : Um[1]) & (uint32_t)t.z) != 0u;
}

// a4/a5 for NPT nodes: per machine pair the max-plus scan of the pair's
// Johnson entries (ent, shared memory, order-major), folded into lb.
// cs / sq: shared columns, machine k of node j at [k * SB + slot[j]].
template <int MT, int NPT, int NW>
__device__ __forceinline__ void fsp_pair_scan(int n, const FspEntry *__restrict__ ent, const int32_t *cs,
                                              const int32_t *sq, int SB, const int (&slot)[NPT],
                                              const uint32_t (&Um)[NPT][NW], int32_t (&lb)[NPT])
{
    const int4 *e = reinterpret_cast<const int4 *>(ent);
#pragma unroll 1
    for (int k = 0; k < MT - 1; ++k) {
        int32_t ck[NPT];
#pragma unroll
        for (int j = 0; j < NPT; ++j) ck[j] = cs[k * SB + slot[j]];
#pragma unroll 1
        for (int l = k + 1; l < MT; ++l) {
            int32_t cl[NPT], sql[NPT], E[NPT], M[NPT];
#pragma unroll
            for (int j = 0; j < NPT; ++j) {
                cl[j] = cs[l * SB + slot[j]];
                sql[j] = sq[l * SB + slot[j]];
                E[j] = 0;
                M[j] = FSP_NEG;
            }
#define FSP_STEP2(T)                                                   \
    _Pragma("unroll") for (int j = 0; j < NPT; ++j)                    \
    {                                                                  \
        if (fsp_member<NW>(Um[j], (T))) {                              \
            M[j] = __viaddmax_s32(E[j], (T).x, M[j]);                  \
            E[j] += (T).y;                                             \
        }                                                              \
    }
            int pos = 0;
            for (; pos + 4 <= n; pos += 4) {
                const int4 t0 = e[pos], t1 = e[pos + 1], t2 = e[pos + 2], t3 = e[pos + 3];
                FSP_STEP2(t0) FSP_STEP2(t1) FSP_STEP2(t2) FSP_STEP2(t3)
            }
            for (; pos < n; ++pos) {
                const int4 t0 = e[pos];
                FSP_STEP2(t0)
            }
#undef FSP_STEP2
            e += n;
#pragma unroll
            for (int j = 0; j < NPT; ++j)
                lb[j] = __viaddmax_s32(sql[j], __viaddmax_s32(ck[j], M[j], cl[j]), lb[j]);
        }
    }
}

// Shared memory of a v2 CTA: {p, q} rows, then the C and S + qmin columns of
// its B * NPT node slots.
struct Bound2Smem {
    size_t ent_off, pq_off, cs_off, sq_off, bytes;
};

static inline Bound2Smem bound2_smem_layout(const fsp_instance *I, int B, int NPT, int MT)
{
    Bound2Smem L;
    size_t o = 0;
    L.ent_off = o; o += fsp_align16((size_t)I->P * I->n * sizeof(FspEntry));
    L.pq_off = o; o += fsp_align16((size_t)I->n * I->mp * 8);
    L.cs_off = o; o += fsp_align16((size_t)MT * B * NPT * 4);
    L.sq_off = o; o += fsp_align16((size_t)MT * B * NPT * 4);
    L.bytes = o;
    return L;
}

__device__ __forceinline__ void fsp_stage_pq(const DevInst &I, FspEntry *ent_s, int2 *pq_s)
{
    const int4 *src = reinterpret_cast<const int4 *>(I.ent);
    int4 *dst = reinterpret_cast<int4 *>(ent_s);
    const int tot = I.P * I.n;
    for (int i = threadIdx.x; i < tot; i += blockDim.x) dst[i] = __ldg(src + i);
    const int nm = I.n * I.m;
    for (int i = threadIdx.x; i < nm; i += blockDim.x) {
        const int j = i / I.m, k = i - j * I.m;
        pq_s[j * I.mp + k] = make_int2(__ldg(I.p + i), __ldg(I.q + i));
    }
    __syncthreads();
}
