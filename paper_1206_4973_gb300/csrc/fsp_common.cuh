// fsp_common.cuh -- instance layout and the node-bound device code shared by
// the bounding and the search kernels (sm_103a).
//
// Node bound (two-machine Johnson bounds with time lags over all machine
// pairs plus one-machine bounds; the paper gives its O(m^2 n log n) cost in
// Sec. V-D).  For pair (k,l) the Johnson recurrence over the remaining set U
//     t_k = C_k, t_l = C_l;  per j: t_k += a_j;  t_l = max(t_l, t_k + lag_j) + b_j
// unrolls to
//     t_l = S_l + max(C_l, C_k + M),   M = max_{i in U} (E_{<i} + a_i + lag_i),
// where E_{<i} sums (a - b) over the members of U before i in Johnson order
// and S_l = sum_{U} b.  The kernel evaluates that form: per table position one
// membership test and three integer ops (add, max, add), the Johnson order
// and (w = a + lag, e = a - b) precomputed per pair once per instance.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fsp.h"

#define FSP_NEG (-(1 << 29)) /* "minus infinity" of the max-plus scan */

// One position of a pair's Johnson order: w = a + lag, e = a - b, the job's
// membership bit and word of the remaining-set mask.
struct __align__(16) FspEntry {
    int32_t w;
    int32_t e;
    uint32_t bit;
    int32_t widx;
};

struct fsp_instance {
    int n, m, P;  // jobs, machines, machine pairs m(m-1)/2
    int stride;   // node record bytes
    int mp;       // row stride (words) of the shared-memory p / q tables (odd)
    int device;
    int sm_count;
    int smem_optin;  // max dynamic shared memory per block
    long long total; // sum of all processing times
    int pmax;        // largest processing time
    int32_t *d_p;    // [n][m] processing times
    int32_t *d_q;    // [n][m] tails: sum of p[j][h] for h > k
    int32_t *d_lag;  // [P][n]
    uint8_t *d_order;  // [P][n] Johnson order (job at each position)
    FspEntry *d_ent;   // [P][n] order-major entries
    int2 *d_we;        // [n][P] position-major {w, e}: entry at position i of every pair
    uint8_t *d_rank;   // [P][n] position of job j in pair kl's order
    int *d_status;     // error flag of malformed records
    uint8_t *d_p16;    // image of the packed bounding kernel (fsp_pool16.cu), or NULL
    int var;           // bound variant (FSP_BOUND_*)
    struct FspHostCache *cache;  // events and kernel attributes reused across calls
};

// Host-side objects an instance keeps between calls (fsp_instance.cu): CUDA
// events handed out and taken back, and the dynamic shared memory each
// kernel was last allowed, so repeated searches skip the driver calls.
int fsp_event_take(fsp_instance *I, cudaEvent_t *ev);
void fsp_event_give(fsp_instance *I, cudaEvent_t ev);
int fsp_allow_smem(fsp_instance *I, const void *kernel, size_t bytes);
// Resident CTAs per SM of a kernel at a block size and dynamic shared memory
// (at least 1), remembered per instance.
int fsp_blocks_per_sm(fsp_instance *I, const void *kernel, int block, size_t smem, int *per_sm);
// Pinned host blocks of FSP_PINNED_BYTES for asynchronous read-backs.
#define FSP_PINNED_BYTES 1024
int fsp_pinned_take(fsp_instance *I, void **p);
void fsp_pinned_give(fsp_instance *I, void *p);
// The pinned block and the two events an instance reserves at creation for
// fsp_solve_noalloc (never handed to other calls).
void fsp_noalloc_reserved(fsp_instance *I, void **pin, cudaEvent_t *ev);
// The address at which kernels on the current device read p in place: p for
// memory of this device, the mapped address of pinned host memory (read over
// the host link), nullptr for anything else (pageable or managed memory,
// another device) or when not `align`-byte aligned: such data is copied first.
const void *fsp_device_view(const void *p, int align);

// By-value view for kernels.
struct DevInst {
    int n, m, P, stride, mp;
    const int32_t *p, *q;
    const FspEntry *ent;
    const int2 *we;
    const uint8_t *rank;
    const uint8_t *order;  // [P][n] job at each position of the pair's Johnson order
    int *status;
    int var;  // bound variant (FSP_BOUND_*)
};

static inline DevInst dev_view(const fsp_instance *I)
{
    DevInst d;
    d.n = I->n; d.m = I->m; d.P = I->P; d.stride = I->stride; d.mp = I->mp;
    d.p = I->d_p; d.q = I->d_q; d.ent = I->d_ent; d.status = I->d_status;
    d.we = I->d_we; d.rank = I->d_rank; d.order = I->d_order;
    d.var = I->var;
    return d;
}

// Image of the packed bounding kernel, built at creation when it applies
// (fsp_pool16.cu).
int pool16_build(fsp_instance *I);

// --- host helpers (fsp_instance.cu) ---
void fsp_set_error(const char *fmt, ...);
int fsp_cuda_fail(cudaError_t e, const char *what);
#define FSP_CUDA(call)                                                 \
    do {                                                               \
        cudaError_t e__ = (call);                                      \
        if (e__ != cudaSuccess) return fsp_cuda_fail(e__, #call);      \
    } while (0)

// Mask words for n jobs and machine template for m.
static inline int fsp_nw(int n) { return n <= 32 ? 1 : n <= 64 ? 2 : n <= 128 ? 4 : 8; }
static inline int fsp_mt(int m) { return (m == 5 || m == 10 || m == 20) ? m : 0; }

// --------------------------------------------------------------------------
// Shared-memory layout of a bounding CTA of B threads.
// --------------------------------------------------------------------------
struct BoundSmem {
    size_t ent_off, p_off, q_off, rec_off, cs_off, sq_off, ss_off, bytes;
};

__host__ __device__ static inline size_t fsp_align16(size_t x) { return (x + 15) & ~(size_t)15; }

static inline BoundSmem bound_smem_layout(const fsp_instance *I, int B, bool ent_smem, int MT)
{
    BoundSmem L;
    size_t o = 0;
    L.ent_off = o;
    if (ent_smem) o += fsp_align16((size_t)I->P * I->n * sizeof(FspEntry));
    L.p_off = o; o += fsp_align16((size_t)I->n * I->mp * 4);
    L.q_off = o; o += fsp_align16((size_t)I->n * I->mp * 4);
    L.rec_off = o; o += fsp_align16((size_t)(I->stride / 4) * B * 4);
    L.cs_off = o; o += fsp_align16((size_t)I->m * B * 4);
    L.sq_off = o; o += fsp_align16((size_t)I->m * B * 4);
    L.ss_off = o;
    if (MT == 0) o += fsp_align16((size_t)I->m * B * 4);  // generic path: S and qmin apart
    L.bytes = o;
    return L;
}

// Stage the instance tables into shared memory (whole block).
__device__ __forceinline__ void fsp_stage_tables(const DevInst &I, FspEntry *ent_s, int32_t *p_s,
                                                 int32_t *q_s)
{
    if (ent_s) {
        const int4 *src = reinterpret_cast<const int4 *>(I.ent);
        int4 *dst = reinterpret_cast<int4 *>(ent_s);
        const int tot = I.P * I.n;
        for (int i = threadIdx.x; i < tot; i += blockDim.x) dst[i] = __ldg(src + i);
    }
    const int nm = I.n * I.m;
    for (int i = threadIdx.x; i < nm; i += blockDim.x) {
        const int j = i / I.m, k = i - j * I.m;
        p_s[j * I.mp + k] = __ldg(I.p + i);
        q_s[j * I.mp + k] = __ldg(I.q + i);
    }
    __syncthreads();
}

template <int NW>
__device__ __forceinline__ uint32_t fsp_pick(const uint32_t (&U)[NW], int widx)
{
    if (NW == 1) return U[0];
    uint32_t r = U[0];
#pragma unroll
    for (int w = 1; w < NW; ++w) r = (widx == w) ? U[w] : r;
    return r;
}

__device__ __forceinline__ uint32_t fsp_rec_byte(const uint32_t *rec, int B, int i)
{
    return (rec[(i >> 2) * B] >> ((i & 3) * 8)) & 0xFFu;
}

// Bound of the node whose record sits in the shared-memory column `rec`
// (word w at rec[w*B]).  cs / sq / ss: per-thread machine columns (k at
// [k*B]).  Sets bad for a malformed record (depth > n, id >= n, repeats).
template <int NW, int MT, bool ES>
__device__ __forceinline__ int32_t fsp_node_bound(const DevInst &I, const FspEntry *__restrict__ ent,
                                                  const int32_t *__restrict__ p_s,
                                                  const int32_t *__restrict__ q_s,
                                                  const uint32_t *rec, int32_t *cs, int32_t *sq,
                                                  int32_t *ss, int B, bool &bad)
{
    const int n = I.n;
    const int m = MT > 0 ? MT : I.m;
    const int mp = I.mp;
    uint32_t Um[NW], Am[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) { Um[w] = 0u; Am[w] = 0u; }
    const int d = (int)fsp_rec_byte(rec, B, n);
    bad = d > n;

    constexpr int R = MT > 0 ? MT : 1;
    int32_t C[R], S[R], Q[R];
    if (MT > 0) {
#pragma unroll
        for (int k = 0; k < R; ++k) { C[k] = 0; S[k] = 0; Q[k] = 0x7fffffff; }
    } else {
        for (int k = 0; k < m; ++k) { cs[k * B] = 0; sq[k * B] = 0; ss[k * B] = 0x7fffffff; }
    }

    // a1/a2: release times of the prefix, remaining sums and smallest tails.
    const int nwords = (n + 3) >> 2;
    for (int wi = 0; wi < nwords; ++wi) {
        const uint32_t word = rec[wi * B];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = wi * 4 + b;
            if (i < n) {
                uint32_t j = (word >> (8 * b)) & 0xFFu;
                if (j >= (uint32_t)n) { bad = true; j = 0; }
                const uint32_t bit = 1u << (j & 31u);
                const int wj = (int)(j >> 5);
                const bool pre = i < d;
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    if (w == wj) {
                        if (Am[w] & bit) bad = true;
                        Am[w] |= bit;
                        if (!pre) Um[w] |= bit;
                    }
                }
                const int32_t *row = p_s + j * mp;
                const int32_t *qrow = q_s + j * mp;
                if (MT > 0) {
                    if (pre) {
                        C[0] += row[0];
#pragma unroll
                        for (int k = 1; k < R; ++k) C[k] = max(C[k], C[k - 1]) + row[k];
                    } else {
#pragma unroll
                        for (int k = 0; k < R; ++k) { S[k] += row[k]; Q[k] = min(Q[k], qrow[k]); }
                    }
                } else {
                    if (pre) {
                        int32_t c = cs[0] + row[0];
                        cs[0] = c;
                        for (int k = 1; k < m; ++k) {
                            c = max(cs[k * B], c) + row[k];
                            cs[k * B] = c;
                        }
                    } else {
                        for (int k = 0; k < m; ++k) {
                            sq[k * B] += row[k];
                            ss[k * B] = min(ss[k * B], qrow[k]);
                        }
                    }
                }
            }
        }
    }

    // FSP_BOUND_HEADS: release times raised to the earliest start of any
    // remaining job, R_k = max(C_k, R_{k-1} + min over U of p[j][k-1]).
    if (I.var == FSP_BOUND_HEADS && d < n && !bad) {
        if (MT > 0) {
            int32_t Pm[R];
#pragma unroll
            for (int k = 0; k < R; ++k) Pm[k] = 0x7fffffff;
            for (int i = d; i < n; ++i) {
                const int32_t *row = p_s + fsp_rec_byte(rec, B, i) * mp;
#pragma unroll
                for (int k = 0; k < R; ++k) Pm[k] = min(Pm[k], row[k]);
            }
#pragma unroll
            for (int k = 1; k < R; ++k) C[k] = max(C[k], C[k - 1] + Pm[k - 1]);
        } else {
            int32_t prev = cs[0];
            for (int k = 1; k < m; ++k) {
                int32_t pm = 0x7fffffff;
                for (int i = d; i < n; ++i) pm = min(pm, p_s[fsp_rec_byte(rec, B, i) * mp + k - 1]);
                prev = max(cs[k * B], prev + pm);
                cs[k * B] = prev;
            }
        }
    }

    // a3: one-machine bounds; store C and S + qmin for the pair loop.
    int32_t lb = 0;
    if (MT > 0) {
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int32_t sqk = S[k] + (Q[k] == 0x7fffffff ? 0 : Q[k]);
            cs[k * B] = C[k];
            sq[k * B] = sqk;
            lb = max(lb, C[k] + sqk);
        }
    } else {
        for (int k = 0; k < m; ++k) {
            const int32_t qk = ss[k * B];
            const int32_t sqk = sq[k * B] + (qk == 0x7fffffff ? 0 : qk);
            sq[k * B] = sqk;
            lb = max(lb, cs[k * B] + sqk);
        }
    }

    // a4/a5: two-machine bounds, max over pairs.
    const FspEntry *e = ent;
    for (int k = 0; k < m - 1; ++k) {
        const int32_t ck = cs[k * B];
        for (int l = k + 1; l < m; ++l) {
            const int32_t cl = cs[l * B];
            const int32_t sql = sq[l * B];
            int32_t E = 0, M = FSP_NEG;
            int pos = 0;
#define FSP_STEP(T)                                                        \
    {                                                                      \
        const uint32_t wd = fsp_pick<NW>(Um, (T).widx);                    \
        if (wd & (T).bit) {                                                \
            M = max(M, E + (T).w);                                         \
            E += (T).e;                                                    \
        }                                                                  \
    }
            for (; pos + 4 <= n; pos += 4) {
                const FspEntry t0 = e[pos], t1 = e[pos + 1], t2 = e[pos + 2], t3 = e[pos + 3];
                FSP_STEP(t0) FSP_STEP(t1) FSP_STEP(t2) FSP_STEP(t3)
            }
            for (; pos < n; ++pos) {
                const FspEntry t0 = e[pos];
                FSP_STEP(t0)
            }
#undef FSP_STEP
            e += n;
            lb = max(lb, sql + max(cl, ck + M));
        }
    }
    return lb;
}

// Learned-order features of a node record r (2m+1 floats at xo): C_k / T,
// S_k / T, d / n; also returns the remaining set (U, 8 words), C, S and the
// smallest tails Q (0x7fffffff when none) for callers that need them.
__device__ __forceinline__ void fsp_features(const DevInst &I, const uint8_t *r, float T, float *xo, uint32_t *U,
                                             int32_t *C, int32_t *S, int32_t *Q)
{
    const int n = I.n, m = I.m;
    const int d = r[n] <= n ? r[n] : n;
    for (int w = 0; w < 8; ++w) U[w] = 0u;
    for (int k = 0; k < m; ++k) { C[k] = 0; S[k] = 0; Q[k] = 0x7fffffff; }
    for (int i = 0; i < n; ++i) {
        const int j = r[i] < n ? r[i] : 0;
        const int32_t *row = I.p + j * m;
        if (i < d) {
            C[0] += row[0];
            for (int k = 1; k < m; ++k) C[k] = max(C[k], C[k - 1]) + row[k];
        } else {
            U[j >> 5] |= 1u << (j & 31);
            for (int k = 0; k < m; ++k) { S[k] += row[k]; Q[k] = min(Q[k], I.q[j * m + k]); }
        }
    }
    for (int k = 0; k < m; ++k) {
        xo[k] = __fdiv_rn((float)C[k], T);
        xo[m + k] = __fdiv_rn((float)S[k], T);
    }
    xo[2 * m] = __fdiv_rn((float)d, (float)n);
}
