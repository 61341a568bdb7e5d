// fsp_batch.cu -- many instances of mixed shape in one persistent launch.
//
// Each CTA takes instance indices from a device work queue (one atomic
// counter) and solves each instance completely with CTA-local barriers only:
// per-instance tables built in shared memory, the NEH upper bound, then the
// same pool-synchronous depth-first search as fsp_solve (Sec. II-A
// operators, Sec. III pool of deepest nodes) on its own stack in global
// memory.  A per-instance pool size (tuned per shape on measured
// throughput) and node budget apply.  The queue reset and the persistent
// kernel are captured once in a CUDA graph and replayed.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "fsp_family.cuh"

#define BB 256        // threads per CTA

// Shapes of the batch kernel: machines MT x record vectors NV x mask words NW
// (n <= 15, <= 31, <= 63 jobs; m = 5, 10, 20).
#define FSP_SHAPES_BATCH(X) \
    X(5, 1, 1) X(5, 2, 1) X(5, 4, 2) X(10, 1, 1) X(10, 2, 1) X(10, 4, 2) X(20, 2, 1)
#define SEL_Q 4       // selection candidates per thread per chunk
#define POOL_MAX 4096 // largest per-instance pool

struct BatchDesc {  // one instance (device)
    int n, m;
    long long p_off;  // offset of p (n x m int32) in the flat array
    int pool;
    int ub0;          // 0 = compute NEH
    long long budget; // 0 = none
};

struct BatchOut {  // one result (device; mirrored by fsp_batch_result)
    int cmax, status, ub0, pad;
    long long bounded, branched, pruned, leaves, iterations, updates;
};

struct BatchWs {  // per-CTA scratch in global memory
    uint8_t *stack, *children;
    int32_t *lbs;
    long long cap;  // records per stack
    int stride_max;
};

// Split mode: the work items are (instance, first job) pairs, the subtrees of
// the root; every CTA working on an instance shares its UB and counters.
struct BatchSplit {
    const int *item_inst, *item_job;  // per item
    int items;
    int *ub;                  // per instance: best makespan so far (atomicMin)
    unsigned long long *key;  // per instance: (best makespan << 32) | item that found it, ~0 = none
    long long *cnt;           // per instance: bounded, branched, pruned, leaves, iterations, updates
    int *flags;               // per instance: 1 = a node budget stopped an item, 2 = a stack filled up
    uint8_t *item_perm;       // per item: the best schedule it found (FSP_MAX_JOBS bytes)
};

__device__ __forceinline__ int b_block_incl_scan(int v, int *warp_tot)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) warp_tot[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int t = lane < BB / 32 ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        if (lane < BB / 32) warp_tot[lane] = t;
    }
    __syncthreads();
    const int add = wid > 0 ? warp_tot[wid - 1] : 0;
    __syncthreads();
    return v + add;
}

__device__ __forceinline__ int b_block_sum(int v, int *warp_tot)
{
    const int incl = b_block_incl_scan(v, warp_tot);
    __shared__ int s_total;
    if (threadIdx.x == BB - 1) s_total = incl;
    __syncthreads();
    const int t = s_total;
    __syncthreads();
    return t;
}

// Johnson precedence with lags (same rule as the instance tables).
__device__ __forceinline__ bool b_precedes(int i, int32_t ai, int32_t bi, int32_t li, int j, int32_t aj, int32_t bj,
                                           int32_t lj)
{
    const bool late_i = ai > bi, late_j = aj > bj;
    if (late_i != late_j) return !late_i;
    if (!late_i) {
        const int32_t ki = ai + li, kj = aj + lj;
        if (ki != kj) return ki < kj;
    } else {
        const int32_t ki = bi + li, kj = bj + lj;
        if (ki != kj) return ki > kj;
    }
    return i < j;
}

struct BatchShared {  // static shared state of a CTA
    int warp_tot[BB / 32];
    uint8_t inc[FSP_MAX_JOBS + 1], seq[FSP_MAX_JOBS + 1], ord[FSP_MAX_JOBS + 1];
    int32_t tot[FSP_MAX_JOBS + 1];
    unsigned long long best_key;
};

// Shared memory of a batch CTA for an n x m instance: the family layout
// (fsp_family.cuh) for the CTA's warps, then the parents' first-child offsets.
__host__ __device__ inline size_t batch_smem_nm(int n, int m)
{
    const int mp = (m % 2 == 0) ? m + 1 : m, nv = (n + 1 + 15) / 16;
    return fsp_align16(family_smem_layout_nm(n, m, mp, m, nv, BB / 32).bytes) + (size_t)(POOL_MAX / 2 + 4) * 4;
}

// NEH upper bound: jobs by decreasing total time, each inserted at the
// position of smallest partial makespan, earliest on ties; the sequence is
// left in sh.seq.  All threads of the CTA call it.
template <int MT>
__device__ int b_neh(const int32_t *__restrict__ p, int n, BatchShared &sh)
{
    const int tid = threadIdx.x;
    uint8_t *seq = sh.seq, *ord = sh.ord;
    int32_t *tot = sh.tot;
    unsigned long long &best_key = sh.best_key;
    for (int j = tid; j < n; j += BB) {
        int32_t s = 0;
        for (int k = 0; k < MT; ++k) s += p[j * MT + k];
        tot[j] = s;
    }
    __syncthreads();
    for (int j = tid; j < n; j += BB) {
        int rank = 0;
        for (int i = 0; i < n; ++i) rank += (tot[i] > tot[j]) || (tot[i] == tot[j] && i < j);
        ord[rank] = (uint8_t)j;
    }
    __syncthreads();
    for (int len = 0; len < n; ++len) {
        const int job = ord[len];
        if (tid == 0) best_key = ~0ull;
        __syncthreads();
        for (int pos = tid; pos <= len; pos += BB) {
            int32_t C[MT];
#pragma unroll
            for (int k = 0; k < MT; ++k) C[k] = 0;
            for (int i = 0; i <= len; ++i) {
                const int j = i < pos ? seq[i] : (i == pos ? job : seq[i - 1]);
                C[0] += p[j * MT];
#pragma unroll
                for (int k = 1; k < MT; ++k) C[k] = max(C[k], C[k - 1]) + p[j * MT + k];
            }
            atomicMin(&best_key, ((unsigned long long)(uint32_t)C[MT - 1] << 32) | (unsigned)pos);
        }
        __syncthreads();
        const int at = (int)(best_key & 0xffffffffu);
        if (tid == 0) {
            for (int i = len; i > at; --i) seq[i] = seq[i - 1];
            seq[at] = (uint8_t)job;
        }
        __syncthreads();
    }
    const int ub = (int)(best_key >> 32);
    __syncthreads();
    return ub;
}

// One instance's search (whole instance), or (SPLIT) the subtree of the
// root whose schedule starts with job `job`, sharing the instance's UB and
// counters with the other CTAs; tables_ready: this CTA's shared memory
// already holds the instance's tables.
template <int MT, int NV, int NW, bool SPLIT>
__device__ void b_solve(const int32_t *__restrict__ p, const BatchDesc &D, BatchOut *out, uint8_t *perm_out,
                        const BatchWs &W, unsigned char *smem, BatchShared &sh, const BatchSplit &X, int inst,
                        int item, int job, bool tables_ready)
{
    const int n = D.n, tid = threadIdx.x;
    const int P = MT * (MT - 1) / 2, mp = (MT % 2 == 0) ? MT + 1 : MT;
    const int stride = (n + 1 + 15) / 16 * 16;
    const FamSmem L = family_smem_layout_nm(n, MT, mp, MT, NV, BB / 32);
    const FamView V = fam_view(smem, L, tid >> 5);
    int2 *pq_s = V.pq;
    int *poff = reinterpret_cast<int *>(smem + fsp_align16(L.bytes));
    int *warp_tot = sh.warp_tot;
    uint8_t *inc = sh.inc, *seq = sh.seq, *ord = sh.ord;
    int32_t *tot = sh.tot;
    unsigned long long &best_key = sh.best_key;

    // tables: {p, tail} rows and the Johnson entries of every pair
    if (!SPLIT || !tables_ready) {
    for (int i = tid; i < n * MT; i += BB) {
        const int j = i / MT, k = i - j * MT;
        int32_t q = 0;
        for (int h = k + 1; h < MT; ++h) q += p[j * MT + h];
        pq_s[j * mp + k] = make_int2(p[i], q);
    }
    for (int e = tid; e < P * n; e += BB) {
        const int kl = e / n, j = e - kl * n;
        int k = 0, rem = kl;
        while (rem >= MT - 1 - k) { rem -= MT - 1 - k; ++k; }
        const int l = k + 1 + rem;
        int32_t aj = p[j * MT + k], bj = p[j * MT + l], lj = 0;
        for (int h = k + 1; h < l; ++h) lj += p[j * MT + h];
        int rank = 0;
        for (int i = 0; i < n; ++i) {
            if (i == j) continue;
            int32_t li = 0;
            for (int h = k + 1; h < l; ++h) li += p[i * MT + h];
            rank += b_precedes(i, p[i * MT + k], p[i * MT + l], li, j, aj, bj, lj);
        }
        V.we[rank * P + kl] = make_int2(aj + lj, aj - bj);  // position-major entries
        V.rk8[kl * V.rks8 + j] = (uint8_t)rank;             // each job's position
    }
    __syncthreads();
    fam_tables_finish<MT>(V, n, mp);
    }

    // the UB: NEH unless given (whole instances), or the instance's shared UB (split)
    int ub = D.ub0;
    if (SPLIT) {
        ub = *(volatile int *)&X.ub[inst];
    } else if (ub <= 0) {
        ub = b_neh<MT>(p, n, sh);
        for (int i = tid; i < n; i += BB) inc[i] = seq[i];
    }
    __syncthreads();

    // the search
    long long bounded = 0, branched = 0, pruned = 0, leaves = 0, iters = 0, updates = 0;
    int status = FSP_OK;
    long long S = 1;
    if (SPLIT && job >= 0) {  // the root's child that schedules `job` first (the rest in increasing order)
        for (int i = tid; i < stride; i += BB)
            W.stack[i] = (uint8_t)(i == 0 ? job : i < n ? (i - 1 < job ? i - 1 : i) : i == n ? 1 : 0);
    } else {
        for (int i = tid; i < stride; i += BB) W.stack[i] = (uint8_t)(i < n ? i : 0);
    }
    bool improved = false;
    __shared__ int s_ub;
    __syncthreads();
    const int pool = D.pool;
    const int warp = tid >> 5, lane = tid & 31;
    while (S > 0) {
        if (SPLIT) {  // the instance's UB and node count, as the other CTAs left them
            if (tid == 0) {
                s_ub = min(ub, *(volatile int *)&X.ub[inst]);
                if (D.budget > 0 && *(volatile long long *)&X.cnt[6 * inst] >= D.budget) s_ub = -1;
            }
            __syncthreads();
            const int u = s_ub;
            __syncthreads();
            if (u < 0) { status = FSP_INCOMPLETE; break; }
            ub = u;
        } else if (D.budget > 0 && bounded >= D.budget) {
            status = FSP_INCOMPLETE;
            break;
        }
        // selection: deepest parents while their children fit (at least one)
        const long long cand = S < pool ? S : pool;
        long long running = 0, np = 0;
        for (long long base = 0; base < cand; base += (long long)BB * SEL_Q) {
            int r[SEL_Q], tsum = 0;
#pragma unroll
            for (int q = 0; q < SEL_Q; ++q) {
                const long long i = base + (long long)tid * SEL_Q + q;
                r[q] = i < cand ? n - (int)W.stack[(S - 1 - i) * stride + n] : 0;
                tsum += r[q];
            }
            int run = b_block_incl_scan(tsum, warp_tot) - tsum, taken = 0, tsum_taken = 0;
#pragma unroll
            for (int q = 0; q < SEL_Q; ++q) {
                const long long i = base + (long long)tid * SEL_Q + q;
                if (i < cand && (i == 0 || running + run + r[q] <= pool)) {
                    poff[i] = (int)(running + run);
                    taken++;
                    tsum_taken += r[q];
                }
                run += r[q];
            }
            const int ct = b_block_sum(taken, warp_tot), cts = b_block_sum(tsum_taken, warp_tot);
            np += ct;
            running += cts;
            if (ct < BB * SEL_Q) break;
        }
        const long long nch = running;
        if (tid == 0) poff[np] = (int)nch;
        if (S - np + nch > W.cap) { status = FSP_ERR_CAPACITY; break; }
        if (tid == 0) best_key = ~0ull;
        __syncthreads();
        // branching + bounding: each warp bounds a parent's children together
        for (long long f = warp; f < np; f += BB / 32) {
            if (lane < NV)
                reinterpret_cast<uint4 *>(V.recb)[lane] =
                    reinterpret_cast<const uint4 *>(W.stack + (S - 1 - f) * stride)[lane];
            __syncwarp();
            fam_bound<MT, NV, false, false>(V, V.recb, poff[f], n, mp, stride, ub, W.children, W.lbs, &best_key,
                                            nullptr, 0, nullptr);
            __syncwarp();
        }
        __syncthreads();
        const unsigned long long bk = best_key;
        const int ub_new = (bk != ~0ull && (int)(bk >> 32) < ub) ? (int)(bk >> 32) : ub;
        if (ub_new < ub) {
            const long long idx = (long long)(bk & 0xffffffffull);
            for (int i = tid; i < n; i += BB) inc[i] = W.children[idx * stride + i];
            updates++;
            if (SPLIT) {
                improved = true;
                if (tid == 0) {
                    atomicMin(&X.ub[inst], ub_new);
                    atomicMin(&X.key[inst], ((unsigned long long)(uint32_t)ub_new << 32) | (unsigned)item);
                }
            }
        }
        ub = ub_new;
        // elimination: survivors (non-leaf, bound < UB), pushed in reverse order
        int my_s = 0, my_l = 0;
        for (long long c = tid; c < nch; c += BB) {
            const bool leaf = W.children[c * stride + n] == (uint8_t)(n - 1);
            my_l += leaf;
            my_s += !leaf && W.lbs[c] < ub;
        }
        const int total = b_block_sum(my_s, warp_tot), nleaf = b_block_sum(my_l, warp_tot);
        const long long base_s = S - np;
        long long done = 0;
        for (long long c0 = 0; c0 < nch; c0 += BB) {
            const long long c = c0 + tid;
            const bool surv = c < nch && W.children[c * stride + n] != (uint8_t)(n - 1) && W.lbs[c] < ub;
            const int incl = b_block_incl_scan(surv ? 1 : 0, warp_tot);
            if (surv) {
                const long long q = done + incl - 1;
                const uint4 *src = reinterpret_cast<const uint4 *>(W.children + c * stride);
                uint4 *dst = reinterpret_cast<uint4 *>(W.stack + (base_s + total - 1 - q) * stride);
                for (int v = 0; v < stride / 16; ++v) dst[v] = src[v];
            }
            done += b_block_sum(surv ? 1 : 0, warp_tot);
        }
        S = base_s + total;
        bounded += nch;
        branched += np;
        leaves += nleaf;
        pruned += nch - nleaf - total;
        iters++;
        if (SPLIT && tid == 0) atomicAdd((unsigned long long *)&X.cnt[6 * inst], (unsigned long long)nch);
        __syncthreads();
    }
    if (SPLIT) {  // this item's share of the counters, its flags and its best schedule
        if (tid == 0) {
            unsigned long long *c = (unsigned long long *)&X.cnt[6 * inst];
            atomicAdd(c + 1, (unsigned long long)branched);
            atomicAdd(c + 2, (unsigned long long)pruned);
            atomicAdd(c + 3, (unsigned long long)leaves);
            atomicAdd(c + 4, (unsigned long long)iters);
            atomicAdd(c + 5, (unsigned long long)updates);
            if (status == FSP_INCOMPLETE) atomicOr(&X.flags[inst], 1);
            if (status == FSP_ERR_CAPACITY) atomicOr(&X.flags[inst], 2);
        }
        if (improved)
            for (int i = tid; i < n; i += BB) X.item_perm[(size_t)item * FSP_MAX_JOBS + i] = inc[i];
        __syncthreads();
        return;
    }
    if (tid == 0) {
        out->cmax = ub;
        out->status = status;
        out->bounded = bounded;
        out->branched = branched;
        out->pruned = pruned;
        out->leaves = leaves;
        out->iterations = iters;
        out->updates = updates;
    }
    for (int i = tid; i < n; i += BB) perm_out[i] = inc[i];
    __syncthreads();
}

__global__ void __launch_bounds__(BB) k_batch(const BatchDesc *__restrict__ desc, int count,
                                              const int32_t *__restrict__ p_flat, BatchOut *out, uint8_t *perms,
                                              int *queue, BatchWs W)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_inst;
    __shared__ BatchShared sh;
    BatchWs w = W;
    w.stack = W.stack + (size_t)blockIdx.x * W.cap * W.stride_max;
    w.children = W.children + (size_t)blockIdx.x * (POOL_MAX + FSP_MAX_JOBS) * W.stride_max;
    w.lbs = W.lbs + (size_t)blockIdx.x * (POOL_MAX + FSP_MAX_JOBS);
    for (;;) {
        if (threadIdx.x == 0) s_inst = atomicAdd(queue, 1);
        __syncthreads();
        const int i = s_inst;
        __syncthreads();
        if (i >= count) break;
        const BatchDesc D = desc[i];
        const int32_t *p = p_flat + D.p_off;
        const int nv = (D.n + 1 + 15) / 16, nw = D.n <= 32 ? 1 : 2;
        uint8_t *po = perms + (size_t)i * FSP_MAX_JOBS;
#define B_CASE(MT_, NV_, NW_)                                                                          \
    if (D.m == MT_ && nv == NV_ && nw == NW_) {                                                        \
        b_solve<MT_, NV_, NW_, false>(p, D, out + i, po, w, smem, sh, BatchSplit{}, i, 0, 0, false);   \
        continue;                                                                                      \
    }
        FSP_SHAPES_BATCH(B_CASE)
#undef B_CASE
        if (threadIdx.x == 0) out[i].status = FSP_ERR_ARG;  // shape without a kernel (checked on the host)
    }
}

// Split mode, before the items: each instance's UB (NEH unless given), its
// NEH schedule as the permutation to report if no item improves on it, and
// its shared counters cleared.  One CTA per instance.
__global__ void __launch_bounds__(BB) k_batch_split_init(const BatchDesc *__restrict__ desc,
                                                         const int32_t *__restrict__ p_flat, uint8_t *perms,
                                                         BatchSplit X)
{
    __shared__ BatchShared sh;
    const int i = blockIdx.x;
    const BatchDesc D = desc[i];
    const int32_t *p = p_flat + D.p_off;
    int ub = D.ub0;
    if (ub <= 0) {
        ub = D.m == 5 ? b_neh<5>(p, D.n, sh) : D.m == 10 ? b_neh<10>(p, D.n, sh) : b_neh<20>(p, D.n, sh);
        for (int j = threadIdx.x; j < D.n; j += BB) perms[(size_t)i * FSP_MAX_JOBS + j] = sh.seq[j];
    }
    if (threadIdx.x == 0) {
        X.ub[i] = ub;
        X.key[i] = ~0ull;
        X.flags[i] = 0;
        for (int k = 0; k < 6; ++k) X.cnt[6 * i + k] = 0;
    }
}

// Split mode: the persistent kernel over the work items; a CTA keeps the
// tables of the instance it last worked on (the items of an instance are
// consecutive in the queue).
__global__ void __launch_bounds__(BB) k_batch_split(const BatchDesc *__restrict__ desc,
                                                    const int32_t *__restrict__ p_flat, int *queue, BatchWs W,
                                                    BatchSplit X)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    __shared__ BatchShared sh;
    BatchWs w = W;
    w.stack = W.stack + (size_t)blockIdx.x * W.cap * W.stride_max;
    w.children = W.children + (size_t)blockIdx.x * (POOL_MAX + FSP_MAX_JOBS) * W.stride_max;
    w.lbs = W.lbs + (size_t)blockIdx.x * (POOL_MAX + FSP_MAX_JOBS);
    int cur = -1;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= X.items) break;
        const int i = X.item_inst[item], job = X.item_job[item];
        const BatchDesc D = desc[i];
        const int32_t *p = p_flat + D.p_off;
        const int nv = (D.n + 1 + 15) / 16, nw = D.n <= 32 ? 1 : 2;
        const bool ready = cur == i;
        cur = i;
#define B_CASE(MT_, NV_, NW_)                                                                   \
    if (D.m == MT_ && nv == NV_ && nw == NW_) {                                                 \
        b_solve<MT_, NV_, NW_, true>(p, D, nullptr, nullptr, w, smem, sh, X, i, item, job, ready); \
        continue;                                                                               \
    }
        FSP_SHAPES_BATCH(B_CASE)
#undef B_CASE
        cur = -1;
    }
}

// Split mode, after the items: each instance's result from its shared state.
__global__ void k_batch_split_finish(const BatchDesc *__restrict__ desc, int count, BatchOut *out, uint8_t *perms,
                                     BatchSplit X)
{
    const int i = blockIdx.x;
    if (i >= count) return;
    const unsigned long long key = X.key[i];
    if (key != ~0ull) {
        const int item = (int)(key & 0xffffffffull);
        for (int j = threadIdx.x; j < desc[i].n; j += blockDim.x)
            perms[(size_t)i * FSP_MAX_JOBS + j] = X.item_perm[(size_t)item * FSP_MAX_JOBS + j];
    }
    if (threadIdx.x == 0) {
        BatchOut o;
        o.cmax = X.ub[i];
        o.status = (X.flags[i] & 2) ? FSP_ERR_CAPACITY : (X.flags[i] & 1) ? FSP_INCOMPLETE : FSP_OK;
        o.ub0 = 0;
        o.pad = 0;
        o.bounded = X.cnt[6 * i];
        o.branched = X.cnt[6 * i + 1];
        o.pruned = X.cnt[6 * i + 2];
        o.leaves = X.cnt[6 * i + 3];
        o.iterations = X.cnt[6 * i + 4];
        o.updates = X.cnt[6 * i + 5];
        out[i] = o;
    }
}

// ------------------------------------------------------------------ host --

struct fsp_batch {
    int count, device, sm_count, grid;
    BatchDesc *d_desc;
    int32_t *d_p;
    BatchOut *d_out;
    uint8_t *d_perms;
    int *d_queue;
    BatchWs ws;
    size_t smem;
    std::vector<BatchDesc> desc;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    bool split = false;
    BatchSplit X{};
    int *d_item = nullptr;  // item instances, then item jobs
};

static bool batch_shape_ok(int n, int m)
{
    const int nv = (n + 1 + 15) / 16, nw = n <= 32 ? 1 : 2;
    if (n < 2 || n > 63) return false;
#define B_OK(MT_, NV_, NW_) if (m == MT_ && nv == NV_ && nw == NW_) return true;
    FSP_SHAPES_BATCH(B_OK)
#undef B_OK
    return false;
}


static void batch_free(fsp_batch *B)
{
    if (!B) return;
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    cudaFree(B->d_desc); cudaFree(B->d_p); cudaFree(B->d_out); cudaFree(B->d_perms); cudaFree(B->d_queue);
    cudaFree(B->ws.stack); cudaFree(B->ws.children); cudaFree(B->ws.lbs);
    cudaFree(B->d_item); cudaFree(B->X.ub); cudaFree(B->X.key); cudaFree(B->X.cnt); cudaFree(B->X.flags);
    cudaFree(B->X.item_perm);
    delete B;
}

static int batch_capture(fsp_batch *B)
{
    if (B->exec) { cudaGraphExecDestroy(B->exec); B->exec = nullptr; }
    if (B->graph) { cudaGraphDestroy(B->graph); B->graph = nullptr; }
    cudaStream_t st;
    FSP_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaMemsetAsync(B->d_queue, 0, sizeof(int), st);
    if (e == cudaSuccess && !B->split) {
        k_batch<<<B->grid, BB, B->smem, st>>>(B->d_desc, B->count, B->d_p, B->d_out, B->d_perms, B->d_queue, B->ws);
        e = cudaGetLastError();
    } else if (e == cudaSuccess) {
        k_batch_split_init<<<B->count, BB, 0, st>>>(B->d_desc, B->d_p, B->d_perms, B->X);
        k_batch_split<<<B->grid, BB, B->smem, st>>>(B->d_desc, B->d_p, B->d_queue, B->ws, B->X);
        k_batch_split_finish<<<B->count, 64, 0, st>>>(B->d_desc, B->count, B->d_out, B->d_perms, B->X);
        e = cudaGetLastError();
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(st, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&B->exec, g, 0);
    B->graph = g;
    cudaStreamDestroy(st);
    if (e != cudaSuccess) return fsp_cuda_fail(e, "batch graph capture");
    return FSP_OK;
}

extern "C" int fsp_batch_create(int count, const int32_t *shapes, const int32_t *p_flat, const int64_t *pools,
                                const int64_t *budgets, const int32_t *ub0, fsp_batch **out)
{
    if (!out || count < 1 || !shapes || !p_flat || !pools) {
        fsp_set_error("fsp_batch_create: invalid argument");
        return FSP_ERR_ARG;
    }
    *out = nullptr;
    fsp_batch *B = new fsp_batch();
    B->count = count;
    long long off = 0;
    int n_max = 2, m_max = 5, s_max = 16;
    size_t smem_max = 0;
    for (int i = 0; i < count; ++i) {
        const int n = shapes[2 * i], m = shapes[2 * i + 1];
        if (!batch_shape_ok(n, m) || pools[i] < 1 || pools[i] > POOL_MAX) {
            fsp_set_error("fsp_batch_create: instance %d: shape %dx%d or pool %lld not supported "
                          "(m in {5,10,20}, n <= 63, 1 <= pool <= %d)", i, n, m, (long long)pools[i], POOL_MAX);
            delete B;
            return FSP_ERR_ARG;
        }
        for (long long k = 0; k < (long long)n * m; ++k)
            if (p_flat[off + k] < 1 || p_flat[off + k] > 32767) {
                fsp_set_error("fsp_batch_create: instance %d: processing time outside 1..32767", i);
                delete B;
                return FSP_ERR_ARG;
            }
        BatchDesc d;
        d.n = n; d.m = m; d.p_off = off; d.pool = (int)pools[i];
        d.ub0 = ub0 ? ub0[i] : 0;
        d.budget = budgets ? budgets[i] : 0;
        B->desc.push_back(d);
        off += (long long)n * m;
        if (n > n_max) n_max = n;
        if (m > m_max) m_max = m;
        if (batch_smem_nm(n, m) > smem_max) smem_max = batch_smem_nm(n, m);
        const int s = (n + 1 + 15) / 16 * 16;
        if (s > s_max) s_max = s;
    }
    int rc = FSP_OK;
    cudaError_t e;
#define TRYB(call) do { e = (call); if (e != cudaSuccess) { rc = fsp_cuda_fail(e, #call); goto fail; } } while (0)
    TRYB(cudaGetDevice(&B->device));
    TRYB(cudaDeviceGetAttribute(&B->sm_count, cudaDevAttrMultiProcessorCount, B->device));
    {
        int optin = 0;
        TRYB(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, B->device));
        B->smem = smem_max;
        if ((int)B->smem > optin) {
            fsp_set_error("fsp_batch_create: instances too large for one CTA's shared memory");
            rc = FSP_ERR_ARG;
            goto fail;
        }
        TRYB(cudaFuncSetAttribute((const void *)k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B->smem));
        TRYB(cudaFuncSetAttribute((const void *)k_batch_split, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)B->smem));
        int per_sm = 0;
        TRYB(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, BB, B->smem));
        B->grid = B->sm_count * (per_sm > 0 ? per_sm : 1);
        if (B->grid > count) B->grid = count;
    }
    B->ws.stride_max = s_max;
    B->ws.cap = (long long)n_max * (POOL_MAX + n_max);
    TRYB(cudaMalloc(&B->d_desc, sizeof(BatchDesc) * count));
    TRYB(cudaMalloc(&B->d_p, sizeof(int32_t) * off));
    TRYB(cudaMalloc(&B->d_out, sizeof(BatchOut) * count));
    TRYB(cudaMalloc(&B->d_perms, (size_t)FSP_MAX_JOBS * count));
    TRYB(cudaMalloc(&B->d_queue, sizeof(int)));
    TRYB(cudaMalloc(&B->ws.stack, (size_t)B->grid * B->ws.cap * s_max));
    TRYB(cudaMalloc(&B->ws.children, (size_t)B->grid * (POOL_MAX + FSP_MAX_JOBS) * s_max));
    TRYB(cudaMalloc(&B->ws.lbs, (size_t)B->grid * (POOL_MAX + FSP_MAX_JOBS) * sizeof(int32_t)));
    TRYB(cudaMemcpy(B->d_desc, B->desc.data(), sizeof(BatchDesc) * count, cudaMemcpyHostToDevice));
    TRYB(cudaMemcpy(B->d_p, p_flat, sizeof(int32_t) * off, cudaMemcpyHostToDevice));
#undef TRYB
    if ((rc = batch_capture(B)) != FSP_OK) goto fail;
    *out = B;
    return FSP_OK;
fail:
    batch_free(B);
    return rc;
}

extern "C" int fsp_batch_set_split(fsp_batch *B, int on)
{
    if (!B) { fsp_set_error("fsp_batch_set_split: NULL batch"); return FSP_ERR_ARG; }
    if (on && !B->d_item) {
        // the work items, the instances with the most jobs (the longest searches) first
        std::vector<int> order(B->count);
        for (int i = 0; i < B->count; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            return (long long)B->desc[a].n * B->desc[a].m > (long long)B->desc[b].n * B->desc[b].m;
        });
        std::vector<int> inst, job;
        for (int i : order) {
            if (B->desc[i].n <= 2) {  // the root's children are complete schedules: one item, the root
                inst.push_back(i);
                job.push_back(-1);
                continue;
            }
            for (int j = 0; j < B->desc[i].n; ++j) { inst.push_back(i); job.push_back(j); }
        }
        const int items = (int)inst.size();
        FSP_CUDA(cudaMalloc(&B->d_item, sizeof(int) * 2 * (size_t)items));
        FSP_CUDA(cudaMemcpy(B->d_item, inst.data(), sizeof(int) * items, cudaMemcpyHostToDevice));
        FSP_CUDA(cudaMemcpy(B->d_item + items, job.data(), sizeof(int) * items, cudaMemcpyHostToDevice));
        FSP_CUDA(cudaMalloc(&B->X.ub, sizeof(int) * B->count));
        FSP_CUDA(cudaMalloc(&B->X.key, sizeof(unsigned long long) * B->count));
        FSP_CUDA(cudaMalloc(&B->X.cnt, sizeof(long long) * 6 * B->count));
        FSP_CUDA(cudaMalloc(&B->X.flags, sizeof(int) * B->count));
        FSP_CUDA(cudaMalloc(&B->X.item_perm, (size_t)FSP_MAX_JOBS * items));
        B->X.item_inst = B->d_item;
        B->X.item_job = B->d_item + items;
        B->X.items = items;
    }
    B->split = on != 0;
    return batch_capture(B);
}

extern "C" void fsp_batch_destroy(fsp_batch *B)
{
    if (!B) return;
    cudaDeviceSynchronize();
    batch_free(B);
}

extern "C" int fsp_batch_run(fsp_batch *B, void *stream)
{
    if (!B) { fsp_set_error("fsp_batch_run: NULL batch"); return FSP_ERR_ARG; }
    FSP_CUDA(cudaGraphLaunch(B->exec, (cudaStream_t)stream));
    return FSP_OK;
}

extern "C" int fsp_batch_results(fsp_batch *B, fsp_batch_result *res, int32_t *perms, void *stream)
{
    if (!B || !res) { fsp_set_error("fsp_batch_results: NULL argument"); return FSP_ERR_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    FSP_CUDA(cudaStreamSynchronize(st));
    std::vector<BatchOut> o(B->count);
    FSP_CUDA(cudaMemcpy(o.data(), B->d_out, sizeof(BatchOut) * B->count, cudaMemcpyDeviceToHost));
    std::vector<uint8_t> pb;
    if (perms) {
        pb.resize((size_t)FSP_MAX_JOBS * B->count);
        FSP_CUDA(cudaMemcpy(pb.data(), B->d_perms, pb.size(), cudaMemcpyDeviceToHost));
    }
    for (int i = 0; i < B->count; ++i) {
        res[i].cmax = o[i].cmax;
        res[i].status = o[i].status;
        res[i].nodes_bounded = o[i].bounded;
        res[i].nodes_branched = o[i].branched;
        res[i].nodes_pruned = o[i].pruned;
        res[i].leaves = o[i].leaves;
        res[i].iterations = o[i].iterations;
        res[i].incumbent_updates = o[i].updates;
        res[i].pool = B->desc[i].pool;
        if (perms)
            for (int j = 0; j < B->desc[i].n; ++j) perms[(size_t)i * FSP_MAX_JOBS + j] = pb[(size_t)i * FSP_MAX_JOBS + j];
    }
    return FSP_OK;
}


// Pool size per shape on measured throughput: for each shape, up to `probe`
// of its instances run as a batch with each candidate pool and a node
// budget; the pool with the most nodes bounded per second wins.
extern "C" int fsp_batch_tune_pools(int count, const int32_t *shapes, const int32_t *p_flat, int64_t probe_budget,
                                    int64_t *pools_out)
{
    if (count < 1 || !shapes || !p_flat || !pools_out) { fsp_set_error("fsp_batch_tune_pools: invalid argument"); return FSP_ERR_ARG; }
    const int64_t cands[] = {128, 256, 512, 1024, 2048, 4096};
    std::vector<long long> off(count + 1, 0);
    for (int i = 0; i < count; ++i) off[i + 1] = off[i] + (long long)shapes[2 * i] * shapes[2 * i + 1];
    std::vector<int> done(count, 0);
    for (int i = 0; i < count; ++i) {
        if (done[i]) continue;
        std::vector<int> same;
        for (int j = i; j < count; ++j)
            if (shapes[2 * j] == shapes[2 * i] && shapes[2 * j + 1] == shapes[2 * i + 1]) same.push_back(j);
        const int probe = (int)(same.size() < 8 ? same.size() : 8);
        std::vector<int32_t> sh, pf;
        for (int q = 0; q < probe; ++q) {
            const int j = same[q];
            sh.push_back(shapes[2 * j]);
            sh.push_back(shapes[2 * j + 1]);
            pf.insert(pf.end(), p_flat + off[j], p_flat + off[j + 1]);
        }
        double best = -1.0;
        int64_t best_pool = 1024;
        for (int64_t c : cands) {
            std::vector<int64_t> pools(probe, c), budgets(probe, probe_budget);
            fsp_batch *B = nullptr;
            int rc = fsp_batch_create(probe, sh.data(), pf.data(), pools.data(), budgets.data(), nullptr, &B);
            if (rc != FSP_OK) return rc;
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            cudaEventRecord(e0, 0);
            rc = fsp_batch_run(B, 0);
            cudaEventRecord(e1, 0);
            std::vector<fsp_batch_result> r(probe);
            if (rc == FSP_OK) rc = fsp_batch_results(B, r.data(), nullptr, 0);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            fsp_batch_destroy(B);
            if (rc != FSP_OK) return rc;
            long long nodes = 0;
            for (auto &x : r) nodes += x.nodes_bounded;
            const double rate = ms > 0 ? nodes / (double)ms : 0.0;
            if (rate > best) { best = rate; best_pool = c; }
        }
        for (int j : same) { pools_out[j] = best_pool; done[j] = 1; }
    }
    return FSP_OK;
}
