// fsp_batch.cuh -- many instances of mixed shape in one persistent launch
// (device code; the host side is in fsp_batch.cu).
//
// Each CTA takes instance indices from a device work queue (one atomic
// counter) and solves each instance completely with CTA-local barriers only:
// per-instance tables built in shared memory, the NEH upper bound, then the
// same pool-synchronous depth-first search as fsp_solve (Sec. II-A
// operators, Sec. III pool of deepest nodes) on its own stack in global
// memory.  A per-instance pool size (tuned per shape on measured
// throughput) and node budget apply.  The queue reset and the persistent
// kernel are captured once in a CUDA graph and replayed.
#pragma once

#include <stdlib.h>
#include <string.h>

#include "fsp_family.cuh"

#define BB 256        // threads per CTA of the helper kernels and the default batch CTA
#define BB_MAX 640    // most threads of a batch CTA (20 warps; the block shape is chosen per shape)

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

struct BatchWs {  // per-CTA scratch in global memory (one slice per CTA of a class's launch)
    uint8_t *stack, *children;
    int32_t *lbs;
    unsigned long long *cta_ns;  // per CTA: the global timer (ns) when it started and when it left
    // split mode, donations between the CTAs of one launch: dq = {lock, slots in use (the
    // donated nodes waiting), donated items so far, CTAs waiting for work, items in progress
    // (donated nodes included)}; each slot holds a donated node
    // (instance, item id, record); donated item ids run from ids_base to ids_base + ids_cap
    int *dq;
    int *slot_inst, *slot_id;
    uint8_t *slot_rec;
    int slots, ids_base, ids_cap;
    int idle_cap;      // CTAs of the launch that may wait for donations at a time
    long long cap;     // records per stack
    long long ch_cap;  // children per iteration (the class's largest pool + n)
    int stride_max;
};

#define DQ_GIVE_TRIES 64                // a donor tries the lock this often, then donates later
#define DQ_TAKE_TRIES 1024              // a CTA taking a donated node: tries per look
#define DQ_WAIT_NS 1000000000ull        // every wait on the donations ends after 1 s of global time
#define DQ_GIVE_MAX 4                   // nodes a CTA donates per iteration at most

// Thread 0 only: the donation lock, taken within `tries` tries (false: not
// taken; the caller skips this donation or looks again).
__device__ __forceinline__ bool dq_lock(int *dq, int tries)
{
    for (int spin = 0; spin < tries; ++spin) {
        if (atomicCAS(dq, 0, 1) == 0) {
            __threadfence();
            return true;
        }
        __nanosleep(32);
    }
    return false;
}

__device__ __forceinline__ void dq_unlock(int *dq)
{
    __threadfence();
    atomicExch(dq, 0);
}

__device__ __forceinline__ unsigned long long b_globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Split mode: the work items are (instance, first job) pairs, the subtrees of
// the root; every CTA working on an instance shares its UB and counters.
struct BatchSplit {
    const int *item_inst, *item_job;  // per item
    int items;
    int *ub;                  // per instance: best makespan so far (atomicMin)
    unsigned long long *key;  // per instance: (best makespan << 32) | item that found it, ~0 = none
    long long *cnt;           // per instance: bounded, branched, pruned, leaves, iterations, updates
    int *flags;               // per instance: 1 = a node budget stopped an item, 2 = a stack filled up,
                              // 4 = a wait on the donations ran out with nodes waiting
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
        const int nw = (int)(blockDim.x >> 5);
        int t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        if (lane < nw) warp_tot[lane] = t;
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
    if (threadIdx.x == blockDim.x - 1) s_total = incl;
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
    int warp_tot[BB_MAX / 32];
    uint8_t inc[FSP_MAX_JOBS + 1], seq[FSP_MAX_JOBS + 1], ord[FSP_MAX_JOBS + 1];
    int32_t tot[FSP_MAX_JOBS + 1];
    unsigned long long best_key;
};

// Shared memory of a batch CTA of `warps` warps for an n x m instance: the
// family layout (fsp_family.cuh) for those warps, then the parents'
// first-child offsets.
__host__ __device__ inline size_t batch_smem_nm(int n, int m, bool bidir = false, int warps = BB / 32)
{
    const int mp = (m % 2 == 0) ? m + 1 : m, nv = (n + (bidir ? 2 : 1) + 15) / 16;
    return fsp_align16(family_smem_layout_nm(n, m, mp, m, nv, warps).bytes) + (size_t)(POOL_MAX / 2 + 4) * 4;
}

// NEH upper bound: jobs by decreasing total time, each inserted at the
// position of smallest partial makespan, earliest on ties; the sequence is
// left in sh.seq.  All threads of the CTA call it.
template <int MT>
__device__ int b_neh(const int32_t *__restrict__ p, int n, BatchShared &sh)
{
    const int tid = threadIdx.x, NT = (int)blockDim.x;
    uint8_t *seq = sh.seq, *ord = sh.ord;
    int32_t *tot = sh.tot;
    unsigned long long &best_key = sh.best_key;
    for (int j = tid; j < n; j += NT) {
        int32_t s = 0;
        for (int k = 0; k < MT; ++k) s += p[j * MT + k];
        tot[j] = s;
    }
    __syncthreads();
    for (int j = tid; j < n; j += NT) {
        int rank = 0;
        for (int i = 0; i < n; ++i) rank += (tot[i] > tot[j]) || (tot[i] == tot[j] && i < j);
        ord[rank] = (uint8_t)j;
    }
    __syncthreads();
    for (int len = 0; len < n; ++len) {
        const int job = ord[len];
        if (tid == 0) best_key = ~0ull;
        __syncthreads();
        for (int pos = tid; pos <= len; pos += NT) {
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
// BIDIR: bidirectional branching (records of n+2 bytes, fsp_bidir.cu).
template <int MT, int NV, int NW, bool SPLIT, bool BIDIR>
__device__ void b_solve(const int32_t *__restrict__ p, const BatchDesc &D, BatchOut *out, uint8_t *perm_out,
                        const BatchWs &W, unsigned char *smem, BatchShared &sh, const BatchSplit &X, int inst,
                        int item, int job, bool tables_ready, const uint8_t *start_rec = nullptr)
{
    const int n = D.n, tid = threadIdx.x, NT = (int)blockDim.x, NWP = NT >> 5;
    const int P = MT * (MT - 1) / 2, mp = (MT % 2 == 0) ? MT + 1 : MT;
    const int stride = (n + (BIDIR ? 2 : 1) + 15) / 16 * 16;
    const FamSmem L = family_smem_layout_nm(n, MT, mp, MT, NV, NWP);
    const FamView V = fam_view(smem, L, tid >> 5);
    int2 *pq_s = V.pq;
    int *poff = reinterpret_cast<int *>(smem + fsp_align16(L.bytes));
    int *warp_tot = sh.warp_tot;
    uint8_t *inc = sh.inc, *seq = sh.seq;
    unsigned long long &best_key = sh.best_key;

    // tables: {p, tail} rows and the Johnson entries of every pair
    if (!SPLIT || !tables_ready) {
    for (int i = tid; i < n * MT; i += NT) {
        const int j = i / MT, k = i - j * MT;
        int32_t q = 0;
        for (int h = k + 1; h < MT; ++h) q += p[j * MT + h];
        pq_s[j * mp + k] = make_int2(p[i], q);
    }
    for (int e = tid; e < P * n; e += NT) {
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
        for (int i = tid; i < n; i += NT) inc[i] = seq[i];
    }
    __syncthreads();

    // the search
    long long bounded = 0, branched = 0, pruned = 0, leaves = 0, iters = 0, updates = 0;
    int status = FSP_OK;
    long long S = 1, bot = 0;  // the stack holds records bot..S-1 (bot rises as bottom nodes are donated)
    if (SPLIT && start_rec) {  // a node another CTA donated
        for (int i = tid; i < stride; i += NT) W.stack[i] = start_rec[i];
    } else if (SPLIT && job >= 0) {  // the root's child that schedules `job` first (the rest in increasing order)
        for (int i = tid; i < stride; i += NT)
            W.stack[i] = (uint8_t)(i == 0 ? job : i < n ? (i - 1 < job ? i - 1 : i) : i == n ? 1 : 0);
    } else {
        for (int i = tid; i < stride; i += NT) W.stack[i] = (uint8_t)(i < n ? i : 0);
    }
    bool improved = false;
    __shared__ int s_ub, s_give;
    __syncthreads();
    const int pool = D.pool;
    const int warp = tid >> 5, lane = tid & 31;
    while (S > bot) {
        if (SPLIT) {  // the instance's UB and node count, as the other CTAs left them
            if (tid == 0) {
                s_ub = min(ub, *(volatile int *)&X.ub[inst]);
                if (D.budget > 0 && *(volatile long long *)&X.cnt[6 * inst] >= D.budget) s_ub = -1;
                // CTAs waiting for work take the bottom nodes (the shallowest: the largest
                // subtrees left), while this CTA keeps at least one node
                s_give = 0;
                const int idle = *(volatile int *)&W.dq[3];
                if (s_ub >= 0 && idle > 0 && S - bot >= 2 && dq_lock(W.dq, DQ_GIVE_TRIES)) {
                    int give = min(min(idle, DQ_GIVE_MAX), (int)(S - bot - 1));
                    for (; s_give < give; ++s_give) {
                        const int top = *(volatile int *)&W.dq[1], seq = *(volatile int *)&W.dq[2];
                        if (top >= W.slots || seq >= W.ids_cap) break;
                        W.slot_inst[top] = inst;
                        W.slot_id[top] = W.ids_base + seq;
                        const uint4 *src = reinterpret_cast<const uint4 *>(W.stack + (bot + s_give) * stride);
                        uint4 *dst = reinterpret_cast<uint4 *>(W.slot_rec + (size_t)top * W.stride_max);
                        for (int v = 0; v < stride / 16; ++v) dst[v] = src[v];
                        *(volatile int *)&W.dq[1] = top + 1;
                        *(volatile int *)&W.dq[2] = seq + 1;
                    }
                    dq_unlock(W.dq);
                }
            }
            __syncthreads();
            const int u = s_ub;
            bot += s_give;
            __syncthreads();
            if (u < 0) { status = FSP_INCOMPLETE; break; }
            if (S == bot) break;
            ub = u;
        } else if (D.budget > 0 && bounded >= D.budget) {
            status = FSP_INCOMPLETE;
            break;
        }
        // selection: deepest parents while their children fit (at least one)
        const long long cand = S - bot < pool ? S - bot : pool;
        long long running = 0, np = 0;
        for (long long base = 0; base < cand; base += (long long)NT * SEL_Q) {
            int r[SEL_Q], tsum = 0;
#pragma unroll
            for (int q = 0; q < SEL_Q; ++q) {
                const long long i = base + (long long)tid * SEL_Q + q;
                const uint8_t *rec = W.stack + (S - 1 - i) * stride;
                r[q] = i < cand ? n - (int)rec[n] - (BIDIR ? (int)rec[n + 1] : 0) : 0;
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
            if (ct < NT * SEL_Q) break;
        }
        const long long nch = running;
        if (tid == 0) poff[np] = (int)nch;
        if (S - np + nch > W.cap) { status = FSP_ERR_CAPACITY; break; }
        if (tid == 0) best_key = ~0ull;
        __syncthreads();
        // branching + bounding: each warp bounds a parent's children together
        for (long long f = warp; f < np; f += NWP) {
            if (lane < NV)
                reinterpret_cast<uint4 *>(V.recb)[lane] =
                    reinterpret_cast<const uint4 *>(W.stack + (S - 1 - f) * stride)[lane];
            __syncwarp();
            int fc[4] = {0, 0, 0, 0};  // not reported by the batch
            fam_bound<MT, NV, false, false, BIDIR>(V, V.recb, poff[f], n, mp, stride, ub, W.children, W.lbs,
                                                   &best_key, 0, 0, nullptr, fc);
            __syncwarp();
        }
        __syncthreads();
        const unsigned long long bk = best_key;
        const int ub_new = (bk != ~0ull && (int)(bk >> 32) < ub) ? (int)(bk >> 32) : ub;
        if (ub_new < ub) {
            const long long idx = (long long)(bk & 0xffffffffull);
            for (int i = tid; i < n; i += NT) inc[i] = W.children[idx * stride + i];
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
        auto depth = [&](long long c) {
            const uint8_t *ch = W.children + c * stride;
            return (int)ch[n] + (BIDIR ? (int)ch[n + 1] : 0);
        };
        for (long long c = tid; c < nch; c += NT) {
            const bool leaf = depth(c) == n - 1;
            my_l += leaf;
            my_s += !leaf && W.lbs[c] < ub;
        }
        const int total = b_block_sum(my_s, warp_tot), nleaf = b_block_sum(my_l, warp_tot);
        const long long base_s = S - np;
        long long done = 0;
        for (long long c0 = 0; c0 < nch; c0 += NT) {
            const long long c = c0 + tid;
            const bool surv = c < nch && depth(c) != n - 1 && W.lbs[c] < ub;
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
            for (int i = tid; i < n; i += NT) X.item_perm[(size_t)item * FSP_MAX_JOBS + i] = inc[i];
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
    for (int i = tid; i < n; i += NT) perm_out[i] = inc[i];
    __syncthreads();
}

// The persistent kernels.  A launch serves one class of instances (one shape
// and block shape): the queue hands out positions 0..len-1 of `list`, which
// holds the class's instance indices (whole instances) or item indices (split
// mode); W is the class's scratch, one slice per CTA.
template <bool BIDIR>
__global__ void __launch_bounds__(BB_MAX) k_batch(const BatchDesc *__restrict__ desc, const int *__restrict__ list,
                                                  int len, const int32_t *__restrict__ p_flat, BatchOut *out,
                                                  uint8_t *perms, int *queue, BatchWs W)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_inst;
    __shared__ BatchShared sh;
    BatchWs w = W;
    w.stack = W.stack + (size_t)blockIdx.x * W.cap * W.stride_max;
    w.children = W.children + (size_t)blockIdx.x * W.ch_cap * W.stride_max;
    w.lbs = W.lbs + (size_t)blockIdx.x * W.ch_cap;
    if (threadIdx.x == 0) W.cta_ns[2 * blockIdx.x] = b_globaltimer();
    for (;;) {
        if (threadIdx.x == 0) s_inst = atomicAdd(queue, 1);
        __syncthreads();
        const int q = s_inst;
        __syncthreads();
        if (q >= len) break;
        const int i = list[q];
        const BatchDesc D = desc[i];
        const int32_t *p = p_flat + D.p_off;
        const int nv = (D.n + (BIDIR ? 2 : 1) + 15) / 16, nw = D.n <= 32 ? 1 : 2;
        uint8_t *po = perms + (size_t)i * FSP_MAX_JOBS;
#define B_CASE(MT_, NV_, NW_)                                                                               \
    if (D.m == MT_ && nv == NV_ && nw == NW_) {                                                             \
        b_solve<MT_, NV_, NW_, false, BIDIR>(p, D, out + i, po, w, smem, sh, BatchSplit{}, i, 0, 0, false); \
        continue;                                                                                           \
    }
        FSP_SHAPES_BATCH(B_CASE)
#undef B_CASE
        if (threadIdx.x == 0) out[i].status = FSP_ERR_ARG;  // shape without a kernel (checked on the host)
    }
    if (threadIdx.x == 0) W.cta_ns[2 * blockIdx.x + 1] = b_globaltimer();
}

// Thread 0 only: takes the donated node on top of the donation stack (under
// the lock, within DQ_TAKE_TRIES tries) as the CTA's next item and counts it
// in progress; returns whether the stack was looked at under the lock (taken,
// or found empty).
__device__ __forceinline__ bool dq_take(const BatchWs &W, int &item, int &inst, int &job, uint8_t *rec)
{
    if (!dq_lock(W.dq, DQ_TAKE_TRIES)) return false;
    const int top = *(volatile int *)&W.dq[1];
    if (top > 0) {
        const int sl = top - 1;
        *(volatile int *)&W.dq[1] = sl;
        atomicAdd(&W.dq[4], 1);
        item = __ldcg(W.slot_id + sl);
        inst = __ldcg(W.slot_inst + sl);
        job = -2;
        const uint4 *src = reinterpret_cast<const uint4 *>(W.slot_rec + (size_t)sl * W.stride_max);
        for (int v = 0; v < W.stride_max / 16; ++v) reinterpret_cast<uint4 *>(rec)[v] = __ldcg(src + v);
    }
    dq_unlock(W.dq);
    return true;
}

// Split mode: the persistent kernel over the work items, then over the nodes
// the other CTAs donate; a CTA keeps the tables of the instance it last
// worked on (the items of an instance are consecutive in the list).
// No donated node is left behind: a CTA that finishes an item first takes
// the donated nodes still waiting (whoever donated them), one by one, and
// counts the item done only when it has seen the donation stack empty, so a
// donor is among the CTAs that look after its own donations.  If the lock
// stays taken for DQ_WAIT_NS while nodes wait, the instance is flagged (its
// status becomes FSP_ERR_TIMEOUT: its result may miss a subtree).  With no
// item left, a CTA waits for a donation (at most W.idle_cap at a time, each
// for at most DQ_WAIT_NS) and leaves once no item is in progress and no
// donated node waits; leaving early costs a helper, never a node.
template <bool BIDIR>
__global__ void __launch_bounds__(BB_MAX) k_batch_split(const BatchDesc *__restrict__ desc,
                                                        const int *__restrict__ list, int len,
                                                        const int32_t *__restrict__ p_flat, int *queue, BatchWs W,
                                                        BatchSplit X)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item, s_inst, s_job;
    __shared__ __align__(16) uint8_t s_rec[FSP_MAX_JOBS + 17];
    __shared__ BatchShared sh;
    BatchWs w = W;
    w.stack = W.stack + (size_t)blockIdx.x * W.cap * W.stride_max;
    w.children = W.children + (size_t)blockIdx.x * W.ch_cap * W.stride_max;
    w.lbs = W.lbs + (size_t)blockIdx.x * W.ch_cap;
    if (threadIdx.x == 0) W.cta_ns[2 * blockIdx.x] = b_globaltimer();
    int cur = -1;
    bool next = false;  // thread 0: the end of the last item took a donated node
    for (;;) {
        if (threadIdx.x == 0 && !next) {
            s_item = -1;
            const int q = atomicAdd(queue, 1);
            if (q < len) {
                atomicAdd(&W.dq[4], 1);  // an item in progress
                s_item = list[q];
                s_inst = X.item_inst[s_item];
                s_job = X.item_job[s_item];
            } else if (atomicAdd(&W.dq[3], 1) < W.idle_cap) {  // wait for a donated node
                const unsigned long long t0 = b_globaltimer();
                while (b_globaltimer() - t0 < DQ_WAIT_NS) {
                    if (*(volatile int *)&W.dq[1] > 0 && dq_take(W, s_item, s_inst, s_job, s_rec) && s_item >= 0)
                        break;
                    if (*(volatile int *)&W.dq[4] == 0 && *(volatile int *)&W.dq[1] == 0) break;  // no work left
                    __nanosleep(256);
                }
                atomicSub(&W.dq[3], 1);
            } else {
                atomicSub(&W.dq[3], 1);
            }
        }
        __syncthreads();
        const int item = s_item;
        if (item < 0) break;
        const int i = s_inst, job = s_job;
        const BatchDesc D = desc[i];
        const int32_t *p = p_flat + D.p_off;
        const int nv = (D.n + (BIDIR ? 2 : 1) + 15) / 16, nw = D.n <= 32 ? 1 : 2;
        const bool ready = cur == i;
        cur = i;
        const uint8_t *start = job == -2 ? s_rec : nullptr;
        bool done = false;
#define B_CASE(MT_, NV_, NW_)                                                                                  \
    if (!done && D.m == MT_ && nv == NV_ && nw == NW_) {                                                       \
        b_solve<MT_, NV_, NW_, true, BIDIR>(p, D, nullptr, nullptr, w, smem, sh, X, i, item, job, ready, start); \
        done = true;                                                                                           \
    }
        FSP_SHAPES_BATCH(B_CASE)
#undef B_CASE
        if (!done) cur = -1;
        __syncthreads();
        if (threadIdx.x == 0) {
            // the donated nodes still waiting come first (the next item, if one
            // is taken, is counted in progress before this one is counted done)
            next = false;
            s_item = -1;
            const unsigned long long t0 = b_globaltimer();
            while (*(volatile int *)&W.dq[1] > 0) {
                if (dq_take(W, s_item, s_inst, s_job, s_rec)) {
                    next = s_item >= 0;
                    break;
                }
                if (b_globaltimer() - t0 >= DQ_WAIT_NS) {
                    atomicOr(&X.flags[i], 4);
                    break;
                }
            }
            atomicSub(&W.dq[4], 1);  // the item is done
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) W.cta_ns[2 * blockIdx.x + 1] = b_globaltimer();
}
