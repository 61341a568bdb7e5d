// fsp_solve.cu -- the exact branch-and-bound on the device (Sec. II-A
// operators; Sec. III selection of a pool of the deepest pending nodes).
//
// The paper selects, branches and eliminates on the host and off-loads only
// the bounding (Sec. III).  Here every operator runs on the device and the
// host only launches one iteration after another:
//   K-select  one CTA: pops the deepest parents (top of the depth-first
//             stack) while their children fit in the pool; writes the
//             parents' first-child offsets.
//   K2+K1     one thread per child: builds the child record (prefix + job,
//             remaining set kept in increasing job order) and bounds it;
//             complete schedules race for the incumbent with one 64-bit
//             atomicMin on (bound, child index), which is the first child
//             in pool order among the smallest bounds.
//   K3a       per block: survivors (non-leaf, bound < new UB) and leaves.
//   K3b       stable compaction: survivors pushed in reverse pool order so
//             the first survivor is on top; counters, trace, incumbent.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <mutex>
#include <type_traits>

#include "fsp_family.cuh"

#define SOLVE_B 256        // threads per block of the per-child kernels
#define SELECT_B 1024      // threads of the selection CTA
#define SOLVE_RB 512       // one read-back: the control block (256 bytes), then the incumbent
static_assert(sizeof(SolveCtl) <= 256, "the incumbent follows the control block at byte 256");
static_assert(2 * SOLVE_RB <= FSP_PINNED_BYTES, "two read-back slots per pinned buffer");

struct SolveLayout {
    long long pool_max, max_children, cap, trace_cap, max_parents;
    int max_blocks, topk;
    bool learned;
    size_t off_ctl, off_stack, off_cum, off_iblk, off_children, off_lbs, off_poff, off_blk, off_inc, off_trace, bytes;
    size_t off_list, off_px, off_pscore, off_topk;
};

int fsp_mlp_dims(const fsp_mlp *M, int *F, int *H, int *P);
int fsp_mlp_topk_parents(fsp_mlp *M, const fsp_instance *I, const uint8_t *stack, const long long *s_pop,
                         const long long *n_parents, long long max_parents, int K, int16_t *topk, cudaStream_t st);
int fsp_mlp_forward_dev(fsp_mlp *M, const float *X, const long long *Bdev, int64_t Bmax, float *scores,
                        cudaStream_t st);

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Largest pool the tuner may try: SMs x 2048 resident threads (Sec. III).
static long long tuner_max_pool(const fsp_instance *I) { return (long long)I->sm_count * 2048; }

// Bytes per stack record: forward records, or bidirectional ones (perm, d1, d2).
static int rec_stride(const fsp_instance *I, const fsp_options *o)
{
    return o->branching == FSP_BRANCH_BIDIR ? fsp_node_stride_bidir(I->n) : I->stride;
}

static int solve_layout(const fsp_instance *I, const fsp_options *o, SolveLayout *L)
{
    if (o->branching != FSP_BRANCH_FORWARD && o->branching != FSP_BRANCH_BIDIR) {
        fsp_set_error("unknown branching %d", o->branching);
        return FSP_ERR_ARG;
    }
    const int rs = rec_stride(I, o);
    long long pool = o->pool_size == 0 ? tuner_max_pool(I) : o->pool_size;
    if (pool < 1 || pool > (1LL << 26)) {
        fsp_set_error("pool_size %lld outside 1..2^26", pool);
        return FSP_ERR_ARG;
    }
    long long pmax = pool;
    if (o->schedule && o->schedule_len > 0)
        for (long long i = 0; i < o->schedule_len; ++i) {
            if (o->schedule[i] < 1 || o->schedule[i] > (1LL << 26)) {
                fsp_set_error("schedule[%lld] = %lld outside 1..2^26", i, o->schedule[i]);
                return FSP_ERR_ARG;
            }
            if (o->schedule[i] > pmax) pmax = o->schedule[i];
        }
    L->pool_max = pmax;
    L->max_children = pmax + I->n;
    L->max_blocks = (int)((L->max_children + SOLVE_B - 1) / SOLVE_B);
    const long long init = (o->init_nodes && o->init_count > 0) ? o->init_count : 0;
    L->cap = o->stack_capacity > 0 ? o->stack_capacity : init + (long long)I->n * (pmax + I->n);
    L->trace_cap = (o->trace && o->trace_cap > 0) ? o->trace_cap : 0;
    size_t off = 0;
    L->off_ctl = off; off = align256(off + sizeof(SolveCtl));
    L->off_inc = off; off = align256(off + 256);  // right after the control block: one read-back
    L->off_stack = off; off = align256(off + (size_t)L->cap * rs);
    L->off_cum = off; off = align256(off + (size_t)L->cap * 8);
    L->off_iblk = off; off = align256(off + (size_t)((init + 255) / 256 + 1) * 8);
    L->off_children = off; off = align256(off + (size_t)L->max_children * rs);
    L->off_lbs = off; off = align256(off + (size_t)L->max_children * 4);
    L->off_poff = off; off = align256(off + (size_t)(L->max_children + 2) * 4);
    L->off_blk = off; off = align256(off + (size_t)L->max_blocks * 12);
    L->off_trace = off; off = align256(off + (size_t)L->trace_cap * 32);
    L->learned = o->order == FSP_ORDER_LEARNED;
    L->topk = o->topk > 0 ? o->topk : 4;
    L->max_parents = pmax / 2 + 2;  // stacked nodes have depth <= n-2: >= 2 children each
    L->off_list = L->off_px = L->off_pscore = L->off_topk = off;
    if (L->learned) {
        if (o->order != FSP_ORDER_LEARNED || !o->model || L->topk > 8) {
            fsp_set_error("learned order needs a model and 1 <= topk <= 8");
            return FSP_ERR_ARG;
        }
        int F = 0, H = 0, P = 0;
        fsp_mlp_dims(o->model, &F, &H, &P);
        if (F != 2 * I->m + 1 || P != I->P) {
            fsp_set_error("model has %d inputs and %d outputs; this instance needs %d and %d", F, P,
                          2 * I->m + 1, I->P);
            return FSP_ERR_ARG;
        }
        L->off_list = off; off = align256(off + (size_t)L->max_children * 4);
        L->off_px = off; off = align256(off + (size_t)L->max_parents * F * 4);
        L->off_pscore = off; off = align256(off + (size_t)L->max_parents * P * 4);
        L->off_topk = off; off = align256(off + (size_t)L->max_parents * L->topk * 2);
    } else if (o->order != FSP_ORDER_PLAIN) {
        fsp_set_error("unknown order %d", o->order);
        return FSP_ERR_ARG;
    }
    L->bytes = off;
    return FSP_OK;
}

extern "C" int64_t fsp_solve_workspace_bytes(const fsp_instance *I, const fsp_options *opt)
{
    if (!I) { fsp_set_error("fsp_solve_workspace_bytes: inst is NULL"); return FSP_ERR_ARG; }
    fsp_options d;
    if (!opt) { fsp_default_options(&d); opt = &d; }
    SolveLayout L;
    int rc = solve_layout(I, opt, &L);
    return rc == FSP_OK ? (int64_t)L.bytes : (int64_t)rc;
}

// ---------------------------------------------------------------- kernels --

__global__ void k_solve_init(SolveWs ws, int n, int stride, int ub0)
{
    const int t = threadIdx.x;
    for (int i = t; i < stride; i += blockDim.x) ws.stack[i] = (uint8_t)(i < n ? i : 0);
    if (t == 0) {
        ws.cum[0] = n;
        SolveCtl c;
        memset(&c, 0, sizeof c);
        c.stack_size = 1;
        c.ub = ub0;
        c.ub_iter = ub0;
        c.best_key = ~0ull;
        *ws.ctl = c;
    }
}

// Start from caller records: validate each (a permutation, depth <= n-2) and
// re-sort its remaining part by job index, the order branching relies on.
// n <= 63: the record and the job masks stay in registers (32-bit masks up to
// two 16-byte words, n <= 31); the record is read from `src` (the caller's
// buffer, or the stack itself) and written to `dst` on the stack.  The n jobs
// form a permutation iff all are below n and their bits number n; a remaining
// part already in increasing order is kept as it is.
__device__ __forceinline__ int init_popc(uint32_t x) { return __popc(x); }
__device__ __forceinline__ int init_popc(unsigned long long x) { return __popcll(x); }
__device__ __forceinline__ int init_low(uint32_t x) { return __ffs((int)x) - 1; }
__device__ __forceinline__ int init_low(unsigned long long x) { return __ffsll((long long)x) - 1; }

template <int NV>
__device__ __forceinline__ bool init_node_fast(FspRec<NV> &rec, bool same, uint8_t *dst, int n, int d)
{
    typedef typename std::conditional<(NV <= 2), uint32_t, unsigned long long>::type M;
    bool ok = d <= n - 2, sorted = true;
    M seen = 0, rem = 0;
    int prev = -1;
    // word by word; the words past the n-th byte are skipped (n is the same
    // for every thread, so the exit is uniform)
#pragma unroll
    for (int q = 0; q < 4 * NV; ++q) {
        if (4 * q >= n) break;
        const uint32_t w = rec.w[q];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = 4 * q + b;
            if (i < n) {
                const int j = (int)((w >> (8 * b)) & 0xFFu);
                ok &= j < n;
                const M bit = j < n ? (M)1 << j : (M)0;
                seen |= bit;
                if (i >= d) {
                    rem |= bit;
                    sorted &= j > prev;
                    prev = j;
                }
            }
        }
    }
    if (!ok || init_popc(seen) != n) return false;
    if (sorted) {
        if (!same) fsp_store_rec(rec, dst);
        return true;
    }
#pragma unroll
    for (int q = 0; q < 4 * NV; ++q) {  // positions d..n-1: the remaining jobs in increasing order
        if (4 * q >= n) break;
        if (4 * q + 3 < d) continue;
        uint32_t w = rec.w[q];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = 4 * q + b;
            if (i >= d && i < n) {
                const int j = init_low(rem);
                rem &= rem - (M)1;
                w = (w & ~(0xFFu << (8 * b))) | ((uint32_t)j << (8 * b));
            }
        }
        rec.w[q] = w;
    }
    fsp_store_rec(rec, dst);
    return true;
}

__device__ __forceinline__ int block_incl_scan(int v, int *warp_tot);

// One thread per start record: the control block, the record validated and
// copied (or re-sorted in place when src is the stack), its children summed
// over the block's records up to it (cum[], completed by k_init_cum with the
// blocks before), and the children of each block of 256 records.  A block
// with a malformed record writes -1 there instead and k_init_cum, launched
// after this kernel has set up the control block, raises the status; the
// first selection then does nothing.
template <int NV>
__global__ void __launch_bounds__(SOLVE_B, 8) k_solve_init_nodes(SolveWs ws, const uint8_t *src, int n, int stride,
                                                              long long count, int ub0, int wide)
{
    __shared__ int warp_tot[32];
    // the block's records, copied with coalesced 16-byte loads (each warp
    // instruction reads 512 contiguous bytes, which matters when src is pinned
    // host memory read over the host link); a record stride of 16 (NV | 1)
    // bytes keeps each thread's 16-byte reads of its own record conflict-free
    constexpr int SS = 16 * (NV | 1);
    __shared__ __align__(16) uint8_t recs[SOLVE_B * SS];
    pdl_launch_dependents();
    const long long t = (long long)blockIdx.x * SOLVE_B + threadIdx.x;
    if (!wide) {
        const long long first = (long long)blockIdx.x * SOLVE_B;
        const long long nrec = count - first < SOLVE_B ? count - first : SOLVE_B;
        const uint4 *g = reinterpret_cast<const uint4 *>(src + first * stride);
        for (int c = threadIdx.x; c < nrec * NV; c += SOLVE_B)
            *reinterpret_cast<uint4 *>(recs + (c / NV) * SS + (c % NV) * 16) = __ldg(g + c);
        __syncthreads();
    }
    if (t == 0) {
        SolveCtl c;
        memset(&c, 0, sizeof c);
        c.stack_size = count;
        c.best_key = ~0ull;
        c.ub = ub0;
        c.ub_iter = ub0;
        *ws.ctl = c;
    }
    int d = 0;
    bool bad = false;
    if (t < count) {
        if (!wide) {  // records of n >= 64 jobs: k_solve_init_nodes_wide, on the stack
            const uint8_t *mine = recs + threadIdx.x * SS;
            d = mine[n];  // a byte read: no run-time index into the record's registers
            FspRec<NV> rec;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const uint4 x = reinterpret_cast<const uint4 *>(mine)[v];
                rec.w[4 * v + 0] = x.x;
                rec.w[4 * v + 1] = x.y;
                rec.w[4 * v + 2] = x.z;
                rec.w[4 * v + 3] = x.w;
            }
            bad = !init_node_fast<NV>(rec, src == ws.stack, ws.stack + t * stride, n, d);
        } else {
            d = src[t * stride + n];
        }
    }
    const int incl = block_incl_scan(t < count ? n - d : 0, warp_tot);
    if (t < count) ws.cum[t] = incl;
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) ws.iblk[blockIdx.x] = bad ? -1 : warp_tot[SOLVE_B / 32 - 1];
}

// The same for n >= 64 (records of 80 bytes or more): masks of 8 words.
__global__ void k_solve_init_nodes_wide(SolveWs ws, int n, int stride, long long count)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    uint8_t *r = ws.stack + t * stride;
    const int d = r[n];
    uint32_t seen[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint32_t rem[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    bool bad = d > n - 2;
    for (int i = 0; i < n; ++i) {
        const int j = r[i];
        if (j >= n) { bad = true; continue; }
        const uint32_t bit = 1u << (j & 31);
        if (seen[j >> 5] & bit) bad = true;
        seen[j >> 5] |= bit;
        if (i >= d) rem[j >> 5] |= bit;
    }
    if (bad) {
        atomicExch(&ws.ctl->status, FSP_ERR_ARG);
        return;
    }
    int o = d;
    for (int w = 0; w < 8; ++w) {
        uint32_t x = rem[w];
        while (x) {
            const int b = __ffs(x) - 1;
            x &= x - 1;
            r[o++] = (uint8_t)(w * 32 + b);
        }
    }
}

// n == 1: the only schedule; its makespan is the sum of the job's times.
__global__ void k_solve_single(SolveWs ws, const int32_t *p, int m, int ub0)
{
    if (threadIdx.x != 0) return;
    int32_t c = 0;
    for (int k = 0; k < m; ++k) c += p[k];
    SolveCtl *ctl = ws.ctl;
    memset(ctl, 0, sizeof(SolveCtl));
    ctl->ub = ub0;
    if (c < ub0) {
        ctl->ub = c;
        ctl->cnt[5] = 1;
        ws.inc[0] = 0;
    }
}

// Sum of one long long per thread over the block (blockDim.x = SOLVE_B).
__device__ __forceinline__ long long block_sum_ll(long long v, long long *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    long long s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    __syncthreads();
    return s;
}

// Running children counts of the start records (stack order): each block of
// 256 records adds the children of the blocks before it (summed by
// k_solve_init_nodes) to its records' prefixes within the block.  Up to
// INIT_SCAN_BLOCKS blocks each block sums the blocks before it itself; above,
// k_init_scan first turns the block sums into exclusive prefixes (scanned = 1).
#define INIT_SCAN_BLOCKS 2048

__global__ void __launch_bounds__(SOLVE_B) k_init_cum(SolveWs ws, int n, int stride, long long count, int scanned)
{
    __shared__ long long red[SOLVE_B / 32];
    pdl_launch_dependents();
    pdl_wait();
    long long before = 0;
    if (scanned) {
        before = ws.iblk[blockIdx.x];
    } else {
        for (int i = threadIdx.x; i < (int)blockIdx.x; i += SOLVE_B) before += ws.iblk[i];
        before = block_sum_ll(before, red);
        if (threadIdx.x == 0 && ws.iblk[blockIdx.x] < 0) atomicExch(&ws.ctl->status, FSP_ERR_ARG);
    }
    const long long t = (long long)blockIdx.x * SOLVE_B + threadIdx.x;
    if (t < count) ws.cum[t] += before;
}

// One CTA: exclusive prefix sums of the nb block sums, in place; a block
// marked malformed (-1) raises the status.
__global__ void __launch_bounds__(1024) k_init_scan(SolveWs ws, long long nb)
{
    __shared__ long long part[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long carry = 0;
    bool bad = false;
    for (long long base = 0; base < nb; base += 1024) {
        const long long i = base + threadIdx.x;
        long long v = i < nb ? ws.iblk[i] : 0;
        if (v < 0) { bad = true; v = 0; }
        long long x = v;  // inclusive warp scan
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += u;
        }
        if (lane == 31) part[wid] = x;
        __syncthreads();
        if (wid == 0) {
            long long w = part[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long u = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += u;
            }
            part[lane] = w;  // inclusive over warps
        }
        __syncthreads();
        const long long incl = x + (wid > 0 ? part[wid - 1] : 0);
        if (i < nb) ws.iblk[i] = carry + incl - v;
        carry += part[31];
        __syncthreads();
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(&ws.ctl->status, FSP_ERR_ARG);
}

// Inclusive block scan of one int per thread (blockDim.x a multiple of 32).
__device__ __forceinline__ int block_incl_scan(int v, int *warp_tot)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) warp_tot[wid] = v;
    __syncthreads();
    if (wid == 0) {
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

// Selection (Sec. III): deepest pending nodes first, while their children fit.
// cum[] holds the running children counts of the stack, so the children of
// the top i records are cum[S-1] - cum[S-1-i]: the number of parents is the
// largest i <= min(S, pool) whose children fit the pool (at least one),
// found by a parallel search that narrows the interval SELECT_B-fold per
// round.  The parents' first-child offsets follow from cum directly: written
// to poff for the per-child kernels (write_poff), read from cum by the family
// kernel itself.
__global__ void __launch_bounds__(SELECT_B) k_select(SolveWs ws, int n, int stride, long long pool,
                                                    long long budget, long long max_it, int write_poff)
{
    pdl_launch_dependents();  // the bounding kernel stages its tables meanwhile
    pdl_wait();
    SolveCtl *ctl = ws.ctl;
    const long long S = ctl->stack_size;
    // nothing to do: an error (a malformed start record), an empty stack, or
    // a stop the host reads one iteration later (node budget, iteration cap)
    if (ctl->status != 0 || S == 0 || (budget > 0 && ctl->cnt[0] >= budget) ||
        (max_it > 0 && ctl->cnt[4] >= max_it)) {
        if (threadIdx.x == 0) {
            ctl->n_parents = 0;
            ctl->n_children = 0;
            ctl->s_pop = S;
            ctl->n_list = 0;
            ctl->early = 0;
            ctl->fam_next = 0;
            ctl->best_key = ~0ull;
            ctl->ub_iter = ctl->ub;
            ws.poff[0] = 0;
        }
        return;
    }
    const long long cand = S < pool ? S : pool;
    const long long top = ws.cum[S - 1];
    // children of the top i records, 0 <= i <= S
    auto prefix = [&](long long i) -> long long { return top - (i < S ? ws.cum[S - 1 - i] : 0); };
    // every i <= lo is taken (lo = 1 always is); no i >= hi fits or exists
    long long lo = 1, hi = cand + 1;
    while (hi - lo > 1) {
        const long long step = (hi - lo + SELECT_B - 1) / SELECT_B;
        const long long i = lo + (long long)(threadIdx.x + 1) * step;
        const int c = __syncthreads_count(i < hi && prefix(i) <= pool);
        lo += (long long)c * step;
        hi = min(hi, lo + step);
    }
    const long long np = lo;
    const long long running = prefix(np);
    if (write_poff)
        for (long long i = threadIdx.x; i <= np; i += SELECT_B) ws.poff[i] = (int)prefix(i);
    if (threadIdx.x == 0) {
        ctl->n_list = 0;
        ctl->early = 0;
        ctl->fam_next = 0;
        ctl->best_key = ~0ull;
        ctl->ub_iter = ctl->ub;
        if (S - np + running > ws.cap) {  // could overflow: keep the stack intact
            ctl->status = FSP_ERR_CAPACITY;
            ctl->n_parents = 0;
            ctl->n_children = 0;
            ctl->s_pop = S;
        } else {
            ctl->n_parents = np;
            ctl->n_children = running;
            ctl->s_pop = S - np;
        }
    }
}


// Branching + bounding, one thread per child.
template <int NW, int MT, bool ES>
__global__ void __launch_bounds__(256) k_branch_bound(DevInst I, SolveWs ws, BoundSmem L)
{
    const SolveCtl *ctl = ws.ctl;
    const long long nch = ctl->n_children;
    const int B = blockDim.x, tid = threadIdx.x;
    if ((long long)blockIdx.x * B >= nch) return;
    extern __shared__ __align__(16) unsigned char smem[];
    FspEntry *ent_s = ES ? reinterpret_cast<FspEntry *>(smem + L.ent_off) : nullptr;
    int32_t *p_s = reinterpret_cast<int32_t *>(smem + L.p_off);
    int32_t *q_s = reinterpret_cast<int32_t *>(smem + L.q_off);
    uint32_t *rec = reinterpret_cast<uint32_t *>(smem + L.rec_off) + tid;
    int32_t *cs = reinterpret_cast<int32_t *>(smem + L.cs_off) + tid;
    int32_t *sq = reinterpret_cast<int32_t *>(smem + L.sq_off) + tid;
    int32_t *ss = reinterpret_cast<int32_t *>(smem + L.ss_off) + tid;
    fsp_stage_tables(I, ent_s, p_s, q_s);
    const FspEntry *ent = ES ? ent_s : I.ent;

    const long long c = (long long)blockIdx.x * B + tid;
    if (c >= nch) return;
    const int n = I.n, stride = I.stride, nvec = stride >> 4;
    const int np = (int)ctl->n_parents;
    const int pi = solve_parent_of(ws.poff, np, c);
    const long long S = ctl->s_pop + np;
    const uint4 *src = reinterpret_cast<const uint4 *>(ws.stack + (S - 1 - pi) * stride);
    for (int v = 0; v < nvec; ++v) {
        const uint4 x = src[v];
        rec[(4 * v + 0) * B] = x.x;
        rec[(4 * v + 1) * B] = x.y;
        rec[(4 * v + 2) * B] = x.z;
        rec[(4 * v + 3) * B] = x.w;
    }
    // Child of rank ci: prefix, then job par[d+ci], then par[d..n) without it
    // (the remaining set stays in increasing job order).
    const int d = (int)fsp_rec_byte(rec, B, n);
    const int ci = (int)(c - ws.poff[pi]);
    const uint32_t x = fsp_rec_byte(rec, B, d + ci);
    uint32_t prev = 0;
    for (int w = 0; w < (stride >> 2); ++w) {
        const uint32_t in = rec[w * B];
        uint32_t out = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = 4 * w + b;
            const uint32_t cur = (in >> (8 * b)) & 0xFFu;
            const uint32_t prv = b > 0 ? (in >> (8 * (b - 1))) & 0xFFu : (prev >> 24) & 0xFFu;
            uint32_t v;
            if (i < d) v = cur;
            else if (i == d) v = x;
            else if (i <= d + ci) v = prv;
            else if (i < n) v = cur;
            else if (i == n) v = (uint32_t)(d + 1);
            else v = 0u;
            out |= v << (8 * b);
        }
        rec[w * B] = out;
        prev = in;
    }
    bool bad;
    const int32_t lb = fsp_node_bound<NW, MT, ES>(I, ent, p_s, q_s, rec, cs, sq, ss, B, bad);
    if (bad) atomicOr(I.status, 2);
    ws.lbs[c] = lb;
    uint4 *dst = reinterpret_cast<uint4 *>(ws.children + c * stride);
    for (int v = 0; v < nvec; ++v)
        dst[v] = make_uint4(rec[(4 * v) * B], rec[(4 * v + 1) * B], rec[(4 * v + 2) * B],
                            rec[(4 * v + 3) * B]);
    if (d + 1 == n - 1 && lb < ctl->ub_iter)
        atomicMin(&ws.ctl->best_key, ((unsigned long long)(uint32_t)lb << 32) | (unsigned long long)c);
}

__device__ __forceinline__ int solve_ub_new(const SolveCtl *ctl)
{
    const unsigned long long k = ctl->best_key;
    const int ubi = ctl->ub_iter;
    if (k == ~0ull) return ubi;
    const int b = (int)(k >> 32);
    return b < ubi ? b : ubi;
}

// Elimination (Sec. II-A), step 1: survivors (not complete schedules, bound
// below the new UB) and leaves per block of 256 children.  Both elimination
// kernels are held to 32 registers: 8 blocks of 256 per SM, one wave for a
// pool of 2^18 children.
__global__ void __launch_bounds__(SOLVE_B, 8) k_count(SolveWs ws, int n, int stride)
{
    pdl_launch_dependents();
    pdl_wait();
    const SolveCtl *ctl = ws.ctl;
    const long long nch = ctl->n_children;
    const int ubn = solve_ub_new(ctl);
    const long long c = (long long)blockIdx.x * SOLVE_B + threadIdx.x;
    bool leaf = false, surv = false;
    int dch = 0;
    if (c < nch) {
        dch = solve_depth(ws, ws.children + c * stride, n);
        leaf = dch == n - 1;
        surv = !leaf && ws.lbs[c] < ubn;
    }
    __shared__ long long red[SOLVE_B / 32];
    const int cs = __syncthreads_count(surv);
    const int cl = __syncthreads_count(leaf);
    const long long cr = block_sum_ll(surv ? n - dch : 0, red);
    if (threadIdx.x == 0) {
        ws.blk[3 * blockIdx.x] = cs;
        ws.blk[3 * blockIdx.x + 1] = cl;
        ws.blk[3 * blockIdx.x + 2] = (int)cr;
    }
}

// Elimination, step 2: stable compaction onto the stack in reverse pool
// order (the pool's first survivor on top), with each survivor's running
// children count; block 0 applies the iteration to the control block.
__global__ void __launch_bounds__(SOLVE_B, 8) k_push(SolveWs ws, int n, int stride)
{
    __shared__ long long red[5][SOLVE_B / 32];
    __shared__ int wcnt[SOLVE_B / 32], wr[SOLVE_B / 32];
    pdl_wait();
    SolveCtl *ctl = ws.ctl;
    if (ctl->n_parents == 0) return;  // an iteration that did nothing changes nothing
    const long long nch = ctl->n_children;
    const int ubn = solve_ub_new(ctl);
    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    // this thread's child first (its loads overlap the block sums below)
    const long long c = (long long)b * SOLVE_B + tid;
    int dch = n - 1;
    int32_t lbc = 0;
    if (c < nch) {
        dch = solve_depth(ws, ws.children + c * stride, n);
        lbc = ws.lbs[c];
    }
    // survivors and leaves per iteration stay below 2^27 (pool <= 2^26): int;
    // survivors' children (up to 255 each) need 64 bits
    int before = 0, total = 0, leaves = 0;
    long long before_r = 0, total_r = 0;
#pragma unroll 4
    for (int i = tid; i < (int)gridDim.x; i += SOLVE_B) {
        const int s = ws.blk[3 * i];
        const long long sr = ws.blk[3 * i + 2];
        total += s;
        total_r += sr;
        leaves += ws.blk[3 * i + 1];
        if (i < b) { before += s; before_r += sr; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        before += __shfl_xor_sync(0xffffffffu, before, o);
        total += __shfl_xor_sync(0xffffffffu, total, o);
        leaves += __shfl_xor_sync(0xffffffffu, leaves, o);
        before_r += __shfl_xor_sync(0xffffffffu, before_r, o);
        total_r += __shfl_xor_sync(0xffffffffu, total_r, o);
    }
    if (lane == 0) {
        red[0][wid] = before; red[1][wid] = total; red[2][wid] = leaves;
        red[3][wid] = before_r; red[4][wid] = total_r;
    }
    const bool surv = c < nch && dch != n - 1 && lbc < ubn;
    const int rc = surv ? n - dch : 0;
    const unsigned bal = __ballot_sync(0xffffffffu, surv);
    int rincl = rc;  // survivors' children up to this one, in the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, rincl, o);
        if (lane >= o) rincl += u;
    }
    if (lane == 0) wcnt[wid] = __popc(bal);
    if (lane == 31) wr[wid] = rincl;
    __syncthreads();
    before = total = leaves = before_r = total_r = 0;
    int woff = 0, wroff = 0;
    for (int w = 0; w < SOLVE_B / 32; ++w) {
        before += red[0][w];
        total += red[1][w];
        leaves += red[2][w];
        before_r += red[3][w];
        total_r += red[4][w];
        if (w < wid) { woff += wcnt[w]; wroff += wr[w]; }
    }
    const long long s_pop = ctl->s_pop;
    if (surv) {
        const long long q = before + woff + __popc(bal & ((1u << lane) - 1u));
        const long long pos = s_pop + total - 1 - q;
        const uint4 *src = reinterpret_cast<const uint4 *>(ws.children + c * stride);
        uint4 *dst = reinterpret_cast<uint4 *>(ws.stack + pos * stride);
        for (int v = 0; v < (stride >> 4); ++v) dst[v] = src[v];
        // the survivors at or below pos are this one and those after it in pool order
        const long long base = s_pop > 0 ? ws.cum[s_pop - 1] : 0;
        ws.cum[pos] = base + total_r - (before_r + wroff + rincl - rc);
    }
    if (b == 0) {
        const int ubi = ctl->ub_iter;
        const bool improved = ubn < ubi;
        if (improved) {
            const long long idx = (long long)(ctl->best_key & 0xffffffffull);
            for (int i = tid; i < n; i += SOLVE_B) ws.inc[i] = ws.children[idx * stride + i];
        }
        if (tid == 0) {
            const long long it = ctl->cnt[4];
            ctl->cnt[0] += nch;
            ctl->cnt[1] += ctl->n_parents;
            ctl->cnt[2] += nch - leaves - total;
            ctl->cnt[3] += leaves;
            ctl->cnt[4] = it + 1;
            if (improved) ctl->cnt[5] += 1;
            ctl->cnt[6] += ctl->early;
            ctl->ub = ubn;
            ctl->stack_size = s_pop + total;
            if (it < ws.trace_cap) {
                ws.trace[4 * it + 0] = ctl->n_parents;
                ws.trace[4 * it + 1] = nch;
                ws.trace[4 * it + 2] = total;
                ws.trace[4 * it + 3] = ubn;
            }
        }
    }
}

// Branching + bounding, fast path: NPT children per thread (fsp_bound2.cuh).
template <int MT, int NV, int NW>
__global__ void __launch_bounds__(FSP_B2) k_branch_bound2(DevInst I, SolveWs ws, Bound2Smem L)
{
    constexpr int NPT = FSP_NPT;
    const SolveCtl *ctl = ws.ctl;
    const long long nch = ctl->n_children;
    const int B = blockDim.x, tid = threadIdx.x, SB = B * NPT;
    if ((long long)blockIdx.x * SB >= nch) return;
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
    int slot[NPT];
    uint32_t Um[NPT][NW];
    int32_t lb[NPT];
    int dch[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        slot[j] = tid + j * B;
        const long long c = (long long)blockIdx.x * SB + slot[j];
        FspRec<NV> ch;
        if (c < nch) {
            const int pi = solve_parent_of(ws.poff, np, c);
            const int ci = (int)(c - __ldg(ws.poff + pi));
            FspRec<NV> par;
            fsp_load_rec(par, ws.stack + (S - 1 - pi) * stride);
            fsp_make_child(par, n, ci, ch);
            fsp_store_rec(ch, ws.children + c * stride);
        } else {
#pragma unroll
            for (int q = 0; q < 4 * NV; ++q) ch.w[q] = 0u;
        }
        dch[j] = (int)fsp_rec_byte_dyn(ch, n);
        int32_t C[MT], SQ[MT];
        bool bad;
        fsp_prologue<MT, NV, NW>(ch, n, pq_s, I.mp, Um[j], C, SQ, lb[j], bad, I.var);
#pragma unroll
        for (int k = 0; k < MT; ++k) {
            cs[k * SB + slot[j]] = C[k];
            sq[k * SB + slot[j]] = SQ[k];
        }
    }
    fsp_pair_scan<MT, NPT, NW>(n, ent_s, cs, sq, SB, slot, Um, lb);
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        const long long c = (long long)blockIdx.x * SB + slot[j];
        if (c < nch) {
            ws.lbs[c] = lb[j];
            if (dch[j] == n - 1 && lb[j] < ub_iter)
                atomicMin(&ws.ctl->best_key,
                          ((unsigned long long)(uint32_t)lb[j] << 32) | (unsigned long long)c);
        }
    }
}

typedef void (*BranchBound2Fn)(DevInst, SolveWs, Bound2Smem);

static BranchBound2Fn pick_branch_bound2(int mt, int nv, int nw)
{
#define FSP_CASE2(MT_, NV_, NW_) \
    if (mt == MT_ && nv == NV_ && nw == NW_) return &k_branch_bound2<MT_, NV_, NW_>;
    FSP_SHAPES2(FSP_CASE2)
#undef FSP_CASE2
    return nullptr;
}

typedef void (*BranchBoundFn)(DevInst, SolveWs, BoundSmem);

static BranchBoundFn pick_branch_bound(int nw, int mt, bool es)
{
#define FSP_CASE(NW_, MT_, ES_) \
    if (nw == NW_ && mt == MT_ && es == ES_) return &k_branch_bound<NW_, MT_, ES_>;
    FSP_SHAPES(FSP_CASE)
#undef FSP_CASE
    return nullptr;
}

// ------------------------------------------------------------------ host --

// Pool-size tuning while searching (Sec. III, Algorithm 1), on measured
// throughput: a trial runs `window` iterations at one pool size and scores
// nodes bounded per second of wall time.  The first pool is (nodes per CTA)
// x (SM count); it doubles while the score improves and the pool stays
// within SMs x 2048; then a binary search between the neighbours of the
// best pool (halving the interval each round, a few rounds) refines it, and
// the best pool is kept for the rest of the search.
struct PoolTuner {
    bool on = false;
    int phase = 0;  // 0 doubling, 1 refining, 2 settled
    long long unit = 256, max_pool = 0, cur = 0, best = 0, lo = 0, hi = 0;
    double best_eff = -1e300;  // no trial yet
    long long window = 8, it_in = 0, b0 = 0;
    double t0 = 0.0;
    long long cand[2] = {0, 0};
    int ncand = 0, icand = 0, rounds = 0;

    long long round_unit(long long x) const
    {
        x = (x + unit / 2) / unit * unit;
        if (x < unit) x = unit;
        if (x > max_pool) x = max_pool;
        return x;
    }
    void start(long long unit_, long long sms, long long maxp, long long win)
    {
        on = true;
        unit = unit_ > 0 ? unit_ : 256;
        max_pool = maxp / unit * unit;
        if (max_pool < unit) max_pool = unit;
        cur = round_unit(unit * sms);
        best = cur;
        window = win > 0 ? win : 8;
    }
    bool next_candidates()
    {
        ncand = icand = 0;
        if (rounds >= 3 || hi - lo <= 2 * unit) return false;
        const long long a = round_unit((lo + best) / 2), b = round_unit((best + hi) / 2);
        if (a != best && a != lo) cand[ncand++] = a;
        if (b != best && b != hi && b != a) cand[ncand++] = b;
        rounds++;
        return ncand > 0;
    }
    void decide(double eff)
    {
        const long long tried = cur;
        if (eff > best_eff) { best_eff = eff; best = tried; }
        if (phase == 0) {
            // Algorithm 1 doubles the blocks every nb_iterations while threads x
            // blocks stays within the device's active threads, keeping the best
            // pool so far (one slower trial does not end the doubling)
            if (tried * 2 <= max_pool) { cur = tried * 2; return; }
            phase = 1;
            lo = round_unit(best / 2);
            hi = round_unit(best * 2);
        } else {
            if (++icand < ncand) { cur = cand[icand]; return; }
            // shrink the interval around the best of this round
            if (best < lo || best > hi) { lo = round_unit(best / 2); hi = round_unit(best * 2); }
            const long long half = (hi - lo) / 4;
            lo = round_unit(best - half > lo ? best - half : lo);
            hi = round_unit(best + half < hi ? best + half : hi);
        }
        if (next_candidates()) cur = cand[0];
        else { phase = 2; cur = best; }
    }
    // Called before each iteration with the nodes bounded so far.
    void observe(long long bounded, double now)
    {
        if (!on || phase == 2) return;
        if (it_in == window) {
            const double dt = now - t0;
            decide(dt > 0 ? (double)(bounded - b0) / dt : 0.0);
            it_in = 0;
        }
        if (phase == 2) return;
        if (it_in == 0) { t0 = now; b0 = bounded; }
        it_in++;
    }
};

// Block shape of the family kernel (warps per CTA), chosen after the pool
// settled: each candidate runs `window` iterations and the best nodes bounded
// per second of wall time is kept (the bounds do not depend on it).
struct BlockTuner {
    bool on = false, settled = true;
    int n = 0, cur = 0, best = 0, tried = 0;
    double best_eff = -1e300;
    long long window = 8, it_in = 0, b0 = 0;
    double t0 = 0.0;
    void start(int ncand, long long win)
    {
        n = ncand;
        on = n > 1;
        settled = !on;
        cur = best = n - 1;  // start from the most warps
        window = win > 0 ? win : 8;
    }
    void observe(long long bounded, double now)
    {
        if (settled) return;
        if (it_in == window) {
            const double dt = now - t0;
            const double eff = dt > 0 ? (double)(bounded - b0) / dt : 0.0;
            if (eff > best_eff) { best_eff = eff; best = cur; }
            it_in = 0;
            if (++tried == n) { settled = true; cur = best; return; }
            cur = (cur + 1) % n;
        }
        if (it_in == 0) { t0 = now; b0 = bounded; }
        it_in++;
    }
};

static double wall_seconds()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Options, workspace layout and kernels of one search.
// Launch with programmatic stream serialization (the kernel may start while
// the one ahead of it on the stream finishes; it calls pdl_wait() before it
// reads what that one writes); on = false (FSP_PDL=0, read once per call)
// launches in plain stream order.
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(bool on, void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem,
                              cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = on ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

struct SolvePlan {
    fsp_options o;
    SolveLayout L;
    BoundShape shp;
    BranchBoundFn bb;
    BranchBound2Fn bb2;
    BranchFamilyFn bf;   // families of children bounded together (NULL: per child)
    FamSmem famL;        // its layout at the most warps that fit
    FamSmem famC[4];     // the block shapes the tuner tries (ascending warps; famL last)
    int nfam;
    BranchLearnedFn bl;  // learned order (NULL: plain)
    BoundListFn blist;
    int per_cta;
    int list_grid;       // persistent grid of the list kernel
    bool bidir;          // bidirectional branching
    int rs;              // bytes per stack record
};

// A block shape fixed by the caller (opt->warps): the one candidate, so the
// block tuner has nothing to choose.
static int family_fixed_warps(const fsp_instance *I, int mt, int nv, int most, int warps, SolvePlan *P)
{
    if (warps == 0) return FSP_OK;
    if (warps < 0 || warps > most) {
        fsp_set_error("fsp_solve: warps = %d; this shape's bounding kernel takes 1..%d", warps, most);
        return FSP_ERR_ARG;
    }
    const int K = P->famL.K;
    P->famC[0] = family_smem_layout(I, mt, nv, warps);
    P->famC[0].K = K;
    P->nfam = 1;
    return FSP_OK;
}

static int solve_prepare(fsp_instance *I, int32_t *cmax, int32_t *perm, const fsp_options *opt, SolvePlan *P)
{
    if (!I || !cmax || !perm) { fsp_set_error("fsp_solve: NULL argument"); return FSP_ERR_ARG; }
    if (opt) P->o = *opt; else fsp_default_options(&P->o);
    const fsp_options &o = P->o;
    int rc = solve_layout(I, &o, &P->L);
    if (rc != FSP_OK) return rc;
    P->bidir = o.branching == FSP_BRANCH_BIDIR;
    P->rs = rec_stride(I, &o);
    if (P->bidir) {
        if ((o.init_nodes && o.init_count > 0) || o.order != FSP_ORDER_PLAIN || o.log_nodes) {
            fsp_set_error("fsp_solve: bidirectional branching starts from the root, in the plain order, "
                          "without node logging");
            return FSP_ERR_ARG;
        }
        P->bb = nullptr;
        P->bb2 = nullptr;
        P->bf = nullptr;
        P->nfam = 0;
        P->bl = nullptr;
        P->blist = nullptr;
        P->list_grid = 0;
        P->per_cta = 256;
        // the family kernel with bidirectional records where its tables fit
        // (FSP_FAMILY=0: children, the pool bound and the leaf pass, one by one)
        const int mt = fsp_mt(I->m), nv = P->rs / 16;
        const char *ev = getenv("FSP_FAMILY");
        const int w = (mt == 0 || nv > 4 || (ev && ev[0] == '0')) ? 0 : family_warps(I, mt, nv);
        if (w > 0 && (P->bf = pick_branch_family(mt, nv, false, false, true)) != nullptr) {
            P->famL = family_smem_layout(I, mt, nv, w);
            P->famL.K = 0;
            const int cand[3] = {4, 8, 12};
            for (int c = 0; c < 3; ++c)
                if (cand[c] < w) P->famC[P->nfam++] = family_smem_layout(I, mt, nv, cand[c]);
            P->famC[P->nfam++] = P->famL;
            if ((rc = family_fixed_warps(I, mt, nv, w, o.warps, P)) != FSP_OK) return rc;
            if ((rc = fsp_allow_smem(I, (const void *)P->bf, P->famL.bytes)) != FSP_OK) return rc;
        }
        if (o.workspace && ((uintptr_t)o.workspace & 255) != 0) {
            fsp_set_error("fsp_solve: workspace must be 256-byte aligned");
            return FSP_ERR_ARG;
        }
        return FSP_OK;
    }
    if ((rc = fsp_bound_shape(I, &P->shp)) != FSP_OK) return rc;
    const BoundShape &shp = P->shp;
    P->bb = nullptr;
    P->bb2 = nullptr;
    if (shp.ver == 2) {
        P->bb2 = pick_branch_bound2(shp.mt, shp.nv, shp.nw);
        if (!P->bb2) { fsp_set_error("fsp_solve: no kernel for this shape"); return FSP_ERR_ARG; }
        if ((rc = fsp_allow_smem(I, (const void *)P->bb2, shp.L2.bytes)) != FSP_OK) return rc;
    } else {
        P->bb = pick_branch_bound(shp.nw, shp.mt, shp.es);
        if (!P->bb) { fsp_set_error("fsp_solve: no kernel for this shape"); return FSP_ERR_ARG; }
        if ((rc = fsp_allow_smem(I, (const void *)P->bb, shp.L.bytes)) != FSP_OK) return rc;
    }
    P->per_cta = shp.ver == 2 ? shp.B * FSP_NPT : shp.B;
    // each parent's children are bounded together where the family kernel's
    // tables fit (FSP_FAMILY=0 keeps the per-child kernels)
    P->bf = nullptr;
    P->nfam = 0;
    if (shp.ver == 2) {
        const char *ev = getenv("FSP_FAMILY");
        const int w = (ev && ev[0] == '0') ? 0 : family_warps(I, shp.mt, shp.nv);
        if (w > 0 && (P->bf = pick_branch_family(shp.mt, shp.nv, P->L.learned, I->var == FSP_BOUND_HEADS)) !=
                         nullptr) {
            P->famL = family_smem_layout(I, shp.mt, shp.nv, w);
            P->famL.K = P->L.learned ? P->L.topk : 0;
            P->nfam = 0;
            const int cand[3] = {4, 8, 12};
            for (int c = 0; c < 3; ++c)
                if (cand[c] < w) {
                    P->famC[P->nfam] = family_smem_layout(I, shp.mt, shp.nv, cand[c]);
                    P->famC[P->nfam++].K = P->famL.K;
                }
            P->famC[P->nfam++] = P->famL;
            if ((rc = family_fixed_warps(I, shp.mt, shp.nv, w, o.warps, P)) != FSP_OK) return rc;
            if ((rc = fsp_allow_smem(I, (const void *)P->bf, P->famL.bytes)) != FSP_OK) return rc;
        }
    }
    P->bl = nullptr;
    P->blist = nullptr;
    P->list_grid = 0;
    if (P->L.learned && shp.ver == 2 && !P->bf) {  // other shapes run the plain order
        P->bl = pick_branch_learned(shp.mt, shp.nv, shp.nw);
        P->blist = pick_bound_list(shp.mt, shp.nv, shp.nw);
        if (!P->bl || !P->blist) { fsp_set_error("fsp_solve: no learned kernel for this shape"); return FSP_ERR_ARG; }
        if ((rc = fsp_allow_smem(I, (const void *)P->bl, shp.L2.bytes)) != FSP_OK) return rc;
        if ((rc = fsp_allow_smem(I, (const void *)P->blist, shp.L2.bytes)) != FSP_OK) return rc;
        int per_sm = 1;
        if ((rc = fsp_blocks_per_sm(I, (const void *)P->blist, shp.B, shp.L2.bytes, &per_sm)) != FSP_OK) return rc;
        P->list_grid = I->sm_count * per_sm;
    }
    if (o.workspace && ((uintptr_t)o.workspace & 255) != 0) {
        fsp_set_error("fsp_solve: workspace must be 256-byte aligned");
        return FSP_ERR_ARG;
    }
    if (o.init_nodes && o.init_count > 0) {
        if (I->n < 2) { fsp_set_error("fsp_solve: init_nodes need n >= 2"); return FSP_ERR_ARG; }
        if (o.init_count > P->L.cap) {
            fsp_set_error("fsp_solve: %lld init nodes exceed the stack capacity %lld",
                          (long long)o.init_count, P->L.cap);
            return FSP_ERR_CAPACITY;
        }
    }
    return FSP_OK;
}

// One search with its scratch at `base` (P->L.bytes bytes, 256-byte aligned).
// timed: CUDA events give time_ms and, with opt->profile, the phase times,
// and the read-back block and events come from the instance's cache (created
// when the cache is empty); without it the search reports zero times and
// uses only the block and events the instance reserved at creation, so it
// creates nothing.
static int solve_run(fsp_instance *I, int32_t ub0, int32_t *cmax, int32_t *perm, fsp_stats *stats,
                     const SolvePlan *P, uint8_t *base, bool timed)
{
    const fsp_options &o = P->o;
    const SolveLayout &L = P->L;
    const BoundShape &shp = P->shp;
    const BranchBoundFn bb = P->bb;
    const BranchBound2Fn bb2 = P->bb2;
    const int per_cta = P->per_cta;
    const bool prof = timed && o.profile;
    const char *pdl_env = getenv("FSP_PDL");
    const bool pdl = !(pdl_env && pdl_env[0] == '0');  // programmatic dependent launch of the step's kernels
    int rc = FSP_OK;
    cudaStream_t st = (cudaStream_t)o.stream;
    SolveWs ws;
    ws.ctl = (SolveCtl *)(base + L.off_ctl);
    ws.stack = base + L.off_stack;
    ws.cap = L.cap;
    ws.children = base + L.off_children;
    ws.lbs = (int32_t *)(base + L.off_lbs);
    ws.poff = (int *)(base + L.off_poff);
    ws.blk = (int *)(base + L.off_blk);
    ws.cum = (long long *)(base + L.off_cum);
    ws.iblk = (long long *)(base + L.off_iblk);
    ws.inc = base + L.off_inc;
    ws.trace = (long long *)(base + L.off_trace);
    ws.trace_cap = L.trace_cap;
    ws.max_children = L.max_children;
    ws.max_blocks = L.max_blocks;
    ws.list = (int *)(base + L.off_list);
    ws.px = (float *)(base + L.off_px);
    ws.pscore = (float *)(base + L.off_pscore);
    ws.topk = (int16_t *)(base + L.off_topk);
    ws.max_parents = L.max_parents;
    ws.bidir = P->bidir ? 1 : 0;
    const int rs = P->rs;
    const DevInst D = dev_view(I);
    const float T = (float)I->total / (float)I->m;
    long long logged = 0;

    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t pe[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t rb[2] = {nullptr, nullptr};  // read-backs launched ahead
    void *pin = nullptr;                     // two pinned read-back slots of SOLVE_RB bytes
    const uint8_t *last = nullptr;           // the slot h was taken from (its incumbent at byte 256)
    bool idle = false;                       // nothing enqueued since the last read-back's sync
    double t_sel = 0, t_bb = 0, t_cmp = 0, t_inf = 0;
    PoolTuner tuner;
    BlockTuner btuner;
    int fam_i = P->bf ? P->nfam - 1 : 0;
    SolveCtl h;
    memset(&h, 0, sizeof h);
    cudaError_t e = cudaSuccess;
#define TRY(call)                                                      \
    do {                                                               \
        e = (call);                                                    \
        if (e != cudaSuccess) { rc = fsp_cuda_fail(e, #call); goto out; } \
    } while (0)
    if (timed) {
        if ((rc = fsp_event_take(I, &ev0)) != FSP_OK || (rc = fsp_event_take(I, &ev1)) != FSP_OK) goto out;
    }
    if (prof)
        for (int i = 0; i < 5; ++i)
            if ((rc = fsp_event_take(I, &pe[i])) != FSP_OK) goto out;
    if (timed) {
        if ((rc = fsp_pinned_take(I, &pin)) != FSP_OK) goto out;
    } else {
        fsp_noalloc_reserved(I, &pin, rb);
    }
    if (timed) TRY(cudaEventRecord(ev0, st));
    if (o.pool_size == 0) tuner.start(per_cta, I->sm_count, tuner_max_pool(I), o.tune_window);
    if (o.pool_size == 0 && P->bf) btuner.start(P->nfam, o.tune_window);
    if (I->n == 1) {
        k_solve_single<<<1, 32, 0, st>>>(ws, I->d_p, I->m, ub0);
        TRY(cudaGetLastError());
        if (timed) TRY(cudaEventRecord(ev1, st));
        TRY(cudaMemcpyAsync(pin, ws.ctl, 256 + I->n, cudaMemcpyDeviceToHost, st));
        TRY(cudaStreamSynchronize(st));
        last = (const uint8_t *)pin;
        memcpy(&h, last, sizeof h);
        idle = true;
    } else {
        if (o.init_nodes && o.init_count > 0) {
            const bool wide = I->n > 63;
            // records on this device or in pinned host memory are read in place
            // by the start kernel; others (and records of n >= 64 jobs) are copied first
            const uint8_t *src = wide ? nullptr : (const uint8_t *)fsp_device_view(o.init_nodes, 16);
            if (!src) {
                TRY(cudaMemcpyAsync(ws.stack, o.init_nodes, (size_t)o.init_count * I->stride, cudaMemcpyDefault, st));
                src = ws.stack;
            }
            const unsigned gi = (unsigned)((o.init_count + SOLVE_B - 1) / SOLVE_B);
            const int nv = wide ? 1 : I->stride >> 4;  // wide: block sums only, the records follow
            auto init_fn = nv == 1 ? &k_solve_init_nodes<1> : nv == 2 ? &k_solve_init_nodes<2>
                         : nv == 3 ? &k_solve_init_nodes<3> : &k_solve_init_nodes<4>;
            init_fn<<<gi, SOLVE_B, 0, st>>>(ws, src, I->n, I->stride, o.init_count, ub0, wide);
            if (wide) k_solve_init_nodes_wide<<<gi, SOLVE_B, 0, st>>>(ws, I->n, I->stride, o.init_count);
            const int scanned = gi > INIT_SCAN_BLOCKS;
            if (scanned) k_init_scan<<<1, 1024, 0, st>>>(ws, gi);
            TRY(launch_pdl(pdl, k_init_cum, gi, SOLVE_B, 0, st, ws, I->n, I->stride, (long long)o.init_count, scanned));
        } else {
            k_solve_init<<<1, 128, 0, st>>>(ws, I->n, rs, ub0);
        }
        TRY(cudaGetLastError());
        // the start state is known here, so the first iteration goes out
        // without a read-back (a malformed start record sets the device
        // status, that iteration does nothing and the next read-back reports it)
        memset(&h, 0, sizeof h);
        h.stack_size = (o.init_nodes && o.init_count > 0) ? o.init_count : 1;
        h.ub = ub0;
        // one iteration on the stream with pool size `pool`
        auto launch_iter = [&](long long pool) -> int {
            cudaError_t le;
#define LTRY(call)                                                  \
    do {                                                            \
        le = (call);                                                \
        if (le != cudaSuccess) return fsp_cuda_fail(le, #call);     \
    } while (0)
            const int grid = (int)((pool + I->n + SOLVE_B - 1) / SOLVE_B);
            const int grid_bb = (int)((pool + I->n + per_cta - 1) / per_cta);
            idle = false;
            if (prof) LTRY(cudaEventRecord(pe[0], st));
            LTRY(launch_pdl(pdl, k_select, 1, SELECT_B, 0, st, ws, I->n, rs, pool, (long long)o.node_budget,
                            (long long)o.max_iterations, (int)(P->bf == nullptr)));
            if (prof) LTRY(cudaEventRecord(pe[1], st));
            if (P->bidir && !P->bf) {  // children, their bounds, then the exact values of the complete ones
                const long long mc = pool + I->n;
                bidir_launch_children(ws, I->n, rs, mc, st);
                const int brc = bidir_bound(I, ws.children, mc, &ws.ctl->n_children, ws.lbs, st);
                if (brc != FSP_OK) return brc;
                bidir_launch_leaves(ws, I, rs, mc, st);
            } else if (P->bl) {
                const long long npar = pool / 2 + 2;  // stacked nodes have >= 2 children
                int frc = fsp_mlp_topk_parents(o.model, I, ws.stack, &ws.ctl->s_pop, &ws.ctl->n_parents, npar,
                                               L.topk, ws.topk, st);
                if (frc == FSP_ERR_ARG) {  // network shape without the fused kernel
                    launch_parent_features(D, ws, T, npar, st);
                    frc = fsp_mlp_forward_dev(o.model, ws.px, &ws.ctl->n_parents, npar, ws.pscore, st);
                    if (frc == FSP_OK) launch_topk(ws, I->P, L.topk, npar, st);
                }
                if (frc != FSP_OK) return frc;
                if (prof) LTRY(cudaEventRecord(pe[4], st));
                const int grid_l = (int)((pool + I->n + 255) / 256);
                P->bl<<<grid_l, 256, shp.L2.bytes, st>>>(D, ws, shp.L2, L.topk);
                P->blist<<<P->list_grid, shp.B, shp.L2.bytes, st>>>(D, ws, shp.L2);
            } else if (P->bf) {
                if (P->L.learned) {  // each parent's predicted pairs first
                    const long long npar = pool / 2 + 2;
                    int frc = fsp_mlp_topk_parents(o.model, I, ws.stack, &ws.ctl->s_pop, &ws.ctl->n_parents, npar,
                                                   L.topk, ws.topk, st);
                    if (frc == FSP_ERR_ARG) {  // network shape without the fused kernel
                        launch_parent_features(D, ws, T, npar, st);
                        frc = fsp_mlp_forward_dev(o.model, ws.px, &ws.ctl->n_parents, npar, ws.pscore, st);
                        if (frc == FSP_OK) launch_topk(ws, I->P, L.topk, npar, st);
                    }
                    if (frc != FSP_OK) return frc;
                    if (prof) LTRY(cudaEventRecord(pe[4], st));
                }
                // at most pool / 2 + 1 parents: stacked nodes have >= 2 children
                const FamSmem &FL = P->famC[fam_i];
                const long long fam = (pool / 2 + 1 + FL.warps - 1) / FL.warps;
                const int grid_f = (int)(fam < I->sm_count ? fam : I->sm_count);
                DevInst Df = D;
                Df.stride = rs;  // bidirectional records are wider
                LTRY(launch_pdl(pdl, P->bf, (unsigned)grid_f, FL.warps * 32, FL.bytes, st, Df, ws, FL));
            } else if (bb2) {
                bb2<<<grid_bb, shp.B, shp.L2.bytes, st>>>(D, ws, shp.L2);
            } else {
                bb<<<grid_bb, shp.B, shp.L.bytes, st>>>(D, ws, shp.L);
            }
            if (prof) LTRY(cudaEventRecord(pe[2], st));
            LTRY(launch_pdl(pdl, k_count, (unsigned)grid, SOLVE_B, 0, st, ws, I->n, rs));
            LTRY(launch_pdl(pdl, k_push, (unsigned)grid, SOLVE_B, 0, st, ws, I->n, rs));
            if (prof) LTRY(cudaEventRecord(pe[3], st));
            LTRY(cudaGetLastError());
#undef LTRY
            return FSP_OK;
        };
        auto pool_of = [&](long long it) -> long long {  // fixed, replayed, or the settled tuner's
            long long pool = tuner.on ? tuner.cur : o.pool_size;
            if (o.schedule && o.schedule_len > 0) pool = o.schedule[it < o.schedule_len ? it : o.schedule_len - 1];
            if (o.schedule_out && it < o.schedule_out_cap) o.schedule_out[it] = pool;
            return pool;
        };
        // Without logging or phase times, and once the tuner (if any) has
        // settled, the next iteration depends on nothing the host reads back,
        // so it is launched before the read-back of the previous one:
        // k_select makes an iteration past a stop (empty stack, budget,
        // iteration cap, error) do nothing, and the host stops one read-back
        // later.  Until then iterations go out one at a time.
        const bool may_ahead = !prof && !o.log_nodes;
        long long it0 = -1;  // first iteration launched ahead
        for (long long it = 0;; ++it) {
            if (it > 0) {
                if (timed) TRY(cudaEventRecord(ev1, st));  // the end of the search if it stops here
                TRY(cudaMemcpyAsync(pin, ws.ctl, 256 + I->n, cudaMemcpyDeviceToHost, st));
                TRY(cudaStreamSynchronize(st));
                last = (const uint8_t *)pin;
                memcpy(&h, last, sizeof h);
                idle = true;
            }
            if (prof && it > 0) {
                float a = 0, b = 0, c = 0;
                TRY(cudaEventElapsedTime(&a, pe[0], pe[1]));
                TRY(cudaEventElapsedTime(&b, pe[1], pe[2]));
                TRY(cudaEventElapsedTime(&c, pe[2], pe[3]));
                t_sel += a;
                t_cmp += c;
                if (P->L.learned && (P->bl || P->bf)) {  // the network's share is not bounding
                    float d = 0;
                    TRY(cudaEventElapsedTime(&d, pe[1], pe[4]));
                    t_inf += d;
                    b -= d;
                }
                t_bb += b;
            }
            if (h.status != 0) {
                rc = h.status;
                fsp_set_error(rc == FSP_ERR_CAPACITY ? "fsp_solve: stack capacity exceeded"
                              : rc == FSP_ERR_ARG ? "fsp_solve: malformed init node (not a permutation "
                                                    "or depth > n-2)"
                                                  : "fsp_solve: device error");
                break;
            }
            if (o.log_nodes && it > 0 && logged < o.log_cap && h.n_children > 0) {
                const long long k = h.n_children < o.log_cap - logged ? h.n_children : o.log_cap - logged;
                idle = false;
                TRY(cudaMemcpyAsync(o.log_nodes + logged * I->stride, ws.children, (size_t)k * I->stride,
                                    cudaMemcpyDeviceToDevice, st));
                if (o.log_lbs)
                    TRY(cudaMemcpyAsync(o.log_lbs + logged, ws.lbs, (size_t)k * 4, cudaMemcpyDeviceToDevice, st));
                logged += k;
            }
            if (h.stack_size == 0) break;
            if (o.node_budget > 0 && h.cnt[0] >= o.node_budget) { rc = FSP_INCOMPLETE; break; }
            if (o.max_iterations > 0 && it >= o.max_iterations) { rc = FSP_INCOMPLETE; break; }
            if (tuner.on && tuner.phase == 2 && !btuner.settled) {  // then the block shape
                btuner.observe(h.cnt[0], wall_seconds());
                fam_i = btuner.cur;
            }
            if (may_ahead && ((o.schedule && o.schedule_len > 0) || !tuner.on || (tuner.phase == 2 && btuner.settled))) {
                it0 = it;
                break;
            }
            long long pool = o.pool_size;
            if (o.schedule && o.schedule_len > 0)
                pool = o.schedule[it < o.schedule_len ? it : o.schedule_len - 1];
            else if (tuner.on) {
                tuner.observe(h.cnt[0], wall_seconds());
                pool = tuner.cur;
            }
            if (o.schedule_out && it < o.schedule_out_cap) o.schedule_out[it] = pool;
            if ((rc = launch_iter(pool)) != FSP_OK) goto out;
        }
        if (it0 >= 0) {
            if (timed && ((rc = fsp_event_take(I, &rb[0])) != FSP_OK || (rc = fsp_event_take(I, &rb[1])) != FSP_OK))
                goto out;
            uint8_t *hb = reinterpret_cast<uint8_t *>(pin);
            if ((rc = launch_iter(pool_of(it0))) != FSP_OK) goto out;
            if (timed) TRY(cudaEventRecord(ev1, st));  // moved to each later read-back
            TRY(cudaMemcpyAsync(hb + (it0 & 1) * SOLVE_RB, ws.ctl, 256 + I->n, cudaMemcpyDeviceToHost, st));
            TRY(cudaEventRecord(rb[it0 & 1], st));
            long long pending = it0;  // the last iteration launched, with its read-back
            for (long long it = it0 + 1;; ++it) {
                // an iteration at or past the iteration cap would do nothing: not launched
                if (!(o.max_iterations > 0 && it >= o.max_iterations)) {
                    if ((rc = launch_iter(pool_of(it))) != FSP_OK) goto out;
                    if (timed) TRY(cudaEventRecord(ev1, st));
                    TRY(cudaMemcpyAsync(hb + (it & 1) * SOLVE_RB, ws.ctl, 256 + I->n, cudaMemcpyDeviceToHost, st));
                    TRY(cudaEventRecord(rb[it & 1], st));
                    pending = it;
                }
                TRY(cudaEventSynchronize(rb[(it - 1) & 1]));
                // the state after `it` iterations; iteration it + 1, if launched
                // ahead, does nothing when the search stops here, so this slot
                // (its incumbent included) is the final state
                last = hb + ((it - 1) & 1) * SOLVE_RB;
                memcpy(&h, last, sizeof h);
                if (h.status != 0) {
                    rc = h.status;
                    fsp_set_error(rc == FSP_ERR_CAPACITY ? "fsp_solve: stack capacity exceeded"
                                  : rc == FSP_ERR_ARG ? "fsp_solve: malformed init node (not a permutation "
                                                        "or depth > n-2)"
                                                      : "fsp_solve: device error");
                    break;
                }
                if (h.stack_size == 0) break;
                if (o.node_budget > 0 && h.cnt[0] >= o.node_budget) { rc = FSP_INCOMPLETE; break; }
                if (o.max_iterations > 0 && it >= o.max_iterations) { rc = FSP_INCOMPLETE; break; }
            }
            // the last read-back follows everything launched and the last ev1
            TRY(cudaEventSynchronize(rb[pending & 1]));
            idle = true;
        }
    }
    if (!idle) {  // after a read-back the stream is already idle and ev1 recorded before it
        if (timed) {
            TRY(cudaEventRecord(ev1, st));
            TRY(cudaEventSynchronize(ev1));
        } else {
            TRY(cudaStreamSynchronize(st));
        }
    }
    *cmax = h.ub;
    if (h.cnt[5] > 0 && last) {  // the incumbent came with the control block
        for (int i = 0; i < I->n; ++i) perm[i] = last[256 + i];
    } else if (o.ub0_perm) {
        for (int i = 0; i < I->n; ++i) perm[i] = o.ub0_perm[i];
    }
    if (L.trace_cap > 0) {
        const long long rows = h.cnt[4] < L.trace_cap ? h.cnt[4] : L.trace_cap;
        if (rows > 0)
            TRY(cudaMemcpy(o.trace, ws.trace, (size_t)rows * 32, cudaMemcpyDeviceToHost));
    }
    if (o.out_count) *o.out_count = h.stack_size;
    if (o.log_count) *o.log_count = logged;
    if (o.out_nodes && h.stack_size > 0 && h.stack_size <= o.out_cap && I->n > 1)
        TRY(cudaMemcpy(o.out_nodes, ws.stack, (size_t)h.stack_size * rs, cudaMemcpyDefault));
    if (stats) {
        stats->select_ms = t_sel;
        stats->bound_ms = t_bb;
        stats->compact_ms = t_cmp;
        stats->nodes_bounded = h.cnt[0];
        stats->nodes_branched = h.cnt[1];
        stats->nodes_pruned = h.cnt[2];
        stats->leaves = h.cnt[3];
        stats->iterations = h.cnt[4];
        stats->incumbent_updates = h.cnt[5];
        stats->tuned_pool = tuner.on ? tuner.best : o.pool_size;
        stats->tuned_warps = P->bf ? P->famC[fam_i].warps : 0;
        stats->early_pruned = h.cnt[6];
        stats->families_closed_lb1 = h.fam[0];
        stats->families_closed_predicted = h.fam[1];
        stats->exact_pair_evals = h.fam[2];
        stats->infer_ms = t_inf;
        float ms = 0.f;
        if (timed) cudaEventElapsedTime(&ms, ev0, ev1);
        stats->time_ms = ms;
    }
#undef TRY
out:
    fsp_event_give(I, ev0);
    fsp_event_give(I, ev1);
    if (timed) {  // the reserved block and events stay with the instance
        fsp_event_give(I, rb[0]);
        fsp_event_give(I, rb[1]);
        fsp_pinned_give(I, pin);
    }
    for (int i = 0; i < 5; ++i) fsp_event_give(I, pe[i]);
    return rc;
}

extern "C" int fsp_solve(fsp_instance *I, int32_t ub0, int32_t *cmax, int32_t *perm, fsp_stats *stats,
                         const fsp_options *opt)
{
    SolvePlan P;
    int rc = solve_prepare(I, cmax, perm, opt, &P);
    if (rc != FSP_OK) return rc;
    uint8_t *base = (uint8_t *)P.o.workspace;
    bool owned = false;
    if (!base) {
        FSP_CUDA(cudaMalloc(&base, P.L.bytes));
        owned = true;
    }
    rc = solve_run(I, ub0, cmax, perm, stats, &P, base, true);
    if (owned) cudaFree(base);
    return rc;
}

// ---------------------------------------------------------------------------
// fsp_solve_noalloc: the same search with its scratch in a fixed device array
// of this library instead of memory allocated per call.  For callers that
// must not allocate device memory while they run (their device memory is
// reserved up front by a pool or a fixed budget, or they are plugins handed
// only input and output buffers, or cudaMalloc's implicit synchronisation of
// the whole device is unacceptable on their path).  The array occupies
// FSP_NOALLOC_SCRATCH_BYTES on every device that loads this library, until
// the process exits.
// ---------------------------------------------------------------------------
static __device__ __align__(256) uint8_t g_noalloc_scratch[FSP_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array on the current device.  In host code
// the array's name only stands for the symbol; the usable address comes from
// cudaGetSymbolAddress with the device current.  It is looked up on every
// call: a cached address would be stale after the device's context is torn
// down and made again (cudaDeviceReset), and the lookup allocates nothing
// once this library's device code is loaded on the device (the first call).
static int noalloc_scratch(uint8_t **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return fsp_cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    *out = (uint8_t *)p;
    return FSP_OK;
}

extern "C" int fsp_solve_noalloc(fsp_instance *I, int32_t ub0, int32_t *cmax, int32_t *perm, fsp_stats *stats,
                                 const fsp_options *opt)
{
    if (opt && opt->workspace) {
        fsp_set_error("fsp_solve_noalloc: takes no workspace (it uses its fixed scratch)");
        return FSP_ERR_ARG;
    }
    if (opt && (opt->order != FSP_ORDER_PLAIN || opt->log_nodes || opt->log_lbs)) {
        fsp_set_error("fsp_solve_noalloc: the learned order and node logging are not available without allocation");
        return FSP_ERR_ARG;
    }
    SolvePlan P;
    int rc = solve_prepare(I, cmax, perm, opt, &P);
    if (rc != FSP_OK) return rc;
    if (P.L.bytes > (size_t)FSP_NOALLOC_SCRATCH_BYTES) {
        fsp_set_error("fsp_solve_noalloc: this search needs %zu bytes of scratch, the fixed scratch holds %zu "
                      "(lower pool_size, stack_capacity, trace_cap or init_count, or use fsp_solve)",
                      P.L.bytes, (size_t)FSP_NOALLOC_SCRATCH_BYTES);
        return FSP_ERR_CAPACITY;
    }
    int dev = -1;
    FSP_CUDA(cudaGetDevice(&dev));
    if (dev != I->device) {
        fsp_set_error("fsp_solve_noalloc: make the instance's device (%d) current (current: %d)", I->device, dev);
        return FSP_ERR_ARG;
    }
    uint8_t *base = nullptr;
    if ((rc = noalloc_scratch(&base)) != FSP_OK) return rc;
    return solve_run(I, ub0, cmax, perm, stats, &P, base, false);
}

// The tuner's decisions against a caller-supplied score (no GPU involved).
extern "C" int64_t fsp_block_tune_simulate(int ncand, int64_t window, double (*score)(int64_t cand, void *user),
                                           void *user, int64_t *cands_out, int64_t cap, int64_t *best_out)
{
    if (ncand < 1 || window < 1 || !score || (cap > 0 && !cands_out)) {
        fsp_set_error("fsp_block_tune_simulate: invalid argument");
        return FSP_ERR_ARG;
    }
    BlockTuner b;
    b.start(ncand, window);
    long long bounded = 0;
    double now = 0.0;
    int64_t k = 0;
    while (!b.settled && k < 4096) {  // one iteration per step: it runs with shape b.cur
        const int c = b.cur;
        if (k < cap) cands_out[k] = c;
        ++k;
        now += 1.0;
        bounded += llround(score(c, user));
        b.observe(bounded, now);
    }
    if (best_out) *best_out = b.cur;
    return k;
}

extern "C" int64_t fsp_tune_simulate(int64_t nodes_per_cta, int sms, int64_t max_pool,
                                     double (*score)(int64_t pool, void *user), void *user, int64_t *pools_out,
                                     int64_t cap, int64_t *best_out)
{
    if (nodes_per_cta < 1 || sms < 1 || max_pool < 1 || !score || (cap > 0 && !pools_out)) {
        fsp_set_error("fsp_tune_simulate: invalid argument");
        return FSP_ERR_ARG;
    }
    PoolTuner t;
    t.start(nodes_per_cta, sms, max_pool, 1);
    int64_t k = 0;
    while (t.phase != 2 && k < 64) {
        if (k < cap) pools_out[k] = t.cur;
        ++k;
        t.decide(score(t.cur, user));
    }
    if (best_out) *best_out = t.best;
    return k;
}
