// fsp_solve.cuh -- state shared by the search kernels (fsp_solve.cu) and the
// learned-order kernels (fsp_learned.cu).
#pragma once

#include "fsp_bound.cuh"

// Programmatic dependent launch (sm_90 and later): a kernel launched with the
// programmatic stream serialization attribute may start while the kernel
// ahead of it on the stream is still running.  pdl_wait() returns once that
// kernel has completed and its memory operations are visible (at once for a
// kernel launched without the attribute); the code before it touches nothing
// the kernel ahead writes.  pdl_launch_dependents() lets the kernel behind
// this one be scheduled before this one completes (it then waits in its own
// pdl_wait()).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

struct SolveCtl {
    long long stack_size;   // records on the stack
    long long s_pop;        // stack size after this iteration's pops
    long long n_parents;
    long long n_children;
    unsigned long long best_key;  // (bound << 32) | child index of the best leaf
    int ub;                 // current upper bound
    int ub_iter;            // upper bound at the start of the iteration
    int status;             // FSP_ERR_* raised on the device, 0 if none
    int pad0;
    long long cnt[7];       // bounded, branched, pruned, leaves, iterations, updates, early cuts
    long long n_list;       // learned order: children left for the full bound
    long long early;        // learned order: children cut by their predicted pairs
    long long fam_next;     // family kernel: next parent to take
    long long fam[3];       // family kernel, summed over the search: families whose children
                            // all reach the UB by their one-machine bounds; families closed
                            // by their predicted pairs alone (learned order); exact pair
                            // evaluations (pairs left uncertified, per family)
};

struct SolveWs {
    SolveCtl *ctl;
    uint8_t *stack;
    long long *cum;         // cum[s]: children of stack records 0..s (n - depth each), summed
    long long *iblk;        // start records: children per block of 256
    long long cap;
    uint8_t *children;
    int32_t *lbs;
    int *poff;              // first child of each popped parent; poff[np] = children
    int *blk;               // per block of 256 children: survivors, leaves, survivors' children
    uint8_t *inc;
    long long *trace;
    long long trace_cap;
    long long max_children;
    int max_blocks;
    // learned order
    int *list;              // children left for the full bound
    float *px;              // parent features [max_parents][2m+1]
    float *pscore;          // parent pair scores [max_parents][P]
    int16_t *topk;          // best pairs of each parent [max_parents][K]
    long long max_parents;
    int bidir;              // bidirectional records: depth = d1 (byte n) + d2 (byte n+1)
};

// Scheduled jobs of a record: its depth, or d1 + d2 for a bidirectional one.
__device__ __forceinline__ int solve_depth(const SolveWs &ws, const uint8_t *rec, int n)
{
    return ws.bidir ? rec[n] + rec[n + 1] : rec[n];
}

// Bidirectional branching (fsp_bidir.cu).
int bidir_bound(fsp_instance *I, const uint8_t *nodes, long long count, const long long *dcount, int32_t *lb_out,
                cudaStream_t st);
void bidir_launch_children(const SolveWs &ws, int n, int stride, long long max_children, cudaStream_t st);
void bidir_launch_leaves(const SolveWs &ws, const fsp_instance *I, int stride, long long max_children,
                         cudaStream_t st);
extern "C" int fsp_node_stride_bidir(int n);


// Parent of child c: the last p with poff[p] <= c (poff increasing, poff[0] = 0).
__device__ __forceinline__ int solve_parent_of(const int *__restrict__ poff, int np, long long c)
{
    int lo = 0, hi = np;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if ((long long)__ldg(poff + mid) <= c) lo = mid;
        else hi = mid;
    }
    return lo;
}

typedef void (*BranchLearnedFn)(DevInst, SolveWs, Bound2Smem, int);
typedef void (*BoundListFn)(DevInst, SolveWs, Bound2Smem);

// Learned-order kernels (fsp_learned.cu).
BranchLearnedFn pick_branch_learned(int mt, int nv, int nw);
BoundListFn pick_bound_list(int mt, int nv, int nw);
void launch_parent_features(const DevInst &D, const SolveWs &ws, float T, long long npar, cudaStream_t st);
void launch_topk(const SolveWs &ws, int P, int K, long long npar, cudaStream_t st);
