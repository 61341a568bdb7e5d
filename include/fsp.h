/*
 * fsp.h -- C ABI of the GB300 (sm_103a) parallel-bounding library for the
 * permutation flow-shop branch-and-bound (Chakroun & Melab, "An Adaptative
 * Multi-GPU based Branch-and-Bound. A Case Study: the Flow-Shop Scheduling
 * Problem").
 *
 * Problem (Sec. II-B): n jobs, m machines, every job visits machines 0..m-1
 * in that order, every machine processes the jobs in the same order (a
 * permutation), p[j][k] is the time of job j on machine k; minimise the
 * makespan (completion time of the last job on the last machine).
 *
 * A subproblem ("node", Sec. II-B: node i is the subproblem with job J_i
 * scheduled first) is a scheduled prefix plus the set of remaining jobs.  Its
 * record is `fsp_node_stride(n)` bytes: bytes 0..n-1 hold a permutation of
 * 0..n-1 whose first d entries are the prefix in order and whose last n-d
 * entries are the remaining set in any order; byte n holds d (0 <= d <= n);
 * the rest is zero padding.  Records are contiguous, 16-byte aligned.
 *
 * The lower bound (the paper states only its O(m^2 n log n) cost, Sec. V-D)
 * is the maximum of
 *   - the one-machine bounds  C_k + S_k + qmin_k  for every machine k, and
 *   - the two-machine bounds with time lags for every machine pair k < l:
 *     the remaining jobs in Johnson's order for the pair (jobs with
 *     p_k <= p_l by increasing p_k + lag, then the others by decreasing
 *     p_l + lag; equal keys by job index), t_k = C_k, t_l = C_l,
 *     t_k += p_k(j), t_l = max(t_l, t_k + lag(j)) + p_l(j), plus qmin_l,
 * where C_k is machine k's completion time after the prefix, S_k the remaining
 * work on k, qmin_k the smallest remaining tail after k (0 if none remain),
 * and lag(j) job j's time on the machines strictly between k and l.
 *
 * Conventions: all functions return an int status (FSP_OK = 0, FSP_INCOMPLETE
 * = 1 when a node budget stopped a search, negative on error) unless stated;
 * after an error fsp_last_error() returns a message (per thread).  Device
 * pointers are CUDA device memory of the device current at
 * fsp_create_instance; host pointers are ordinary host memory.  The caller
 * owns every buffer it passes; the library never frees caller memory.  A
 * `stream` argument is a cudaStream_t (NULL = the legacy default stream).
 */
#ifndef FSP_H
#define FSP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FSP_OK 0
#define FSP_INCOMPLETE 1
#define FSP_ERR_ARG (-1)
#define FSP_ERR_CUDA (-2)
#define FSP_ERR_OOM (-3)
#define FSP_ERR_CAPACITY (-4)
#define FSP_ERR_TIMEOUT (-5)

#define FSP_UB_INF 2147483647 /* "no upper bound yet" */
#define FSP_LB_INVALID (-1)   /* lb_out value of a malformed node record */

#define FSP_MAX_JOBS 255
#define FSP_MAX_MACHINES 64

/* Opaque instance: processing times plus the per-instance tables (tails,
 * lags and Johnson order of every machine pair) resident on the device. */
typedef struct fsp_instance fsp_instance;

/* Search counters (Sec. II-A operators). */
typedef struct {
    int64_t nodes_bounded;     /* children whose bound was computed        */
    int64_t nodes_branched;    /* parents decomposed (the root included)   */
    int64_t nodes_pruned;      /* non-leaf children with bound >= UB       */
    int64_t leaves;            /* children at depth n-1 (complete schedules)*/
    int64_t iterations;        /* pool iterations                          */
    int64_t incumbent_updates; /* strict improvements of the UB            */
    double time_ms;            /* wall time of the search on the stream    */
    double select_ms;          /* device time in selection (opt->profile)  */
    double bound_ms;           /* device time in branching + bounding (the
                                  network's infer_ms not included)         */
    double compact_ms;         /* device time in elimination + compaction  */
    int64_t tuned_pool;        /* pool size the tuner settled on (pool_size = 0), else the pool */
    int64_t early_pruned;      /* children cut by their predicted pairs alone (order = learned) */
    double infer_ms;           /* device time in the network + top-K (learned, opt->profile) */
    int64_t tuned_warps;       /* warps per CTA of the family kernel (chosen on measured
                                  throughput with pool_size = 0); 0 if the per-child
                                  kernels ran */
    /* family kernel only (0 otherwise), summed over the search: */
    int64_t families_closed_lb1;       /* parents whose children all reach the UB of the
                                          iteration by their one-machine bounds (any order) */
    int64_t families_closed_predicted; /* learned order: parents whose children not cut by
                                          their one-machine bounds are all cut by the
                                          predicted pairs (the 190-pair work then skipped) */
    int64_t exact_pair_evals;          /* pairs evaluated exactly (not certified), per family */
} fsp_stats;

#define FSP_ORDER_PLAIN 0   /* every child gets its full bound */
#define FSP_ORDER_LEARNED 1 /* predicted pairs first; survivors get the full bound */

typedef struct fsp_mlp fsp_mlp;

/* Options of fsp_solve; fsp_default_options() fills the defaults. */
typedef struct {
    int64_t pool_size;      /* children bounded per iteration (Sec. III pool); default 1024;
                               0 = tune it while searching (Sec. III, Algorithm 1): start at
                               (nodes per CTA) x (SM count), double every tune_window iterations
                               while it stays within SMs x 2048, keeping the pool with the most
                               nodes bounded per second, then refine around the best and keep it */
    int64_t node_budget;    /* stop (FSP_INCOMPLETE) before an iteration once this many
                               nodes are bounded; 0 = no limit */
    int64_t stack_capacity; /* node records in the device stack; 0 = init_count + n * (pool + n) */
    const int32_t *ub0_perm;/* host, n entries or NULL: a schedule whose makespan is ub0 */
    int64_t *trace;         /* host or NULL: per iteration {parents, children, survivors,
                               UB after}, int64 x 4 */
    int64_t trace_cap;      /* rows available in trace */
    const int64_t *schedule;/* host or NULL: pool size of each iteration (the last entry
                               repeats), e.g. replaying an autotuned run */
    int64_t schedule_len;
    void *workspace;        /* device or NULL: caller-owned scratch of at least
                               fsp_solve_workspace_bytes() bytes, 256-byte aligned;
                               NULL = the library allocates and frees its own */
    void *stream;           /* cudaStream_t; NULL = legacy default stream */
    const uint8_t *init_nodes; /* host or device or NULL: start from these node records
                               (bottom of the stack first) instead of the root; each
                               must have depth <= n-2; the remaining part of each
                               record is re-sorted by job index on the device.  Memory
                               of the current device or pinned host memory, 16-byte
                               aligned and n <= 63, is read in place by the start
                               kernel (never written); anything else is copied to the
                               stack first */
    int64_t init_count;
    int64_t max_iterations; /* stop (FSP_INCOMPLETE) after this many iterations; 0 = no limit */
    uint8_t *out_nodes;     /* host or device or NULL: receives the stack left when the
                               search stops (bottom first), if it holds <= out_cap records */
    int64_t out_cap;
    int64_t *out_count;     /* host or NULL: records left on the stack */
    int profile;            /* nonzero: fill the *_ms phase times of fsp_stats */
    int64_t tune_window;    /* iterations per tuning trial (pool_size = 0); 0 = 8 */
    int64_t *schedule_out;  /* host or NULL: pool size used by each iteration (replayable
                               through `schedule`), up to schedule_out_cap entries */
    int64_t schedule_out_cap;
    int order;              /* FSP_ORDER_PLAIN (default) or FSP_ORDER_LEARNED: each parent's
                               features go through `model`; its children first evaluate
                               only the `topk` best-scored machine pairs, and a child whose
                               partial bound already reaches the UB of the iteration is cut;
                               the others get the full bound.  Cuts, survivors, counters and
                               the incumbent are those of the plain order.  Shapes without a
                               fast-path kernel run the plain order. */
    int topk;               /* pairs evaluated first (1..8); 0 = 4 */
    fsp_mlp *model;         /* network with 2m+1 inputs and m(m-1)/2 outputs (order = learned) */
    uint8_t *log_nodes;     /* device or NULL: the children of each iteration are appended
                               here (training data) until log_cap records are stored */
    int64_t log_cap;
    int64_t *log_count;     /* host or NULL: records stored in log_nodes */
    int32_t *log_lbs;       /* device or NULL: with log_nodes, the bound of each logged
                               record (log_cap entries; in the learned order a child cut
                               by its predicted pairs logs that partial bound, which is
                               >= the UB of its iteration) */
    int branching;          /* FSP_BRANCH_FORWARD (default): a node is a scheduled prefix
                               and its children append a job (Sec. II-B).
                               FSP_BRANCH_BIDIR: a node is a prefix, a suffix and the jobs
                               between them (records of fsp_node_stride_bidir(n) bytes,
                               bound of fsp_bound_pool_bidir); a parent with prefix length
                               d1 <= suffix length d2 appends a job to the prefix, otherwise
                               puts one in front of the suffix; a child with one job left
                               is its completion.  Starts from the root (init_nodes must be
                               NULL), plain order, base bound, no node logging; out_nodes
                               receives bidirectional records. */
    int warps;              /* block shape of the search's bounding kernel where it bounds
                               each parent's children together: warps per CTA, 1..20; 0 =
                               the most whose tables fit (with pool_size = 0, chosen among
                               4, 8, 12 and that most on measured throughput).  The search
                               does not depend on it.  FSP_ERR_ARG if its tables do not fit
                               a CTA; ignored by the per-child kernels of other shapes. */
} fsp_options;

#define FSP_BRANCH_FORWARD 0
#define FSP_BRANCH_BIDIR 1

/* Fill *opt with the defaults (pool 1024, no budget, default capacity). */
int fsp_default_options(fsp_options *opt);

/* Bytes per node record for n jobs: n + 1 rounded up to 16. */
int fsp_node_stride(int n);

/* Sec. II-B instance.  p: host, n*m int32, job-major (p[j*m + k]), each in
 * 1..32767; 1 <= n <= 255, 2 <= m <= 64.  Copies p to the current device and
 * builds the per-instance tables there (one kernel; synchronous).  *out
 * receives a handle to release with fsp_destroy_instance.
 * Errors: FSP_ERR_ARG (shape or values), FSP_ERR_OOM, FSP_ERR_CUDA. */
int fsp_create_instance(int n, int m, const int32_t *p, fsp_instance **out);

/* Release the instance and its device tables (synchronises its device). */
void fsp_destroy_instance(fsp_instance *inst);

/* Bound variants (an instance setting, used by every later fsp_bound_pool and
 * fsp_solve on it; fsp_batch_* always use the base bound).
 * FSP_BOUND_BASE: the bound of Sec. V-D as read here (one-machine bounds and
 *   two-machine Johnson bounds with lags over every machine pair).
 * FSP_BOUND_HEADS: the same bound with each machine's release time raised to
 *   the earliest start of any remaining job, R_0 = C_0 and
 *   R_k = max(C_k, R_{k-1} + min over the remaining jobs of p[j][k-1]) (a
 *   refinement of the Lageweg-Lenstra-Rinnooy Kan family of bounds; never
 *   below the base bound, equal to it at depth n-1).  No counterpart in the
 *   paper, which plans other bounds as future work (Sec. VI). */
#define FSP_BOUND_BASE 0
#define FSP_BOUND_HEADS 1
/* Set the bound variant of inst.  Errors: FSP_ERR_ARG (NULL inst or unknown
 * variant). */
int fsp_set_bound(fsp_instance *inst, int variant);

/* Copy the device tables back for inspection (synchronous).  Any pointer may
 * be NULL.  q: host n*m int32 (q[j*m+k] = time of job j after machine k);
 * lag: host P*n int32; order: host P*n uint8 (Johnson order of pair kl);
 * pairs numbered k-major: (0,1), (0,2), ..., (0,m-1), (1,2), ... */
int fsp_instance_tables(const fsp_instance *inst, int32_t *q, int32_t *lag, uint8_t *order);

/* Sec. III parallel bounding (Type 1 model): the bound of `count` node
 * records.  nodes: device, count * fsp_node_stride(n) bytes.  lb_out: device,
 * count int32.  Every node gets its full bound, whatever `ub` (reserved for
 * modes that stop early once a partial bound reaches ub).  Asynchronous on
 * `stream`.  A malformed record (depth > n, a job id >= n or repeated) gets
 * FSP_LB_INVALID and sets the instance's error flag, which fsp_check_status
 * reports.  Errors (immediate): FSP_ERR_ARG for count < 0 or NULL buffers,
 * FSP_ERR_CUDA for a failed launch. */
int fsp_bound_pool(fsp_instance *inst, const uint8_t *nodes, int64_t count, int32_t ub,
                   int32_t *lb_out, void *stream);

/* Bidirectional nodes (no counterpart in the paper, which branches forward
 * only, Sec. II-B; it leaves other branchings to future work, Sec. VI).  A
 * record of fsp_node_stride_bidir(n) = n + 2 rounded up to 16 bytes holds a
 * permutation of 0..n-1 whose first d1 entries are the scheduled prefix,
 * whose last d2 entries are the scheduled suffix (both in schedule order) and
 * whose middle holds the remaining set U in any order; byte n holds d1, byte
 * n+1 holds d2 (d1 + d2 <= n), the rest is zero. */
int fsp_node_stride_bidir(int n);

/* The bound of `count` bidirectional records (device, count x
 * fsp_node_stride_bidir(n) bytes) into lb_out (device, count int32): the
 * bound of fsp_bound_pool with each machine's tail qmin_k replaced by
 * T_k = max(D_k, qmin_k), where D_k, the suffix's delivery time, is the
 * length of the longest path from the suffix's first job on machine k to its
 * last job on machine m-1 (after machine k finishes U it still runs the
 * suffix, and the last job of U still visits the machines after k).  With no
 * suffix it is fsp_bound_pool's bound (base variant); with U empty it is the
 * makespan.  Malformed records (d1 + d2 > n, not a permutation) get
 * FSP_LB_INVALID and set the error flag fsp_check_status reports.
 * Asynchronous on `stream`.  Errors (immediate): FSP_ERR_ARG (count < 0, NULL
 * or misaligned buffers), FSP_ERR_CUDA. */
int fsp_bound_pool_bidir(fsp_instance *inst, const uint8_t *nodes, int64_t count, int32_t *lb_out, void *stream);

/* Synchronise `stream` and report (then clear) the instance's error flag:
 * FSP_ERR_ARG if a malformed record was seen since the last check. */
int fsp_check_status(fsp_instance *inst, void *stream);

/* Device scratch bytes fsp_solve needs with these options (opt may be NULL). */
int64_t fsp_solve_workspace_bytes(const fsp_instance *inst, const fsp_options *opt);

/* Exact branch-and-bound (Sec. II-A operators, Sec. III pool of deepest
 * nodes), entirely on the device.  The search starts from the root (nothing
 * scheduled) with UB = ub0 (FSP_UB_INF = none) and repeats: pop parents from
 * the top of the depth-first stack while their children fit in the pool
 * (at least one parent); bound every child (children of a parent in
 * increasing job index of the appended job); complete schedules (depth n-1)
 * lower the UB, first in that order winning ties; keep the other children
 * whose bound is below the UB; push the survivors so the first is on top.
 * A search resumes from a checkpoint by passing the stack it left
 * (out_nodes) as init_nodes together with its cmax as ub0 and its permutation
 * as ub0_perm.
 * Outputs: *cmax = final UB (the optimum when the search completes); perm:
 * host, n int32, receives the optimal permutation if the search improved on
 * ub0 (else opt->ub0_perm if given, else left untouched); stats (may be NULL).
 * Returns FSP_OK, FSP_INCOMPLETE (node or iteration budget reached; cmax is
 * the best so far),
 * FSP_ERR_CAPACITY (stack full; nothing was lost), FSP_ERR_ARG, FSP_ERR_OOM
 * or FSP_ERR_CUDA.  Synchronous. */
int fsp_solve(fsp_instance *inst, int32_t ub0, int32_t *cmax, int32_t *perm, fsp_stats *stats,
              const fsp_options *opt);

/* Bytes of the fixed scratch array fsp_solve_noalloc uses (16 MiB). */
#define FSP_NOALLOC_SCRATCH_BYTES (16u << 20)

/* fsp_solve without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc while they
 * run -- processes whose device memory is reserved up front by a pool or a
 * fixed budget, plugins handed only their input and output buffers, and
 * paths where cudaMalloc's implicit synchronisation of the device is not
 * acceptable.  It runs the same search as fsp_solve, with the same
 * arguments, options and results, but its scratch is a device array of
 * FSP_NOALLOC_SCRATCH_BYTES that the library defines at file scope; every
 * device that loads the library holds that array until the process exits.
 *   - It allocates nothing (no cudaMalloc, cudaFree, cudaMallocHost, CUDA
 *     event or other allocating call), from the first call on a newly
 *     created instance on: its one pinned read-back block and two read-back
 *     events are reserved by fsp_create_instance for this entry point alone
 *     (fsp_instance_host_objects counts what an instance has created).  It
 *     therefore reports time_ms and the phase times as 0; opt->profile has
 *     no effect.  opt->workspace must be NULL; the learned order and node
 *     logging are refused (FSP_ERR_ARG).
 *   - The instance's device must be current.  Every call looks up the
 *     array's device address (cudaGetSymbolAddress) with that device
 *     current; the first call on a device also loads the library's device
 *     code there, so make it before any stream capture on that device.
 *   - A search whose scratch (fsp_solve_workspace_bytes) exceeds
 *     FSP_NOALLOC_SCRATCH_BYTES is rejected with FSP_ERR_CAPACITY and a
 *     message; nothing runs.
 *   - All calls share the one array: it keeps the last call's contents
 *     (every search initialises what it reads), and calls whose work overlaps
 *     on the GPU -- on different streams or host threads -- race on it.
 *     Serialise them. */
int fsp_solve_noalloc(fsp_instance *inst, int32_t ub0, int32_t *cmax, int32_t *perm, fsp_stats *stats,
                      const fsp_options *opt);

/* Host-side CUDA objects an instance has created so far: pinned read-back
 * blocks (cudaMallocHost) and CUDA events, counting the block and the two
 * events fsp_create_instance reserves for fsp_solve_noalloc.  Either pointer
 * (host) may be NULL.  A diagnostic with no counterpart in the paper: a
 * caller checks with it that a call created nothing.  Errors: FSP_ERR_ARG
 * (NULL inst). */
int fsp_instance_host_objects(const fsp_instance *inst, int64_t *pinned_blocks, int64_t *events);

/* NEH insertion heuristic on the device (an initial UB; the paper starts
 * from a given UB and has no counterpart): jobs by decreasing total time
 * (ties: smaller index first), each inserted at the position of smallest
 * partial makespan (ties: earliest position).  cmax: host, the makespan;
 * perm: host, n int32.  Synchronous. */
int fsp_neh(fsp_instance *inst, int32_t *cmax, int32_t *perm);

/* The pool-size tuner of fsp_solve (pool_size = 0; Sec. III, Algorithm 1)
 * run against a score function instead of measured throughput: trial k uses
 * pools_out[k] (host, up to cap entries) and receives score(pool, user).
 * Starts at nodes_per_cta x sms, doubles while the pool stays <= max_pool
 * (keeping the best score so far), then binary-searches around the best.  Returns the
 * number of trials (<= 64) and the best pool in *best_out (may be NULL), or
 * FSP_ERR_ARG.  Pure host code. */
int64_t fsp_tune_simulate(int64_t nodes_per_cta, int sms, int64_t max_pool,
                          double (*score)(int64_t pool, void *user), void *user, int64_t *pools_out,
                          int64_t cap, int64_t *best_out);

/* The block-shape tuner of fsp_solve (pool_size = 0, after the pool tuner
 * settles; the shape the paper's tuner also varies, Sec. III) run against a
 * score function: candidate shapes 0..ncand-1 (the family kernel's warps per
 * CTA, fewest first), one iteration per step.  It starts from the last
 * candidate, discards one warm-up iteration, then gives every candidate in
 * turn (last, 0, 1, ...) `window` iterations, adding score(cand, user) nodes
 * per iteration, and keeps the highest nodes per iteration (ties: the one
 * tried first).  cands_out (host, up to cap entries) receives the candidate
 * of each iteration.  Returns the number of iterations and the kept
 * candidate in *best_out (may be NULL), or FSP_ERR_ARG.  Pure host code. */
int64_t fsp_block_tune_simulate(int ncand, int64_t window, double (*score)(int64_t cand, void *user), void *user,
                                int64_t *cands_out, int64_t cap, int64_t *best_out);

/* ---------------------------------------------------------------------
 * Learned pair ordering (not in the paper; see fsp_options.order).  A small MLP scores the m(m-1)/2
 * machine pairs of a node from its features so that the pair most likely to
 * give the node's largest two-machine bound is evaluated first.
 * Features of a node (2m+1 float32): C_k / T, S_k / T for k < m (release
 * times, remaining work), d / n, with T = float32(total time) / float32(m).
 * Label: the first pair (k-major) whose two-machine bound is the largest.
 * Network: x -> relu(x W1 + b1) -> relu(. W2 + b2) -> . W3 + b3; the weights
 * are used as bf16 (nearest even) and every product accumulates in fp32 on
 * the tensor cores; inputs, hidden activations and back-propagated errors
 * are rounded to bf16 where they enter a product.  Parameters (fp32 master
 * copy, flat): W1 [F][H], b1 [H], W2 [H][H], b2 [H], W3 [H][P], b3 [P].
 * --------------------------------------------------------------------- */

/* Features (x: device, count x (2m+1) float32) and labels (label: device,
 * count int32, may be NULL) of count node records (device).  Asynchronous. */
int fsp_node_features(fsp_instance *inst, const uint8_t *nodes, int64_t count, float *x, int32_t *label,
                      void *stream);

/* A network with F inputs, H hidden units per layer, P outputs; weights
 * Glorot-uniform from a hash of (seed, index), biases 0.  Synchronous. */
int fsp_mlp_create(int in_dim, int hidden, int out_dim, uint64_t seed, fsp_mlp **out);
void fsp_mlp_destroy(fsp_mlp *mlp);
int64_t fsp_mlp_num_params(const fsp_mlp *mlp);
/* Copy the fp32 parameters out (host) / in (host; resets the optimiser). */
int fsp_mlp_get_params(const fsp_mlp *mlp, float *host);
int fsp_mlp_set_params(fsp_mlp *mlp, const float *host);
/* scores (device, B x P) = network(X) for X (device, B x F float32).  Async. */
int fsp_mlp_forward(fsp_mlp *mlp, const float *X, int64_t B, float *scores, void *stream);
/* Mean softmax cross-entropy of X (device, B x F) against labels (device, B)
 * and its gradient: loss (host, may be NULL; synchronises), grad (device or
 * host, num_params floats, may be NULL). */
int fsp_mlp_loss_grad(fsp_mlp *mlp, const float *X, const int32_t *labels, int64_t B, float *loss, float *grad,
                      void *stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) on that loss; loss (host, may be NULL). */
int fsp_mlp_train_step(fsp_mlp *mlp, const float *X, const int32_t *labels, int64_t B, float lr, float *loss,
                       void *stream);

/* The k (1..8) best-scored machine pairs of each of count node records
 * (device) by the network (128 hidden units, 2m+1 inputs, m(m-1)/2 outputs,
 * m in {5, 10, 20}), best first, ties to the lower pair index: topk (device, count x k
 * int16), pair numbering k-major.  The fused tensor-core kernel the learned
 * search uses on its parents.  Synchronous. */
int fsp_pair_order(fsp_instance *inst, fsp_mlp *mlp, const uint8_t *nodes, int64_t count, int k, int16_t *topk,
                   void *stream);

/* ---------------------------------------------------------------------
 * Batches: many instances of mixed shape solved in one persistent launch
 * (not in the paper, which solves one instance at a time).  Each CTA takes
 * the next instance from a device work queue and runs the whole search of
 * fsp_solve for it (same rules, the instance's own pool size) with the
 * NEH makespan as initial UB (or the given ub0), under the instance's node
 * budget.  Instances are grouped into classes of one shape and one block
 * shape (warps per CTA, 8 by default, set per instance with
 * fsp_batch_set_warps); each class is one launch of the persistent kernel
 * with its own CTA size, shared memory, grid (its occupancy times the SMs)
 * and work queue, and the launches of all classes are parallel branches of
 * one CUDA graph, captured at creation and replayed by fsp_batch_run.
 * Shapes: m = 5 or 10 with n <= 15, 16..31 or 48..63 jobs, and m = 20 with
 * 16..31 jobs.
 * --------------------------------------------------------------------- */
typedef struct fsp_batch fsp_batch;

typedef struct {
    int32_t cmax;              /* best makespan found (the optimum when status = FSP_OK) */
    int32_t status;            /* FSP_OK, FSP_INCOMPLETE (budget), FSP_ERR_CAPACITY, or
                                  FSP_ERR_TIMEOUT (split mode: a wait on the donations ran
                                  out, so the result may miss a subtree) */
    int64_t nodes_bounded, nodes_branched, nodes_pruned, leaves, iterations, incumbent_updates;
    int64_t pool;              /* pool size used */
} fsp_batch_result;

/* count instances: shapes (host, count x {n, m}), p_flat (host, the n*m
 * job-major times of each instance back to back), pools (host, count, 1..4096),
 * budgets (host or NULL: nodes; 0 = none), ub0 (host or NULL: initial UB;
 * 0 = NEH).  Uploads the data, sizes the per-CTA scratch and captures the
 * graph.  Errors: FSP_ERR_ARG (shape, pool or time out of range), FSP_ERR_OOM,
 * FSP_ERR_CUDA. */
int fsp_batch_create(int count, const int32_t *shapes, const int32_t *p_flat, const int64_t *pools,
                     const int64_t *budgets, const int32_t *ub0, fsp_batch **out);
void fsp_batch_destroy(fsp_batch *batch);
/* Launch the captured graph on `stream` (asynchronous); every launch solves
 * all instances again from scratch. */
int fsp_batch_run(fsp_batch *batch, void *stream);
/* Synchronise `stream` and copy the results out: res (host, count), perms
 * (host or NULL, count x 255 int32: instance i's permutation at i*255; valid
 * when the UB came from NEH or improved). */
int fsp_batch_results(fsp_batch *batch, fsp_batch_result *res, int32_t *perms, void *stream);
/* Split mode (on != 0; off by default, and again with on = 0): the work
 * queue holds the subtrees of the roots instead of whole instances -- for
 * each instance (the ones with the most jobs first) the n subtrees whose
 * schedules start with job 0, 1, ..., n-1 -- so idle CTAs take parts of the
 * instances still being searched instead of waiting for them; once the
 * queue is empty, a CTA still searching hands the bottom nodes of its stack
 * (its largest subtrees) to CTAs waiting for work.  A CTA that finishes an
 * item first takes the donated nodes still waiting, so every donated node is
 * searched; every wait on the donations (for the lock, for a node) ends after
 * 1 s, and an instance whose donated nodes could not be taken in that time
 * gets status FSP_ERR_TIMEOUT (the kernel returns; the context stays usable).  The CTAs
 * working on an instance share its UB (an atomic minimum, read before every
 * iteration) and its node count: the node budget then caps the instance's
 * total.  Results: the optimum (status FSP_OK) and a schedule attaining
 * cmax, like the whole-instance mode; the counters are the instance's
 * totals over its subtrees, explored in another order than one stack's, so
 * they differ from the whole-instance search's.  Re-captures the graph.
 * Errors: FSP_ERR_ARG, FSP_ERR_OOM, FSP_ERR_CUDA. */
int fsp_batch_set_split(fsp_batch *batch, int on);

/* Test hook for the wait limit of split mode (on != 0; off with on = 0): every
 * launch starts with each class's donation lock taken and one donated node
 * marked waiting, and nothing releases them, so every wait on the donations
 * runs out (1 s each) and every instance whose items finish gets status
 * FSP_ERR_TIMEOUT.  No fault, trap or endless wait.  Not in the paper.
 * Re-captures the graph.  Errors: FSP_ERR_ARG, FSP_ERR_CUDA. */
int fsp_batch_set_test_hold(fsp_batch *batch, int on);

/* Bidirectional branching (on != 0; FSP_BRANCH_BIDIR of fsp_options) for
 * every instance of the batch, in either mode; off again with on = 0.
 * Whole-instance mode then runs the search of fsp_solve with branching =
 * FSP_BRANCH_BIDIR (from the root, NEH UB or the given ub0).  Needs a
 * bidirectional batch shape for every instance (records of n + 2 bytes: not
 * n = 30, 31 or 63).  Re-captures the graph.  Errors: FSP_ERR_ARG (a shape
 * without the kernel; nothing changes), FSP_ERR_CUDA. */
int fsp_batch_set_bidir(fsp_batch *batch, int on);

/* Pool size per shape on measured throughput (Algorithm 1's purpose, per
 * shape): up to 8 instances of each shape run with pools 128 .. 4096 under
 * probe_budget nodes each; the fastest pool (nodes bounded per second) is
 * written for every instance of that shape to pools_out (host, count). */
int fsp_batch_tune_pools(int count, const int32_t *shapes, const int32_t *p_flat, int64_t probe_budget,
                         int64_t *pools_out);

/* Block shape per instance: warps (host, count; 0 = the default 8, else
 * 1..20) warps per CTA of the launch that solves it; NULL resets all to 8.
 * Instances of one shape with one block shape form a class (one launch).
 * The results do not depend on the block shape (whole-instance searches are
 * the same search; split mode reaches the same optima).  Synchronises the
 * device, rebuilds the classes' scratch and re-captures the graph.  Errors:
 * FSP_ERR_ARG (a count outside 0..20, or a block shape whose shared memory
 * does not fit a CTA; nothing changes), FSP_ERR_OOM, FSP_ERR_CUDA. */
int fsp_batch_set_warps(fsp_batch *batch, const int32_t *warps);

/* Load balance of the last completed fsp_batch_run: one entry per class
 * (instances of one shape run with one block shape, in launch order), from
 * the global timer each persistent CTA reads when it starts and when it
 * leaves (no work left in its queue).  Times in ms from the earliest CTA
 * start of the whole launch; launch_span_ms is the time from that start to
 * the last CTA's exit, the same for every class.  Synchronises the device.
 * out (host, cap entries) may be NULL when cap = 0; *count receives the
 * number of classes.  Errors: FSP_ERR_ARG, FSP_ERR_CUDA. */
typedef struct {
    int32_t n, m, warps;   /* the class: shape and warps per CTA */
    int32_t ctas;          /* CTAs of its launch */
    int32_t instances;     /* its instances */
    int32_t items;         /* its work items (instances, or split-mode subtrees) */
    int32_t donated;       /* split mode: nodes its CTAs handed to CTAs waiting for work */
    double busy_mean_ms, busy_min_ms, busy_max_ms;  /* CTA lifetimes */
    double first_start_ms, last_end_ms;             /* its first CTA start, its last CTA exit */
    double launch_span_ms;
} fsp_batch_class_info;

int fsp_batch_class_stats(fsp_batch *batch, fsp_batch_class_info *out, int cap, int *count);

/* Block shape per shape on measured throughput: for each shape, up to 8 of
 * its instances (pools from `pools`, probe_budget nodes each), repeated until
 * their split-mode items fill every SM twice at 4 warps per CTA, run as one
 * split-mode batch with 4, 8, 12, 16 and 20 warps per CTA (those whose shared memory
 * fits); the block shape with the most nodes bounded per second is written
 * for every instance of that shape to warps_out (host, count).  Not in the
 * paper, which tunes the pool size only (Algorithm 1). */
int fsp_batch_tune_warps(int count, const int32_t *shapes, const int32_t *p_flat, const int64_t *pools,
                         int64_t probe_budget, int32_t *warps_out);

/* Message of the last error on this thread ("" if none). */
const char *fsp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FSP_H */
