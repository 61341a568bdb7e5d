/*
 * fsp_oracle.c -- plain, serial CPU oracle for the permutation flow-shop
 * branch-and-bound of Chakroun & Melab, "An Adaptative Multi-GPU based
 * Branch-and-Bound. A Case Study: the Flow-Shop Scheduling Problem".
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this code.  It shares no
 * source, header, table or helper with the CUDA library: it recomputes every
 * table from the processing times with the plainest loops that follow the
 * definitions, in the paper's order, so that a reader can check it by eye.
 *
 * All arithmetic is int32 (processing times 1..32767, n <= 255, m <= 64, so
 * every sum stays below 2^31).
 *
 * Definitions followed (the paper prints no lower-bound formula; it states
 * only the O(m^2 n log n) cost in Sec. V-D, which is the two-machine Johnson
 * bound with time lags over all machine pairs):
 *   problem, permutation schedule ........... Sec. II-B
 *   node = scheduled prefix + remaining set .. Sec. II-B (node i = job J_i first)
 *   bounding / elimination / selection ....... Sec. II-A
 *   pool of deepest nodes per iteration ...... Sec. III, Algorithm 1
 *   insertion heuristic (NEH) for the first UB: not in the paper.
 *
 * Pins (checked by tests/test_oracle_pins.py, none of them re-uses this code):
 *   makespan            brute-force schedule simulation, hand-worked 2x2/3x3
 *   Johnson with lags   brute force over every order of the remaining set
 *   lower bound         <= makespan of every completion (brute force, n <= 8)
 *                       == makespan at depth n-1 and n
 *                       == optimum at m = 2 (Johnson's theorem)
 *   solver optimum      brute force over all n! permutations (n <= 9)
 *   solver counts       pool size 1: a recursive textbook DFS;
 *                       ub0 = optimum: the order-free closed set of survivors
 *   The exact interleaving of a pool > 1 search once the incumbent improves
 *   has no independent pin: parity unpinned beyond the invariants above.
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_INCOMPLETE 1
#define ORC_ERR_ARG (-1)
#define ORC_ERR_OOM (-3)

#define ORC_MAXN 255
#define ORC_MAXM 64

static int32_t imax(int32_t a, int32_t b) { return a > b ? a : b; }
static int32_t imin(int32_t a, int32_t b) { return a < b ? a : b; }

/* p is job-major: p[j*m + k] is the time of job j on machine k (Sec. II-B). */
static int32_t pt(const int32_t *p, int m, int j, int k) { return p[(size_t)j * m + k]; }

int orc_num_pairs(int m) { return m * (m - 1) / 2; }

/* Machine pairs (k, l), k < l, numbered k-major: (0,1), (0,2), ..., (1,2), ... */
int orc_pair_index(int m, int k, int l)
{
    int idx = 0;
    for (int a = 0; a < m; a++)
        for (int b = a + 1; b < m; b++) {
            if (a == k && b == l) return idx;
            idx++;
        }
    return -1;
}

/* Sec. II-B: completion times of the jobs perm[0..len) processed in that order
 * on every machine.  C[k] after the loop is the completion time of the last
 * job on machine k ("release time" of machine k for the rest of the jobs). */
void orc_release_times(int n, int m, const int32_t *p, const uint8_t *perm, int len, int32_t *C)
{
    (void)n;
    for (int k = 0; k < m; k++) C[k] = 0;
    for (int i = 0; i < len; i++) {
        int j = perm[i];
        C[0] = C[0] + pt(p, m, j, 0);
        for (int k = 1; k < m; k++) C[k] = imax(C[k], C[k - 1]) + pt(p, m, j, k);
    }
}

/* Makespan = completion time of the last job on the last machine. */
int32_t orc_makespan(int n, int m, const int32_t *p, const uint8_t *perm, int len)
{
    int32_t C[ORC_MAXM];
    orc_release_times(n, m, p, perm, len, C);
    return len > 0 ? C[m - 1] : 0;
}

/* Tails: q[j][k] = sum of job j's times on the machines after k. */
void orc_tails(int n, int m, const int32_t *p, int32_t *q)
{
    for (int j = 0; j < n; j++)
        for (int k = 0; k < m; k++) {
            int32_t s = 0;
            for (int h = k + 1; h < m; h++) s += pt(p, m, j, h);
            q[(size_t)j * m + k] = s;
        }
}

/* Lags of the two-machine relaxation on pair (k,l): lag[kl][j] = sum of job
 * j's times on the machines strictly between k and l (the minimum delay
 * between its end on k and its start on l). */
void orc_lags(int n, int m, const int32_t *p, int32_t *lag)
{
    int kl = 0;
    for (int k = 0; k < m; k++)
        for (int l = k + 1; l < m; l++) {
            for (int j = 0; j < n; j++) {
                int32_t s = 0;
                for (int h = k + 1; h < l; h++) s += pt(p, m, j, h);
                lag[(size_t)kl * n + j] = s;
            }
            kl++;
        }
}

/* Johnson's rule with time lags for pair (k,l): with a_j = p[j][k],
 * b_j = p[j][l], lag_j: first the jobs with a_j <= b_j by increasing
 * a_j + lag_j, then the jobs with a_j > b_j by decreasing b_j + lag_j; equal
 * keys keep the smaller job index first.  Returns 1 when job i goes before
 * job j. */
static int johnson_before(int i, int j, int32_t ai, int32_t bi, int32_t li,
                          int32_t aj, int32_t bj, int32_t lj)
{
    int gi = ai <= bi ? 0 : 1;
    int gj = aj <= bj ? 0 : 1;
    if (gi != gj) return gi < gj;
    if (gi == 0) {
        if (ai + li != aj + lj) return ai + li < aj + lj;
    } else {
        if (bi + li != bj + lj) return bi + li > bj + lj;
    }
    return i < j;
}

/* order[kl][pos] = job at position pos of pair kl's Johnson order (insertion
 * sort: the n log n of Sec. V-D is this sort, done once per instance here). */
void orc_johnson_orders(int n, int m, const int32_t *p, const int32_t *lag, uint8_t *order)
{
    int kl = 0;
    for (int k = 0; k < m; k++)
        for (int l = k + 1; l < m; l++) {
            uint8_t *o = order + (size_t)kl * n;
            const int32_t *lg = lag + (size_t)kl * n;
            for (int t = 0; t < n; t++) {
                int j = t, pos = t;
                while (pos > 0) {
                    int i = o[pos - 1];
                    if (johnson_before(j, i, pt(p, m, j, k), pt(p, m, j, l), lg[j],
                                       pt(p, m, i, k), pt(p, m, i, l), lg[i])) {
                        o[pos] = o[pos - 1];
                        pos--;
                    } else {
                        break;
                    }
                }
                o[pos] = (uint8_t)j;
            }
            kl++;
        }
}

/* 1 if perm[0..n) is a permutation of 0..n-1 and 0 <= d <= n. */
int orc_check_node(int n, const uint8_t *perm, int d)
{
    int seen[ORC_MAXN + 1];
    if (d < 0 || d > n) return 0;
    for (int j = 0; j < n; j++) seen[j] = 0;
    for (int i = 0; i < n; i++) {
        if (perm[i] >= n || seen[perm[i]]) return 0;
        seen[perm[i]] = 1;
    }
    return 1;
}

/* The node bound.  The node is perm[0..d) scheduled (prefix), perm[d..n)
 * remaining (set U, any order).
 *   C_k      release time of machine k after the prefix (Sec. II-B)
 *   S_k      sum over U of p[j][k]
 *   qmin_k   min over U of q[j][k], 0 when U is empty
 *   LB1      max_k C_k + S_k + qmin_k                       (one machine)
 *   LB_kl    t_k = C_k, t_l = C_l; for j of U in Johnson order of (k,l):
 *              t_k += a_j; t_l = max(t_l, t_k + lag_j) + b_j;
 *            LB_kl = t_l + qmin_l                            (two machines)
 *   LB       max(LB1, max over pairs LB_kl)
 * variant 1 (release times strengthened by the smallest head, one of the
 * refinements of the Lageweg-Lenstra-Rinnooy Kan family of bounds): a
 * remaining job starts on machine k only after the prefix frees k and after
 * it has been processed on machine k-1, so with U non-empty
 *     R_0 = C_0,   R_k = max(C_k, R_{k-1} + min over U of p[j][k-1]),
 * and every C_k above is replaced by R_k (variant 0: R = C).
 * lb1_out (may be NULL) receives LB1; pair_out (may be NULL) receives the
 * m(m-1)/2 values LB_kl in pair order. */
int32_t orc_lb(int n, int m, const int32_t *p, const int32_t *q, const int32_t *lag,
               const uint8_t *order, const uint8_t *perm, int d, int variant,
               int32_t *lb1_out, int32_t *pair_out)
{
    int32_t C[ORC_MAXM], S[ORC_MAXM], qmin[ORC_MAXM];
    int inU[ORC_MAXN + 1];

    orc_release_times(n, m, p, perm, d, C);
    for (int j = 0; j < n; j++) inU[j] = 0;
    for (int i = d; i < n; i++) inU[perm[i]] = 1;

    for (int k = 0; k < m; k++) {
        int32_t s = 0, mn = 0;
        int first = 1;
        for (int j = 0; j < n; j++) {
            if (!inU[j]) continue;
            s += pt(p, m, j, k);
            if (first || q[(size_t)j * m + k] < mn) mn = q[(size_t)j * m + k];
            first = 0;
        }
        S[k] = s;
        qmin[k] = mn;
    }

    if (variant == 1 && d < n) {
        /* the smallest time any remaining job spends on machine k-1 */
        for (int k = 1; k < m; k++) {
            int32_t mn = 0;
            int first = 1;
            for (int j = 0; j < n; j++) {
                if (!inU[j]) continue;
                if (first || pt(p, m, j, k - 1) < mn) mn = pt(p, m, j, k - 1);
                first = 0;
            }
            C[k] = imax(C[k], C[k - 1] + mn);  /* C[k-1] already holds R_{k-1} */
        }
    }

    int32_t lb1 = 0;
    for (int k = 0; k < m; k++) lb1 = imax(lb1, C[k] + S[k] + qmin[k]);
    if (lb1_out) *lb1_out = lb1;

    int32_t lb = lb1;
    int kl = 0;
    for (int k = 0; k < m; k++)
        for (int l = k + 1; l < m; l++) {
            const uint8_t *o = order + (size_t)kl * n;
            const int32_t *lg = lag + (size_t)kl * n;
            int32_t tk = C[k], tl = C[l];
            for (int pos = 0; pos < n; pos++) {
                int j = o[pos];
                if (!inU[j]) continue;
                tk = tk + pt(p, m, j, k);
                tl = imax(tl, tk + lg[j]) + pt(p, m, j, l);
            }
            int32_t v = tl + qmin[l];
            if (pair_out) pair_out[kl] = v;
            lb = imax(lb, v);
            kl++;
        }
    return lb;
}

/* Instance tables recomputed from p (tails, lags, Johnson orders). */
typedef struct {
    int n, m, npairs;
    int32_t *q, *lag;
    uint8_t *order;
} orc_tables;

static int tables_make(orc_tables *t, int n, int m, const int32_t *p)
{
    t->n = n;
    t->m = m;
    t->npairs = orc_num_pairs(m);
    t->q = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * m);
    t->lag = (int32_t *)malloc(sizeof(int32_t) * (size_t)(t->npairs > 0 ? t->npairs : 1) * n);
    t->order = (uint8_t *)malloc((size_t)(t->npairs > 0 ? t->npairs : 1) * n);
    if (!t->q || !t->lag || !t->order) return ORC_ERR_OOM;
    orc_tails(n, m, p, t->q);
    orc_lags(n, m, p, t->lag);
    orc_johnson_orders(n, m, p, t->lag, t->order);
    return ORC_OK;
}

static void tables_free(orc_tables *t)
{
    free(t->q);
    free(t->lag);
    free(t->order);
}

static int shape_ok(int n, int m, const int32_t *p)
{
    if (n < 1 || n > ORC_MAXN || m < 2 || m > ORC_MAXM || !p) return 0;
    for (size_t i = 0; i < (size_t)n * m; i++)
        if (p[i] < 1 || p[i] > 32767) return 0;
    return 1;
}

/* Bound a pool of node records: record t is nodes[t*stride ..], perm bytes
 * 0..n-1, depth at byte n.  Returns ORC_ERR_ARG if any record is invalid. */
int orc_bound_pool(int n, int m, const int32_t *p, const uint8_t *nodes, int64_t count,
                   int stride, int variant, int32_t *lb_out)
{
    orc_tables t;
    if (!shape_ok(n, m, p) || count < 0 || stride < n + 1) return ORC_ERR_ARG;
    if (tables_make(&t, n, m, p) != ORC_OK) { tables_free(&t); return ORC_ERR_OOM; }
    int rc = ORC_OK;
    for (int64_t i = 0; i < count; i++) {
        const uint8_t *rec = nodes + (size_t)i * stride;
        if (!orc_check_node(n, rec, rec[n])) { rc = ORC_ERR_ARG; break; }
        lb_out[i] = orc_lb(n, m, p, t.q, t.lag, t.order, rec, rec[n], variant, NULL, NULL);
    }
    tables_free(&t);
    return rc;
}

/* The same pool bound with the nodes split over `threads` host threads
 * (OpenMP; 0 = all the host's cores): each node's bound is orc_lb exactly
 * as above, only the loop over nodes runs in parallel.  For the all-core
 * CPU baseline.  Returns the number of threads used, or ORC_ERR_ARG /
 * ORC_ERR_OOM. */
int orc_bound_pool_threads(int n, int m, const int32_t *p, const uint8_t *nodes, int64_t count, int stride,
                           int variant, int32_t *lb_out, int threads)
{
    orc_tables t;
    if (!shape_ok(n, m, p) || count < 0 || stride < n + 1 || threads < 0) return ORC_ERR_ARG;
    if (tables_make(&t, n, m, p) != ORC_OK) { tables_free(&t); return ORC_ERR_OOM; }
    int used = threads > 0 ? threads : omp_get_max_threads();
    int bad = 0;
#pragma omp parallel for num_threads(used) schedule(static) reduction(| : bad)
    for (int64_t i = 0; i < count; i++) {
        const uint8_t *rec = nodes + (size_t)i * stride;
        if (!orc_check_node(n, rec, rec[n])) { bad = 1; continue; }
        lb_out[i] = orc_lb(n, m, p, t.q, t.lag, t.order, rec, rec[n], variant, NULL, NULL);
    }
    tables_free(&t);
    return bad ? ORC_ERR_ARG : used;
}

/* Per-node parts: LB1 and every LB_kl of one node (for pins). */
int orc_lb_parts(int n, int m, const int32_t *p, const uint8_t *perm, int d, int variant,
                 int32_t *lb_out, int32_t *lb1_out, int32_t *pair_out)
{
    orc_tables t;
    if (!shape_ok(n, m, p) || !orc_check_node(n, perm, d)) return ORC_ERR_ARG;
    if (tables_make(&t, n, m, p) != ORC_OK) { tables_free(&t); return ORC_ERR_OOM; }
    *lb_out = orc_lb(n, m, p, t.q, t.lag, t.order, perm, d, variant, lb1_out, pair_out);
    tables_free(&t);
    return ORC_OK;
}

/* Table dump (for pins on the tables themselves). */
int orc_tables_dump(int n, int m, const int32_t *p, int32_t *q, int32_t *lag, uint8_t *order)
{
    if (!shape_ok(n, m, p)) return ORC_ERR_ARG;
    orc_tails(n, m, p, q);
    orc_lags(n, m, p, lag);
    orc_johnson_orders(n, m, p, lag, order);
    return ORC_OK;
}

/* Exhaustive search over all n! permutations in lexicographic order; returns
 * the optimum and the lexicographically first optimal permutation. */
int32_t orc_bruteforce(int n, int m, const int32_t *p, uint8_t *best_perm)
{
    uint8_t perm[ORC_MAXN];
    int32_t best = 0;
    int have = 0;
    for (int i = 0; i < n; i++) perm[i] = (uint8_t)i;
    for (;;) {
        int32_t c = orc_makespan(n, m, p, perm, n);
        if (!have || c < best) {
            best = c;
            have = 1;
            memcpy(best_perm, perm, (size_t)n);
        }
        /* next permutation in lexicographic order */
        int i = n - 2;
        while (i >= 0 && perm[i] >= perm[i + 1]) i--;
        if (i < 0) break;
        int j = n - 1;
        while (perm[j] <= perm[i]) j--;
        uint8_t tmp = perm[i]; perm[i] = perm[j]; perm[j] = tmp;
        for (int a = i + 1, b = n - 1; a < b; a++, b--) {
            tmp = perm[a]; perm[a] = perm[b]; perm[b] = tmp;
        }
    }
    return best;
}

/* NEH insertion heuristic (not in the paper; gives the first UB): jobs by
 * decreasing total time (ties: smaller index first), each inserted at the
 * position of smallest partial makespan (ties: earliest position). */
int32_t orc_neh(int n, int m, const int32_t *p, uint8_t *perm_out)
{
    int order[ORC_MAXN];
    int32_t tot[ORC_MAXN];
    uint8_t seq[ORC_MAXN], trial[ORC_MAXN];
    for (int j = 0; j < n; j++) {
        tot[j] = 0;
        for (int k = 0; k < m; k++) tot[j] += pt(p, m, j, k);
        order[j] = j;
    }
    for (int a = 1; a < n; a++) { /* insertion sort, stable */
        int j = order[a], b = a;
        while (b > 0 && tot[order[b - 1]] < tot[j]) { order[b] = order[b - 1]; b--; }
        order[b] = j;
    }
    int len = 0;
    for (int t = 0; t < n; t++) {
        int job = order[t], best_pos = 0;
        int32_t best = 0;
        for (int pos = 0; pos <= len; pos++) {
            int w = 0;
            for (int i = 0; i < pos; i++) trial[w++] = seq[i];
            trial[w++] = (uint8_t)job;
            for (int i = pos; i < len; i++) trial[w++] = seq[i];
            int32_t c = orc_makespan(n, m, p, trial, len + 1);
            if (pos == 0 || c < best) { best = c; best_pos = pos; }
        }
        for (int i = len; i > best_pos; i--) seq[i] = seq[i - 1];
        seq[best_pos] = (uint8_t)job;
        len++;
    }
    memcpy(perm_out, seq, (size_t)n);
    return orc_makespan(n, m, p, seq, n);
}

/* ------------------------------------------------------------------------ */
/* Serial pool-synchronous depth-first branch-and-bound (Sec. II-A, III).    */
/* ------------------------------------------------------------------------ */

enum { ST_BOUNDED = 0, ST_BRANCHED, ST_PRUNED, ST_LEAVES, ST_ITERATIONS, ST_UPDATES, ST_N };

typedef struct {
    uint8_t *rec; /* records of n+1 bytes: perm[0..n), depth */
    int64_t size, cap;
    int w;
} orc_stack;

static int stack_push(orc_stack *s, const uint8_t *perm, int d)
{
    if (s->size == s->cap) {
        int64_t nc = s->cap ? s->cap * 2 : 1024;
        uint8_t *r = (uint8_t *)realloc(s->rec, (size_t)nc * s->w);
        if (!r) return ORC_ERR_OOM;
        s->rec = r;
        s->cap = nc;
    }
    memcpy(s->rec + (size_t)s->size * s->w, perm, (size_t)(s->w - 1));
    s->rec[(size_t)s->size * s->w + s->w - 1] = (uint8_t)d;
    s->size++;
    return ORC_OK;
}

/*
 * Search rules (the paper fixes the operators, Sec. II-A, and the pool of
 * deepest nodes, Sec. III; the rest is this project's reading):
 *   - stack = [root: identity permutation, depth 0]; UB = ub0 (INT32_MAX = +inf)
 *   - each iteration pops parents from the top while the children counted so
 *     far plus this parent's (n - depth) fit in the pool size; at least one.
 *   - children list L: parents in pop order, each parent's children by
 *     increasing job index of the job appended; a child's remaining set is
 *     kept in increasing job order.
 *   - all of L is bounded; children at depth n-1 are complete schedules
 *     (their bound is their makespan): in L order, a bound < UB becomes the
 *     new UB and incumbent.  Every other child survives iff bound < UB, with
 *     UB as just updated (elimination prunes bound >= UB).
 *   - survivors are pushed in reverse L order, so L's first is on top.
 * schedule (may be NULL): pool size of each iteration (the last entry repeats),
 * to replay a tuned run.  trace (may be NULL): per iteration
 * {parents, children, survivors, UB after}, up to trace_cap iterations.
 * node_budget > 0 stops before an iteration once that many nodes are bounded,
 * max_iterations > 0 once that many iterations ran (both return
 * ORC_INCOMPLETE).  init (may be NULL): init_count records of rec_stride bytes
 * (perm, depth at byte n; depth <= n-2) form the starting stack, bottom
 * first, instead of the root.  out (may be NULL): receives the stack left at
 * the end (bottom first, rec_stride bytes per record) if it holds at most
 * out_cap records; *out_count (may be NULL) its size.
 */
int orc_solve(int n, int m, const int32_t *p, int32_t ub0, int64_t pool, int64_t node_budget,
              const int64_t *schedule, int64_t schedule_len,
              const uint8_t *init, int64_t init_count, int rec_stride, int64_t max_iterations,
              int32_t *cmax, uint8_t *perm_out, int64_t *stats,
              int64_t *trace, int64_t trace_cap,
              uint8_t *out, int64_t out_cap, int64_t *out_count, int variant)
{
    if (!shape_ok(n, m, p) || pool < 1 || variant < 0 || variant > 1) return ORC_ERR_ARG;
    if ((init || out) && rec_stride < n + 1) return ORC_ERR_ARG;
    if (init)
        for (int64_t i = 0; i < init_count; i++) {
            const uint8_t *r = init + (size_t)i * rec_stride;
            if (n < 2 || !orc_check_node(n, r, r[n]) || r[n] > n - 2) return ORC_ERR_ARG;
        }
    for (int i = 0; i < ST_N; i++) stats[i] = 0;
    int32_t UB = ub0;

    if (n == 1) { /* the root is already a complete schedule */
        uint8_t only = 0;
        int32_t c = orc_makespan(n, m, p, &only, 1);
        if (c < UB) { UB = c; perm_out[0] = 0; stats[ST_UPDATES] = 1; }
        *cmax = UB;
        return ORC_OK;
    }

    orc_tables t;
    if (tables_make(&t, n, m, p) != ORC_OK) { tables_free(&t); return ORC_ERR_OOM; }
    const int w = n + 1;
    orc_stack st = {NULL, 0, 0, w};
    uint8_t *parents = NULL, *children = NULL;
    int32_t *lbs = NULL;
    int64_t par_cap = 0, ch_cap = 0;
    int rc = ORC_OK;

    if (init) {
        for (int64_t i = 0; i < init_count; i++) {
            const uint8_t *r = init + (size_t)i * rec_stride;
            if ((rc = stack_push(&st, r, r[n])) != ORC_OK) goto done;
        }
    } else {
        uint8_t root[ORC_MAXN];
        for (int i = 0; i < n; i++) root[i] = (uint8_t)i;
        if ((rc = stack_push(&st, root, 0)) != ORC_OK) goto done;
    }

    int64_t it = 0;
    while (st.size > 0) {
        if (node_budget > 0 && stats[ST_BOUNDED] >= node_budget) { rc = ORC_INCOMPLETE; break; }
        if (max_iterations > 0 && it >= max_iterations) { rc = ORC_INCOMPLETE; break; }
        int64_t psz = pool;
        if (schedule && schedule_len > 0) psz = schedule[it < schedule_len ? it : schedule_len - 1];
        if (psz < 1) psz = 1;

        /* selection: deepest (top-of-stack) parents while their children fit */
        int64_t np = 0, nch = 0;
        while (st.size > 0) {
            const uint8_t *top = st.rec + (size_t)(st.size - 1) * w;
            int64_t r = n - top[n];
            if (np > 0 && nch + r > psz) break;
            if (np == par_cap) {
                par_cap = par_cap ? par_cap * 2 : 256;
                uint8_t *x = (uint8_t *)realloc(parents, (size_t)par_cap * w);
                if (!x) { rc = ORC_ERR_OOM; goto done; }
                parents = x;
            }
            memcpy(parents + (size_t)np * w, top, (size_t)w);
            np++;
            nch += r;
            st.size--;
        }

        /* branching: one child per remaining job, by increasing job index */
        if (nch > ch_cap) {
            ch_cap = nch;
            uint8_t *x = (uint8_t *)realloc(children, (size_t)ch_cap * w);
            int32_t *y = (int32_t *)realloc(lbs, sizeof(int32_t) * (size_t)ch_cap);
            if (x) children = x;
            if (y) lbs = y;
            if (!x || !y) { rc = ORC_ERR_OOM; goto done; }
        }
        int64_t c = 0;
        for (int64_t a = 0; a < np; a++) {
            const uint8_t *par = parents + (size_t)a * w;
            int d = par[n];
            uint8_t rem[ORC_MAXN];
            int r = 0;
            for (int i = d; i < n; i++) rem[r++] = par[i];
            for (int x = 1; x < r; x++) { /* increasing job index */
                uint8_t v = rem[x];
                int y = x;
                while (y > 0 && rem[y - 1] > v) { rem[y] = rem[y - 1]; y--; }
                rem[y] = v;
            }
            for (int ci = 0; ci < r; ci++) {
                uint8_t *ch = children + (size_t)c * w;
                memcpy(ch, par, (size_t)d);
                ch[d] = rem[ci];
                int o = d + 1;
                for (int x = 0; x < r; x++)
                    if (x != ci) ch[o++] = rem[x];
                ch[n] = (uint8_t)(d + 1);
                c++;
            }
        }

        /* bounding */
        for (int64_t i = 0; i < nch; i++) {
            const uint8_t *ch = children + (size_t)i * w;
            lbs[i] = orc_lb(n, m, p, t.q, t.lag, t.order, ch, ch[n], variant, NULL, NULL);
        }
        stats[ST_BOUNDED] += nch;
        stats[ST_BRANCHED] += np;

        /* complete schedules update the incumbent, in L order; the UB
         * changes once per iteration, so an update is counted per iteration */
        const int32_t ub_start = UB;
        for (int64_t i = 0; i < nch; i++) {
            const uint8_t *ch = children + (size_t)i * w;
            if (ch[n] != n - 1) continue;
            stats[ST_LEAVES]++;
            if (lbs[i] < UB) {
                UB = lbs[i];
                memcpy(perm_out, ch, (size_t)n);
            }
        }
        if (UB < ub_start) stats[ST_UPDATES]++;

        /* elimination, then push survivors in reverse L order */
        int64_t nsurv = 0;
        for (int64_t i = 0; i < nch; i++) {
            const uint8_t *ch = children + (size_t)i * w;
            if (ch[n] == n - 1) continue;
            if (lbs[i] < UB) nsurv++;
            else stats[ST_PRUNED]++;
        }
        for (int64_t i = nch - 1; i >= 0; i--) {
            const uint8_t *ch = children + (size_t)i * w;
            if (ch[n] == n - 1 || lbs[i] >= UB) continue;
            if ((rc = stack_push(&st, ch, ch[n])) != ORC_OK) goto done;
        }
        if (trace && it < trace_cap) {
            trace[it * 4 + 0] = np;
            trace[it * 4 + 1] = nch;
            trace[it * 4 + 2] = nsurv;
            trace[it * 4 + 3] = UB;
        }
        it++;
        stats[ST_ITERATIONS] = it;
    }
    *cmax = UB;
    if (out_count) *out_count = st.size;
    if (out && st.size <= out_cap)
        for (int64_t i = 0; i < st.size; i++) {
            uint8_t *dst = out + (size_t)i * rec_stride;
            memset(dst, 0, (size_t)rec_stride);
            memcpy(dst, st.rec + (size_t)i * w, (size_t)w);
        }

done:
    free(st.rec);
    free(parents);
    free(children);
    free(lbs);
    tables_free(&t);
    return rc;
}


/* ------------------------------------------------------------------------ */
/* Bidirectional branching.  The paper branches forward only (a node is a    */
/* scheduled prefix, Sec. II-B) and names other bounds and branchings as     */
/* future work (Sec. VI).  Here a node is a prefix sigma1 = perm[0..d1), a   */
/* suffix sigma2 = perm[n-d2..n) (both in schedule order) and the remaining  */
/* set U = perm[d1..n-d2) between them; a parent branches either forward     */
/* (append a job of U to sigma1) or backward (put a job of U in front of     */
/* sigma2).                                                                  */
/* ------------------------------------------------------------------------ */

/* 1 if perm[0..n) is a permutation of 0..n-1 and d1, d2 >= 0, d1 + d2 <= n. */
int orc_check_node2(int n, const uint8_t *perm, int d1, int d2)
{
    if (d1 < 0 || d2 < 0 || d1 + d2 > n) return 0;
    return orc_check_node(n, perm, 0);
}

/* Delivery times of a suffix (its jobs in schedule order): D_k = the length
 * of the longest path from the suffix's first job on machine k to its last
 * job on machine m-1, i.e. how long the schedule runs on after machine k
 * starts the suffix.  The release-time recurrence run backwards: jobs from
 * last to first, machines from m-1 down to 0, D_k = max(D_k, D_{k+1}) + p. */
void orc_delivery_times(int n, int m, const int32_t *p, const uint8_t *suffix, int len, int32_t *D)
{
    (void)n;
    for (int k = 0; k < m; k++) D[k] = 0;
    for (int i = len - 1; i >= 0; i--) {
        int j = suffix[i];
        for (int k = m - 1; k >= 0; k--) {
            int32_t later = k + 1 < m ? D[k + 1] : 0; /* this job, next machine */
            D[k] = imax(D[k], later) + pt(p, m, j, k); /* D[k]: the next suffix job, same machine */
        }
    }
}

/* The bound of a bidirectional node.  With C_k the release times of sigma1,
 * D_k the delivery times of sigma2, S_k and qmin_k the remaining sums and
 * smallest tails over U as in orc_lb:
 *   T_k    max(D_k, qmin_k): after machine k finishes U, it still runs sigma2
 *          (at least D_k) and the last job of U still visits machines > k
 *          (at least qmin_k);
 *   LB1    max_k C_k + S_k + T_k;
 *   LB_kl  the Johnson recurrence of orc_lb over U, t_l + T_l;
 *   LB     max(LB1, max over pairs LB_kl).
 * With sigma2 empty (D = 0, T = qmin) this is orc_lb's bound (variant 0);
 * with U empty it is the makespan max_k C_k + D_k. */
int32_t orc_lb2(int n, int m, const int32_t *p, const int32_t *q, const int32_t *lag, const uint8_t *order,
                const uint8_t *perm, int d1, int d2, int32_t *lb1_out, int32_t *pair_out)
{
    int32_t C[ORC_MAXM], D[ORC_MAXM], S[ORC_MAXM], qmin[ORC_MAXM], T[ORC_MAXM];
    int inU[ORC_MAXN + 1];

    orc_release_times(n, m, p, perm, d1, C);
    orc_delivery_times(n, m, p, perm + (n - d2), d2, D);
    for (int j = 0; j < n; j++) inU[j] = 0;
    for (int i = d1; i < n - d2; i++) inU[perm[i]] = 1;

    for (int k = 0; k < m; k++) {
        int32_t s = 0, mn = 0;
        int first = 1;
        for (int j = 0; j < n; j++) {
            if (!inU[j]) continue;
            s += pt(p, m, j, k);
            if (first || q[(size_t)j * m + k] < mn) mn = q[(size_t)j * m + k];
            first = 0;
        }
        S[k] = s;
        qmin[k] = mn;
        T[k] = imax(D[k], qmin[k]);
    }

    int32_t lb1 = 0;
    for (int k = 0; k < m; k++) lb1 = imax(lb1, C[k] + S[k] + T[k]);
    if (lb1_out) *lb1_out = lb1;

    int32_t lb = lb1;
    int kl = 0;
    for (int k = 0; k < m; k++)
        for (int l = k + 1; l < m; l++) {
            const uint8_t *o = order + (size_t)kl * n;
            const int32_t *lg = lag + (size_t)kl * n;
            int32_t tk = C[k], tl = C[l];
            for (int pos = 0; pos < n; pos++) {
                int j = o[pos];
                if (!inU[j]) continue;
                tk = tk + pt(p, m, j, k);
                tl = imax(tl, tk + lg[j]) + pt(p, m, j, l);
            }
            int32_t v = tl + T[l];
            if (pair_out) pair_out[kl] = v;
            lb = imax(lb, v);
            kl++;
        }
    return lb;
}

/* Bound a pool of bidirectional records: perm bytes 0..n-1, d1 at byte n,
 * d2 at byte n+1.  ORC_ERR_ARG if any record is invalid. */
int orc_bound_pool2(int n, int m, const int32_t *p, const uint8_t *nodes, int64_t count, int stride,
                    int32_t *lb_out)
{
    orc_tables t;
    if (!shape_ok(n, m, p) || count < 0 || stride < n + 2) return ORC_ERR_ARG;
    if (tables_make(&t, n, m, p) != ORC_OK) { tables_free(&t); return ORC_ERR_OOM; }
    int rc = ORC_OK;
    for (int64_t i = 0; i < count; i++) {
        const uint8_t *rec = nodes + (size_t)i * stride;
        if (!orc_check_node2(n, rec, rec[n], rec[n + 1])) { rc = ORC_ERR_ARG; break; }
        lb_out[i] = orc_lb2(n, m, p, t.q, t.lag, t.order, rec, rec[n], rec[n + 1], NULL, NULL);
    }
    tables_free(&t);
    return rc;
}

/* One bidirectional node's bound and parts (for pins). */
int orc_lb2_parts(int n, int m, const int32_t *p, const uint8_t *perm, int d1, int d2, int32_t *lb_out,
                  int32_t *lb1_out, int32_t *pair_out, int32_t *D_out)
{
    orc_tables t;
    if (!shape_ok(n, m, p) || !orc_check_node2(n, perm, d1, d2)) return ORC_ERR_ARG;
    if (tables_make(&t, n, m, p) != ORC_OK) { tables_free(&t); return ORC_ERR_OOM; }
    *lb_out = orc_lb2(n, m, p, t.q, t.lag, t.order, perm, d1, d2, lb1_out, pair_out);
    if (D_out) orc_delivery_times(n, m, p, perm + (n - d2), d2, D_out);
    tables_free(&t);
    return ORC_OK;
}

/*
 * Search with bidirectional branching: the rules of orc_solve with these
 * changes (records of n+2 bytes: perm, d1, d2):
 *   - root: identity permutation, d1 = d2 = 0; a node has r = n - d1 - d2
 *     children;
 *   - direction: a parent with d1 <= d2 branches forward (children append a
 *     job of U to sigma1), otherwise backward (children put a job of U in
 *     front of sigma2): the two ends alternate;
 *   - children of a parent by increasing index of the placed job; U stays in
 *     increasing job order between sigma1 and sigma2;
 *   - a child with one job left (d1 + d2 = n - 1) has a single completion:
 *     it is a complete schedule whose value is that completion's makespan;
 *     every other child gets orc_lb2.
 * Selection, incumbent updates (first in L order wins ties), elimination
 * (bound >= UB) and the push order are those of orc_solve.
 */
int orc_solve_bidir(int n, int m, const int32_t *p, int32_t ub0, int64_t pool, int64_t node_budget,
                    int64_t max_iterations, int32_t *cmax, uint8_t *perm_out, int64_t *stats, int64_t *trace,
                    int64_t trace_cap)
{
    if (!shape_ok(n, m, p) || pool < 1) return ORC_ERR_ARG;
    for (int i = 0; i < ST_N; i++) stats[i] = 0;
    int32_t UB = ub0;
    if (n == 1) {
        uint8_t only = 0;
        int32_t c = orc_makespan(n, m, p, &only, 1);
        if (c < UB) { UB = c; perm_out[0] = 0; stats[ST_UPDATES] = 1; }
        *cmax = UB;
        return ORC_OK;
    }
    orc_tables t;
    if (tables_make(&t, n, m, p) != ORC_OK) { tables_free(&t); return ORC_ERR_OOM; }
    const int w = n + 2;
    uint8_t *stack = NULL, *parents = NULL, *children = NULL;
    int32_t *lbs = NULL;
    int64_t ssz = 0, scap = 0, par_cap = 0, ch_cap = 0;
    int rc = ORC_OK;

    scap = 1024;
    stack = (uint8_t *)malloc((size_t)scap * w);
    if (!stack) { rc = ORC_ERR_OOM; goto done; }
    for (int i = 0; i < n; i++) stack[i] = (uint8_t)i;
    stack[n] = 0;
    stack[n + 1] = 0;
    ssz = 1;

    int64_t it = 0;
    while (ssz > 0) {
        if (node_budget > 0 && stats[ST_BOUNDED] >= node_budget) { rc = ORC_INCOMPLETE; break; }
        if (max_iterations > 0 && it >= max_iterations) { rc = ORC_INCOMPLETE; break; }

        /* selection: deepest parents while their children fit */
        int64_t np = 0, nch = 0;
        while (ssz > 0) {
            const uint8_t *top = stack + (size_t)(ssz - 1) * w;
            int64_t r = n - top[n] - top[n + 1];
            if (np > 0 && nch + r > pool) break;
            if (np == par_cap) {
                par_cap = par_cap ? par_cap * 2 : 256;
                uint8_t *x = (uint8_t *)realloc(parents, (size_t)par_cap * w);
                if (!x) { rc = ORC_ERR_OOM; goto done; }
                parents = x;
            }
            memcpy(parents + (size_t)np * w, top, (size_t)w);
            np++;
            nch += r;
            ssz--;
        }

        /* branching */
        if (nch > ch_cap) {
            ch_cap = nch;
            uint8_t *x = (uint8_t *)realloc(children, (size_t)ch_cap * w);
            int32_t *y = (int32_t *)realloc(lbs, sizeof(int32_t) * (size_t)ch_cap);
            if (x) children = x;
            if (y) lbs = y;
            if (!x || !y) { rc = ORC_ERR_OOM; goto done; }
        }
        int64_t c = 0;
        for (int64_t a = 0; a < np; a++) {
            const uint8_t *par = parents + (size_t)a * w;
            const int d1 = par[n], d2 = par[n + 1];
            const int forward = d1 <= d2;
            uint8_t rem[ORC_MAXN];
            int r = 0;
            for (int i = d1; i < n - d2; i++) rem[r++] = par[i];
            for (int x = 1; x < r; x++) { /* increasing job index */
                uint8_t v = rem[x];
                int y = x;
                while (y > 0 && rem[y - 1] > v) { rem[y] = rem[y - 1]; y--; }
                rem[y] = v;
            }
            for (int ci = 0; ci < r; ci++) {
                uint8_t *ch = children + (size_t)c * w;
                memcpy(ch, par, (size_t)w);
                int o = d1;
                if (forward) ch[o++] = rem[ci];
                for (int x = 0; x < r; x++)
                    if (x != ci) ch[o++] = rem[x];
                if (!forward) ch[o++] = rem[ci];
                ch[n] = (uint8_t)(forward ? d1 + 1 : d1);
                ch[n + 1] = (uint8_t)(forward ? d2 : d2 + 1);
                c++;
            }
        }

        /* bounding: a child with one job left is its completion */
        for (int64_t i = 0; i < nch; i++) {
            const uint8_t *ch = children + (size_t)i * w;
            if (ch[n] + ch[n + 1] == n - 1) lbs[i] = orc_makespan(n, m, p, ch, n);
            else lbs[i] = orc_lb2(n, m, p, t.q, t.lag, t.order, ch, ch[n], ch[n + 1], NULL, NULL);
        }
        stats[ST_BOUNDED] += nch;
        stats[ST_BRANCHED] += np;

        const int32_t ub_start = UB;
        for (int64_t i = 0; i < nch; i++) {
            const uint8_t *ch = children + (size_t)i * w;
            if (ch[n] + ch[n + 1] != n - 1) continue;
            stats[ST_LEAVES]++;
            if (lbs[i] < UB) {
                UB = lbs[i];
                memcpy(perm_out, ch, (size_t)n);
            }
        }
        if (UB < ub_start) stats[ST_UPDATES]++;

        int64_t nsurv = 0;
        for (int64_t i = 0; i < nch; i++) {
            const uint8_t *ch = children + (size_t)i * w;
            if (ch[n] + ch[n + 1] == n - 1) continue;
            if (lbs[i] < UB) nsurv++;
            else stats[ST_PRUNED]++;
        }
        for (int64_t i = nch - 1; i >= 0; i--) {
            const uint8_t *ch = children + (size_t)i * w;
            if (ch[n] + ch[n + 1] == n - 1 || lbs[i] >= UB) continue;
            if (ssz == scap) {
                scap *= 2;
                uint8_t *x = (uint8_t *)realloc(stack, (size_t)scap * w);
                if (!x) { rc = ORC_ERR_OOM; goto done; }
                stack = x;
            }
            memcpy(stack + (size_t)ssz * w, ch, (size_t)w);
            ssz++;
        }
        if (trace && it < trace_cap) {
            trace[it * 4 + 0] = np;
            trace[it * 4 + 1] = nch;
            trace[it * 4 + 2] = nsurv;
            trace[it * 4 + 3] = UB;
        }
        it++;
        stats[ST_ITERATIONS] = it;
    }
    *cmax = UB;
done:
    free(stack);
    free(parents);
    free(children);
    free(lbs);
    tables_free(&t);
    return rc;
}
