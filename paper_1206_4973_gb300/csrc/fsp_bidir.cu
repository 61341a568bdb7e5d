// fsp_bidir.cu -- bidirectional branching: nodes with a scheduled prefix, a
// scheduled suffix and the remaining set between them.
//
// The paper branches forward only (a node is a scheduled prefix, Sec. II-B)
// and leaves other bounds and branching schemes to future work (Sec. VI).
// Here a record holds the prefix sigma1 = perm[0..d1), the suffix sigma2 =
// perm[n-d2..n) (both in schedule order) and the remaining set U =
// perm[d1..n-d2) in increasing job order; d1 sits at byte n, d2 at byte n+1.
// A parent with d1 <= d2 branches forward (its children append a job of U to
// sigma1), otherwise backward (its children put a job of U in front of
// sigma2), so the two ends alternate.
//
// The bound (fsp.h, fsp_bound_pool_bidir): the suffix enters through its
// delivery times D_k, the length of the longest path from the suffix's first
// job on machine k to the end (the release-time recurrence run backwards);
// after machine k finishes U it still runs the suffix (D_k) and the last job
// of U still visits machines > k (qmin_k), so the tail after machine k is
// T_k = max(D_k, qmin_k), used where the forward bound uses qmin_k.  A child
// with one job left has a single completion and gets its makespan.
#include "fsp_solve.cuh"

extern "C" int fsp_node_stride_bidir(int n) { return (n + 2 + 15) / 16 * 16; }

// Any instance, one thread per node, tables from global memory (the packed
// kernel of fsp_pool16.cu takes the eligible instances).
__global__ void __launch_bounds__(128) k_bound_bidir_generic(DevInst I, const uint8_t *__restrict__ nodes,
                                                             long long count, const long long *dcount, int stride,
                                                             int32_t *__restrict__ lb_out)
{
    if (dcount) count = *dcount;
    const int n = I.n, m = I.m;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < count;
         t += (long long)gridDim.x * blockDim.x) {
        const uint8_t *r = nodes + t * stride;
        const int d1 = r[n], d2 = r[n + 1];
        uint32_t U[8] = {0, 0, 0, 0, 0, 0, 0, 0}, seen[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        bool bad = d1 + d2 > n;
        for (int i = 0; i < n; ++i) {
            const int j = r[i];
            if (j >= n || (seen[j >> 5] >> (j & 31)) & 1u) { bad = true; break; }
            seen[j >> 5] |= 1u << (j & 31);
            if (i >= d1 && i < n - d2) U[j >> 5] |= 1u << (j & 31);
        }
        if (bad) {
            lb_out[t] = FSP_LB_INVALID;
            atomicOr(I.status, 1);
            continue;
        }
        int32_t C[FSP_MAX_MACHINES], D[FSP_MAX_MACHINES], SQ[FSP_MAX_MACHINES];
        for (int k = 0; k < m; ++k) { C[k] = 0; D[k] = 0; }
        for (int i = 0; i < d1; ++i) {
            const int32_t *row = I.p + r[i] * m;
            C[0] += row[0];
            for (int k = 1; k < m; ++k) C[k] = max(C[k], C[k - 1]) + row[k];
        }
        for (int i = n - 1; i >= n - d2; --i) {  // the suffix from its last job
            const int32_t *row = I.p + r[i] * m;
            D[m - 1] += row[m - 1];
            for (int k = m - 2; k >= 0; --k) D[k] = max(D[k], D[k + 1]) + row[k];
        }
        int32_t lb = 0;
        for (int k = 0; k < m; ++k) {
            int32_t s = 0, q = 0x7fffffff;
            for (int i = d1; i < n - d2; ++i) {
                s += I.p[r[i] * m + k];
                q = min(q, I.q[r[i] * m + k]);
            }
            SQ[k] = s + max(D[k], q == 0x7fffffff ? 0 : q);
            lb = max(lb, C[k] + SQ[k]);
        }
        // pairs: t_l = S_l + max(C_l, C_k + M), M = max over U of (E_{<i} + w_i)
        const FspEntry *e = I.ent;
        for (int k = 0; k < m - 1; ++k)
            for (int l = k + 1; l < m; ++l, e += n) {
                int32_t E = 0, M = FSP_NEG;
                for (int pos = 0; pos < n; ++pos) {
                    const FspEntry x = e[pos];
                    if (U[x.widx] & x.bit) {
                        M = max(M, E + x.w);
                        E += x.e;
                    }
                }
                lb = max(lb, SQ[l] + max(C[l], C[k] + M));
            }
        lb_out[t] = lb;
    }
}

// The children of the popped parents, one thread per child: parent p (from
// the first-child offsets), its remaining job of rank ci placed at the end
// the parent's depths choose.
__global__ void __launch_bounds__(256) k_bidir_children(SolveWs ws, int n, int stride)
{
    const SolveCtl *ctl = ws.ctl;
    const long long nch = ctl->n_children;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nch) return;
    const int np = (int)ctl->n_parents;
    const int pi = solve_parent_of(ws.poff, np, c);
    const int ci = (int)(c - ws.poff[pi]);
    const long long S = ctl->s_pop + np;  // the stack before the pops; parent 0 was on top
    const uint8_t *par = ws.stack + (S - 1 - pi) * stride;
    uint8_t *ch = ws.children + c * stride;
    const int d1 = par[n], d2 = par[n + 1];
    const bool forward = d1 <= d2;
    const int j = par[d1 + ci];
    for (int i = 0; i < d1; ++i) ch[i] = par[i];
    int o = d1;
    if (forward) ch[o++] = (uint8_t)j;
    for (int i = d1; i < n - d2; ++i)
        if (i != d1 + ci) ch[o++] = par[i];
    if (!forward) ch[o++] = (uint8_t)j;
    for (int i = n - d2; i < n; ++i) ch[i] = par[i];
    ch[n] = (uint8_t)(forward ? d1 + 1 : d1);
    ch[n + 1] = (uint8_t)(forward ? d2 : d2 + 1);
    for (int i = n + 2; i < stride; ++i) ch[i] = 0;
}

// Children with one job left are complete schedules: their value is the
// makespan (the bound kernel's value is replaced), and one below the
// iteration's UB competes for the incumbent (first child on ties).
__global__ void __launch_bounds__(256) k_bidir_leaves(SolveWs ws, const int32_t *__restrict__ p, int n, int m,
                                                      int stride)
{
    const SolveCtl *ctl = ws.ctl;
    const long long nch = ctl->n_children;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nch) return;
    const uint8_t *ch = ws.children + c * stride;
    if (ch[n] + ch[n + 1] != n - 1) return;
    int32_t C[FSP_MAX_MACHINES];
    for (int k = 0; k < m; ++k) C[k] = 0;
    for (int i = 0; i < n; ++i) {
        const int32_t *row = p + ch[i] * m;
        C[0] += row[0];
        for (int k = 1; k < m; ++k) C[k] = max(C[k], C[k - 1]) + row[k];
    }
    const int32_t v = C[m - 1];
    ws.lbs[c] = v;
    if (v < ctl->ub_iter)
        atomicMin(&ws.ctl->best_key, ((unsigned long long)(uint32_t)v << 32) | (unsigned long long)c);
}

// Bound count bidirectional records (count read on the device when dcount
// is not NULL; then count is an upper bound that sizes the grid).
int bidir_bound(fsp_instance *I, const uint8_t *nodes, long long count, const long long *dcount, int32_t *lb_out,
                cudaStream_t st)
{
    if (pool16_bound_ex(I, nodes, count, dcount, true, lb_out, st, 0) == FSP_OK) return FSP_OK;
    if (count <= 0) return FSP_OK;
    long long grid = (count + 127) / 128;
    if (grid > (long long)I->sm_count * 16) grid = (long long)I->sm_count * 16;
    k_bound_bidir_generic<<<(unsigned)grid, 128, 0, st>>>(dev_view(I), nodes, count, dcount,
                                                          fsp_node_stride_bidir(I->n), lb_out);
    FSP_CUDA(cudaGetLastError());
    return FSP_OK;
}

void bidir_launch_children(const SolveWs &ws, int n, int stride, long long max_children, cudaStream_t st)
{
    const unsigned grid = (unsigned)((max_children + 255) / 256);
    k_bidir_children<<<grid, 256, 0, st>>>(ws, n, stride);
}

void bidir_launch_leaves(const SolveWs &ws, const fsp_instance *I, int stride, long long max_children,
                         cudaStream_t st)
{
    const unsigned grid = (unsigned)((max_children + 255) / 256);
    k_bidir_leaves<<<grid, 256, 0, st>>>(ws, I->d_p, I->n, I->m, stride);
}

extern "C" int fsp_bound_pool_bidir(fsp_instance *I, const uint8_t *nodes, int64_t count, int32_t *lb_out,
                                    void *stream)
{
    if (!I) { fsp_set_error("fsp_bound_pool_bidir: inst is NULL"); return FSP_ERR_ARG; }
    if (count < 0) { fsp_set_error("fsp_bound_pool_bidir: count < 0"); return FSP_ERR_ARG; }
    if (count == 0) return FSP_OK;
    if (!nodes || !lb_out) { fsp_set_error("fsp_bound_pool_bidir: NULL buffer"); return FSP_ERR_ARG; }
    if (((uintptr_t)nodes & 15) != 0) {
        fsp_set_error("fsp_bound_pool_bidir: nodes must be 16-byte aligned");
        return FSP_ERR_ARG;
    }
    if (getenv("FSP_BOUND_V1")) {  // the generic kernel whatever the instance (tests)
        long long grid = (count + 127) / 128;
        if (grid > (long long)I->sm_count * 16) grid = (long long)I->sm_count * 16;
        k_bound_bidir_generic<<<(unsigned)grid, 128, 0, (cudaStream_t)stream>>>(
            dev_view(I), nodes, count, nullptr, fsp_node_stride_bidir(I->n), lb_out);
        FSP_CUDA(cudaGetLastError());
        return FSP_OK;
    }
    return bidir_bound(I, nodes, count, nullptr, lb_out, (cudaStream_t)stream);
}
