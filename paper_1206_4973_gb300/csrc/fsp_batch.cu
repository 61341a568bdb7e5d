// fsp_batch.cu -- many instances of mixed shape in one persistent launch:
// the host side, the forward-branching kernels and the split-mode passes
// (device code in fsp_batch.cuh; the bidirectional kernels in
// fsp_batch_bidir.cu).
#include <algorithm>
#include <chrono>
#include <vector>

#include "fsp_batch.cuh"

template __global__ void k_batch<false>(const BatchDesc *, int, const int32_t *, BatchOut *, uint8_t *, int *, BatchWs);
template __global__ void k_batch_split<false>(const BatchDesc *, const int32_t *, int *, BatchWs, BatchSplit);

// The bidirectional instantiations (fsp_batch_bidir.cu).
typedef void (*BatchFn)(const BatchDesc *, int, const int32_t *, BatchOut *, uint8_t *, int *, BatchWs);
typedef void (*BatchSplitFn)(const BatchDesc *, const int32_t *, int *, BatchWs, BatchSplit);
BatchFn batch_kernel_bidir();
BatchSplitFn batch_split_kernel_bidir();

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
    bool split = false, bidir = false;
    BatchSplit X{};
    int *d_item = nullptr;  // item instances, then item jobs
};

static bool batch_shape_ok(int n, int m, bool bidir = false)
{
    const int nv = (n + (bidir ? 2 : 1) + 15) / 16, nw = n <= 32 ? 1 : 2;
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
    const BatchFn kb = B->bidir ? batch_kernel_bidir() : &k_batch<false>;
    const BatchSplitFn ks = B->bidir ? batch_split_kernel_bidir() : &k_batch_split<false>;
    if (e == cudaSuccess && !B->split) {
        kb<<<B->grid, BB, B->smem, st>>>(B->d_desc, B->count, B->d_p, B->d_out, B->d_perms, B->d_queue, B->ws);
        e = cudaGetLastError();
    } else if (e == cudaSuccess) {
        k_batch_split_init<<<B->count, BB, 0, st>>>(B->d_desc, B->d_p, B->d_perms, B->X);
        ks<<<B->grid, BB, B->smem, st>>>(B->d_desc, B->d_p, B->d_queue, B->ws, B->X);
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
        smem_max = std::max(smem_max, std::max(batch_smem_nm(n, m), batch_smem_nm(n, m, true)));
        const int s = (n + 2 + 15) / 16 * 16;  // wide enough for bidirectional records
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
        const void *kern[4] = {(const void *)&k_batch<false>, (const void *)&k_batch_split<false>,
                               (const void *)batch_kernel_bidir(), (const void *)batch_split_kernel_bidir()};
        for (const void *k : kern)
            TRYB(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B->smem));
        int per_sm = 0, per_sm_b = 0;
        TRYB(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern[0], BB, B->smem));
        TRYB(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_b, kern[2], BB, B->smem));
        per_sm = std::min(per_sm, per_sm_b);
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

extern "C" int fsp_batch_set_bidir(fsp_batch *B, int on)
{
    if (!B) { fsp_set_error("fsp_batch_set_bidir: NULL batch"); return FSP_ERR_ARG; }
    if (on)
        for (int i = 0; i < B->count; ++i)
            if (!batch_shape_ok(B->desc[i].n, B->desc[i].m, true)) {
                fsp_set_error("fsp_batch_set_bidir: instance %d (%dx%d) has no bidirectional batch kernel", i,
                              B->desc[i].n, B->desc[i].m);
                return FSP_ERR_ARG;
            }
    B->bidir = on != 0;
    return batch_capture(B);
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
