// fsp_batch.cu -- many instances of mixed shape in one persistent launch:
// the host side, the forward-branching kernels and the split-mode passes
// (device code in fsp_batch.cuh; the bidirectional kernels in
// fsp_batch_bidir.cu).
#include <algorithm>
#include <chrono>
#include <vector>

#include "fsp_batch.cuh"

template __global__ void k_batch<false>(const BatchDesc *, const int *, int, const int32_t *, BatchOut *, uint8_t *,
                                        int *, BatchWs);
template __global__ void k_batch_split<false>(const BatchDesc *, const int *, int, const int32_t *, int *, BatchWs,
                                              BatchSplit);

// The bidirectional instantiations (fsp_batch_bidir.cu).
typedef void (*BatchFn)(const BatchDesc *, const int *, int, const int32_t *, BatchOut *, uint8_t *, int *, BatchWs);
typedef void (*BatchSplitFn)(const BatchDesc *, const int *, int, const int32_t *, int *, BatchWs, BatchSplit);
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
        o.status = (X.flags[i] & 4)   ? FSP_ERR_TIMEOUT
                   : (X.flags[i] & 2) ? FSP_ERR_CAPACITY
                   : (X.flags[i] & 1) ? FSP_INCOMPLETE
                                      : FSP_OK;
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

#define DQ_SLOTS 1024      // donated nodes waiting at a time, per class
#define DQ_IDS 16384       // donated nodes per class and launch at most (their item ids)
#define DQ_IDLE_CAP 4      // CTAs of one class that may wait for donations at a time: waiting CTAs hold
                           // SM slots the other classes' CTAs need (measured: 2-8 best, 16 and more slower)

// The instances of one shape that run with one block shape (warps per CTA):
// one launch of the persistent kernel with its own shared-memory size, grid,
// work list, queue and scratch.  The launches of all classes are parallel
// branches of the batch's graph.
struct BatchClass {
    int n, m, warps;
    std::vector<int> inst;   // instance indices, in batch order
    std::vector<int> items;  // their split-mode items, in item order
    int *d_list = nullptr;   // the instance indices, then the item indices
    size_t smem = 0;         // dynamic shared memory per CTA (the larger of forward and bidirectional)
    int grid_max = 0;        // CTAs the scratch holds
    int grid = 0;            // CTAs of the captured launch
    BatchWs ws{};
};

struct fsp_batch {
    int count, device, sm_count, optin;
    BatchDesc *d_desc;
    int32_t *d_p;
    BatchOut *d_out;
    uint8_t *d_perms;
    int *d_queue = nullptr;  // one counter per class, then 8 donation counters per class
    std::vector<BatchDesc> desc;
    std::vector<int> warps;  // block shape per instance
    std::vector<BatchClass> cls;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    bool split = false, bidir = false;
    bool hold = false;  // test hook: donation locks taken and a node marked waiting at every launch
    BatchSplit X{};
    int *d_item = nullptr;  // item instances, then item jobs
    std::vector<int> item_inst;
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

static void batch_free_classes(fsp_batch *B)
{
    for (BatchClass &c : B->cls) {
        cudaFree(c.d_list);
        cudaFree(c.ws.stack);
        cudaFree(c.ws.children);
        cudaFree(c.ws.lbs);
        cudaFree(c.ws.cta_ns);
        cudaFree(c.ws.slot_inst);
        cudaFree(c.ws.slot_id);
        cudaFree(c.ws.slot_rec);
    }
    B->cls.clear();
    cudaFree(B->d_queue);
    B->d_queue = nullptr;
}

static void batch_free(fsp_batch *B)
{
    if (!B) return;
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    batch_free_classes(B);
    cudaFree(B->d_desc); cudaFree(B->d_p); cudaFree(B->d_out); cudaFree(B->d_perms);
    cudaFree(B->d_item); cudaFree(B->X.ub); cudaFree(B->X.key); cudaFree(B->X.cnt); cudaFree(B->X.flags);
    cudaFree(B->X.item_perm);
    delete B;
}

static const void *batch_kernel(bool split, bool bidir)
{
    if (split) return bidir ? (const void *)batch_split_kernel_bidir() : (const void *)&k_batch_split<false>;
    return bidir ? (const void *)batch_kernel_bidir() : (const void *)&k_batch<false>;
}

// Dynamic shared memory a batch CTA may use: the opt-in limit less the
// kernels' static shared memory.
static int batch_smem_limit(int optin)
{
    size_t st = 0;
    for (int k = 0; k < 4; ++k) {
        cudaFuncAttributes a;
        if (cudaFuncGetAttributes(&a, batch_kernel(k & 1, k >> 1)) == cudaSuccess) st = std::max(st, a.sharedSizeBytes);
    }
    return optin - (int)st;
}

// Group the instances by (shape, warps) and give each class its lists, its
// shared-memory size, the most CTAs it can run at once (the four kernels'
// occupancy at its block shape) and its scratch.
static int batch_build_classes(fsp_batch *B)
{
    batch_free_classes(B);
    for (int i = 0; i < B->count; ++i) {
        const BatchDesc &d = B->desc[i];
        BatchClass *c = nullptr;
        for (BatchClass &x : B->cls)
            if (x.n == d.n && x.m == d.m && x.warps == B->warps[i]) c = &x;
        if (!c) {
            B->cls.emplace_back();
            c = &B->cls.back();
            c->n = d.n;
            c->m = d.m;
            c->warps = B->warps[i];
        }
        c->inst.push_back(i);
    }
    // the classes with the most work per instance (n x m) first: their launches go out first
    std::stable_sort(B->cls.begin(), B->cls.end(), [](const BatchClass &a, const BatchClass &b) {
        return a.n * a.m > b.n * b.m;
    });
    for (int it = 0; it < (int)B->item_inst.size(); ++it)
        for (BatchClass &x : B->cls) {
            const BatchDesc &d = B->desc[B->item_inst[it]];
            if (x.n == d.n && x.m == d.m && x.warps == B->warps[B->item_inst[it]]) x.items.push_back(it);
        }
    size_t smem_max = 0;
    for (BatchClass &c : B->cls) {
        c.smem = std::max(batch_smem_nm(c.n, c.m, false, c.warps), batch_smem_nm(c.n, c.m, true, c.warps));
        const int limit = batch_smem_limit(B->optin);
        if ((int)c.smem > limit) {
            fsp_set_error("fsp_batch: %dx%d instances with %d warps need %zu bytes of shared memory per CTA "
                          "(at most %d)", c.n, c.m, c.warps, c.smem, limit);
            return FSP_ERR_ARG;
        }
        smem_max = std::max(smem_max, c.smem);
    }
    for (int k = 0; k < 4; ++k)
        FSP_CUDA(cudaFuncSetAttribute(batch_kernel(k & 1, k >> 1), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem_max));
    const size_t nc = B->cls.size();
    FSP_CUDA(cudaMalloc(&B->d_queue, sizeof(int) * nc * 9));
    // split-mode schedules of the donated nodes follow the items' (ids items.. in class order)
    cudaFree(B->X.item_perm);
    B->X.item_perm = nullptr;
    FSP_CUDA(cudaMalloc(&B->X.item_perm, (size_t)FSP_MAX_JOBS * ((size_t)B->X.items + nc * DQ_IDS)));
    for (BatchClass &c : B->cls) {
        int per_sm = 1 << 30;
        for (int k = 0; k < 4; ++k) {
            int o = 0;
            FSP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, batch_kernel(k & 1, k >> 1), c.warps * 32,
                                                                   c.smem));
            per_sm = std::min(per_sm, o);
        }
        if (per_sm < 1) {
            fsp_set_error("fsp_batch: no CTA of %d warps fits an SM for %dx%d instances", c.warps, c.n, c.m);
            return FSP_ERR_ARG;
        }
        const int work = (int)std::max(c.inst.size(), c.items.size());
        c.grid_max = std::min(B->sm_count * per_sm, work);
        long long pool_max = 1;
        for (int i : c.inst) pool_max = std::max(pool_max, (long long)B->desc[i].pool);
        c.ws.stride_max = (c.n + 2 + 15) / 16 * 16;  // wide enough for bidirectional records
        c.ws.cap = (long long)c.n * (pool_max + c.n);
        c.ws.ch_cap = pool_max + c.n;
        const size_t g = (size_t)c.grid_max;
        FSP_CUDA(cudaMalloc(&c.ws.stack, g * c.ws.cap * c.ws.stride_max));
        FSP_CUDA(cudaMalloc(&c.ws.children, g * c.ws.ch_cap * c.ws.stride_max));
        FSP_CUDA(cudaMalloc(&c.ws.lbs, g * c.ws.ch_cap * sizeof(int32_t)));
        FSP_CUDA(cudaMalloc(&c.ws.cta_ns, g * 2 * sizeof(unsigned long long)));
        const size_t ci = (size_t)(&c - &B->cls[0]);
        c.ws.dq = B->d_queue + nc + 8 * ci;
        c.ws.slots = DQ_SLOTS;
        c.ws.ids_base = B->X.items + (int)ci * DQ_IDS;
        c.ws.ids_cap = DQ_IDS;
        c.ws.idle_cap = DQ_IDLE_CAP;
        FSP_CUDA(cudaMalloc(&c.ws.slot_inst, sizeof(int) * DQ_SLOTS));
        FSP_CUDA(cudaMalloc(&c.ws.slot_id, sizeof(int) * DQ_SLOTS));
        FSP_CUDA(cudaMalloc(&c.ws.slot_rec, (size_t)DQ_SLOTS * c.ws.stride_max));
        std::vector<int> list(c.inst);
        list.insert(list.end(), c.items.begin(), c.items.end());
        FSP_CUDA(cudaMalloc(&c.d_list, sizeof(int) * list.size()));
        FSP_CUDA(cudaMemcpy(c.d_list, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice));
    }
    return FSP_OK;
}

// The graph: the queues cleared; (split) the instances' UBs; every class's
// persistent kernel on a branch of its own; (split) the results.
static int batch_capture(fsp_batch *B)
{
    if (B->exec) { cudaGraphExecDestroy(B->exec); B->exec = nullptr; }
    if (B->graph) { cudaGraphDestroy(B->graph); B->graph = nullptr; }
    const int nc = (int)B->cls.size();
    cudaStream_t st;
    FSP_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    std::vector<cudaStream_t> side(nc, nullptr);
    std::vector<cudaEvent_t> done(nc, nullptr);
    cudaEvent_t fork = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (int c = 0; c < nc && e == cudaSuccess; ++c) {
        e = cudaStreamCreateWithFlags(&side[c], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done[c], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    const bool capturing = e == cudaSuccess;
    if (e == cudaSuccess) e = cudaMemsetAsync(B->d_queue, 0, sizeof(int) * nc * 9, st);
    for (int c = 0; c < nc && e == cudaSuccess && B->hold; ++c) {  // lock = 1, one node waiting = 1
        e = cudaMemsetAsync(B->d_queue + nc + 8 * c, 1, 1, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(B->d_queue + nc + 8 * c + 1, 1, 1, st);
    }
    if (e == cudaSuccess && B->split) {
        k_batch_split_init<<<B->count, BB, 0, st>>>(B->d_desc, B->d_p, B->d_perms, B->X);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(fork, st);
    const BatchFn kb = B->bidir ? batch_kernel_bidir() : &k_batch<false>;
    const BatchSplitFn ks = B->bidir ? batch_split_kernel_bidir() : &k_batch_split<false>;
    for (int c = 0; c < nc && e == cudaSuccess; ++c) {
        BatchClass &C = B->cls[c];
        e = cudaStreamWaitEvent(side[c], fork, 0);
        if (e != cudaSuccess) break;
        const int len = B->split ? (int)C.items.size() : (int)C.inst.size();
        const int grid = std::min(C.grid_max, len);
        C.grid = grid;
        if (grid > 0) {
            if (B->split)
                ks<<<grid, C.warps * 32, C.smem, side[c]>>>(B->d_desc, C.d_list + C.inst.size(), len, B->d_p,
                                                             B->d_queue + c, C.ws, B->X);
            else
                kb<<<grid, C.warps * 32, C.smem, side[c]>>>(B->d_desc, C.d_list, len, B->d_p, B->d_out, B->d_perms,
                                                             B->d_queue + c, C.ws);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(done[c], side[c]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, done[c], 0);
    }
    if (e == cudaSuccess && B->split) {
        k_batch_split_finish<<<B->count, 64, 0, st>>>(B->d_desc, B->count, B->d_out, B->d_perms, B->X);
        e = cudaGetLastError();
    }
    if (capturing) {
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(st, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&B->exec, g, 0);
        B->graph = g;
    }
    for (int c = 0; c < nc; ++c) {
        if (side[c]) cudaStreamDestroy(side[c]);
        if (done[c]) cudaEventDestroy(done[c]);
    }
    if (fork) cudaEventDestroy(fork);
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
    }
    B->warps.assign(count, BB / 32);
    // split-mode work items: the instances with the most work (n x m) first,
    // each as the n subtrees of its root (the root itself when n <= 2)
    std::vector<int> order(count), item_job;
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (long long)B->desc[a].n * B->desc[a].m > (long long)B->desc[b].n * B->desc[b].m;
    });
    for (int i : order) {
        if (B->desc[i].n <= 2) {
            B->item_inst.push_back(i);
            item_job.push_back(-1);
            continue;
        }
        for (int j = 0; j < B->desc[i].n; ++j) { B->item_inst.push_back(i); item_job.push_back(j); }
    }
    const int items = (int)B->item_inst.size();
    int rc = FSP_OK;
    cudaError_t e;
#define TRYB(call) do { e = (call); if (e != cudaSuccess) { rc = fsp_cuda_fail(e, #call); goto fail; } } while (0)
    TRYB(cudaGetDevice(&B->device));
    TRYB(cudaDeviceGetAttribute(&B->sm_count, cudaDevAttrMultiProcessorCount, B->device));
    TRYB(cudaDeviceGetAttribute(&B->optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, B->device));
    TRYB(cudaMalloc(&B->d_desc, sizeof(BatchDesc) * count));
    TRYB(cudaMalloc(&B->d_p, sizeof(int32_t) * off));
    TRYB(cudaMalloc(&B->d_out, sizeof(BatchOut) * count));
    TRYB(cudaMalloc(&B->d_perms, (size_t)FSP_MAX_JOBS * count));
    TRYB(cudaMemcpy(B->d_desc, B->desc.data(), sizeof(BatchDesc) * count, cudaMemcpyHostToDevice));
    TRYB(cudaMemcpy(B->d_p, p_flat, sizeof(int32_t) * off, cudaMemcpyHostToDevice));
    TRYB(cudaMalloc(&B->d_item, sizeof(int) * 2 * (size_t)items));
    TRYB(cudaMemcpy(B->d_item, B->item_inst.data(), sizeof(int) * items, cudaMemcpyHostToDevice));
    TRYB(cudaMemcpy(B->d_item + items, item_job.data(), sizeof(int) * items, cudaMemcpyHostToDevice));
    TRYB(cudaMalloc(&B->X.ub, sizeof(int) * count));
    TRYB(cudaMalloc(&B->X.key, sizeof(unsigned long long) * count));
    TRYB(cudaMalloc(&B->X.cnt, sizeof(long long) * 6 * count));
    TRYB(cudaMalloc(&B->X.flags, sizeof(int) * count));
#undef TRYB
    B->X.item_inst = B->d_item;
    B->X.item_job = B->d_item + items;
    B->X.items = items;
    if ((rc = batch_build_classes(B)) != FSP_OK) goto fail;
    if ((rc = batch_capture(B)) != FSP_OK) goto fail;
    *out = B;
    return FSP_OK;
fail:
    batch_free(B);
    return rc;
}

extern "C" int fsp_batch_set_warps(fsp_batch *B, const int32_t *warps)
{
    if (!B) { fsp_set_error("fsp_batch_set_warps: NULL batch"); return FSP_ERR_ARG; }
    std::vector<int> w(B->count, BB / 32);
    if (warps)
        for (int i = 0; i < B->count; ++i) {
            if (warps[i] < 0 || warps[i] > BB_MAX / 32) {
                fsp_set_error("fsp_batch_set_warps: instance %d: %d warps (0 = default, 1..%d)", i, warps[i],
                              BB_MAX / 32);
                return FSP_ERR_ARG;
            }
            w[i] = warps[i] ? warps[i] : BB / 32;
        }
    const int limit = batch_smem_limit(B->optin);
    for (int i = 0; i < B->count; ++i) {
        const size_t need = std::max(batch_smem_nm(B->desc[i].n, B->desc[i].m, false, w[i]),
                                     batch_smem_nm(B->desc[i].n, B->desc[i].m, true, w[i]));
        if ((int)need > limit) {
            fsp_set_error("fsp_batch_set_warps: instance %d (%dx%d) with %d warps needs %zu bytes of shared memory "
                          "(at most %d); nothing changed", i, B->desc[i].n, B->desc[i].m, w[i], need, limit);
            return FSP_ERR_ARG;
        }
    }
    FSP_CUDA(cudaDeviceSynchronize());  // the old scratch may still be in use by a launch
    B->warps = w;
    int rc = batch_build_classes(B);
    if (rc != FSP_OK) return rc;
    return batch_capture(B);
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
    B->split = on != 0;
    return batch_capture(B);
}

extern "C" int fsp_batch_set_test_hold(fsp_batch *B, int on)
{
    if (!B) { fsp_set_error("fsp_batch_set_test_hold: NULL batch"); return FSP_ERR_ARG; }
    B->hold = on != 0;
    return batch_capture(B);
}

extern "C" int fsp_batch_class_stats(fsp_batch *B, fsp_batch_class_info *out, int cap, int *count)
{
    if (!B || !count || (cap > 0 && !out)) { fsp_set_error("fsp_batch_class_stats: NULL argument"); return FSP_ERR_ARG; }
    *count = (int)B->cls.size();
    FSP_CUDA(cudaDeviceSynchronize());
    unsigned long long t0 = ~0ull, t1 = 0;
    std::vector<std::vector<unsigned long long>> ns(B->cls.size());
    for (size_t c = 0; c < B->cls.size(); ++c) {
        const BatchClass &C = B->cls[c];
        ns[c].resize(2 * (size_t)C.grid);
        if (C.grid > 0)
            FSP_CUDA(cudaMemcpy(ns[c].data(), C.ws.cta_ns, ns[c].size() * sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost));
        for (int k = 0; k < C.grid; ++k) {
            t0 = std::min(t0, ns[c][2 * k]);
            t1 = std::max(t1, ns[c][2 * k + 1]);
        }
    }
    for (size_t c = 0; c < B->cls.size() && (int)c < cap; ++c) {
        const BatchClass &C = B->cls[c];
        fsp_batch_class_info &o = out[c];
        o.n = C.n;
        o.m = C.m;
        o.warps = C.warps;
        o.ctas = C.grid;
        o.instances = (int32_t)C.inst.size();
        o.items = B->split ? (int32_t)C.items.size() : (int32_t)C.inst.size();
        int dq[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        FSP_CUDA(cudaMemcpy(dq, C.ws.dq, sizeof dq, cudaMemcpyDeviceToHost));
        o.donated = B->split ? dq[2] : 0;
        double sum = 0.0, lo = 1e300, hi = 0.0, first = 1e300, last = 0.0;
        for (int k = 0; k < C.grid; ++k) {
            const double a = (double)(ns[c][2 * k] - t0) * 1e-6, b = (double)(ns[c][2 * k + 1] - t0) * 1e-6;
            sum += b - a;
            lo = std::min(lo, b - a);
            hi = std::max(hi, b - a);
            first = std::min(first, a);
            last = std::max(last, b);
        }
        o.busy_mean_ms = C.grid > 0 ? sum / C.grid : 0.0;
        o.busy_min_ms = C.grid > 0 ? lo : 0.0;
        o.busy_max_ms = hi;
        o.first_start_ms = C.grid > 0 ? first : 0.0;
        o.last_end_ms = last;
        o.launch_span_ms = t1 > t0 ? (double)(t1 - t0) * 1e-6 : 0.0;
    }
    return FSP_OK;
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

// Block shape per shape on measured throughput: for each shape, up to 8 of
// its instances (with their pools and a node budget each), repeated until
// their split-mode items fill every SM twice over at the smallest block
// shape, run as one split-mode batch with each candidate number of warps per
// CTA that fits; the most nodes bounded per second wins.  Filling the GPU is
// what makes the comparison fair: a smaller CTA bounds an instance more
// slowly but more of them share an SM.
extern "C" int fsp_batch_tune_warps(int count, const int32_t *shapes, const int32_t *p_flat, const int64_t *pools,
                                    int64_t probe_budget, int32_t *warps_out)
{
    if (count < 1 || !shapes || !p_flat || !pools || !warps_out) {
        fsp_set_error("fsp_batch_tune_warps: invalid argument");
        return FSP_ERR_ARG;
    }
    const int cands[] = {4, 8, 12, 16, 20};
    int dev = 0, sms = 1, optin = 0;
    FSP_CUDA(cudaGetDevice(&dev));
    FSP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    FSP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int limit = batch_smem_limit(optin);
    std::vector<long long> off(count + 1, 0);
    for (int i = 0; i < count; ++i) off[i + 1] = off[i] + (long long)shapes[2 * i] * shapes[2 * i + 1];
    std::vector<int> done(count, 0);
    for (int i = 0; i < count; ++i) {
        if (done[i]) continue;
        const int n = shapes[2 * i], m = shapes[2 * i + 1];
        std::vector<int> same;
        for (int j = i; j < count; ++j)
            if (shapes[2 * j] == n && shapes[2 * j + 1] == m) same.push_back(j);
        const int probe = (int)(same.size() < 8 ? same.size() : 8);
        const int need_items = 2 * sms * 4, per_copy = probe * (n > 2 ? n : 1);
        const int reps = (need_items + per_copy - 1) / per_copy;
        std::vector<int32_t> sh, pf;
        std::vector<int64_t> pl, budgets;
        for (int r = 0; r < reps; ++r)
            for (int q = 0; q < probe; ++q) {
                const int j = same[q];
                sh.push_back(n);
                sh.push_back(m);
                pf.insert(pf.end(), p_flat + off[j], p_flat + off[j + 1]);
                pl.push_back(pools[j]);
                budgets.push_back(probe_budget);
            }
        const int pc = probe * reps;
        double best = -1.0;
        int best_w = BB / 32;
        for (int w : cands) {
            const size_t need = std::max(batch_smem_nm(n, m, false, w), batch_smem_nm(n, m, true, w));
            if ((int)need > limit) continue;
            fsp_batch *B = nullptr;
            int rc = fsp_batch_create(pc, sh.data(), pf.data(), pl.data(), budgets.data(), nullptr, &B);
            if (rc != FSP_OK) return rc;
            std::vector<int32_t> ws(pc, w);
            rc = fsp_batch_set_warps(B, ws.data());
            if (rc == FSP_OK) rc = fsp_batch_set_split(B, 1);
            if (rc != FSP_OK) { fsp_batch_destroy(B); return rc; }
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            cudaEventRecord(e0, 0);
            rc = fsp_batch_run(B, 0);
            cudaEventRecord(e1, 0);
            std::vector<fsp_batch_result> r(pc);
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
            if (rate > best) { best = rate; best_w = w; }
        }
        for (int j : same) { warps_out[j] = best_w; done[j] = 1; }
    }
    return FSP_OK;
}
