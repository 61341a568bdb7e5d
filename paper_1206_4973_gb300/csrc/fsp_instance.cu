// fsp_instance.cu -- instance creation and the per-instance tables (K0):
// tails, lags and the Johnson order of every machine pair, computed on the
// device once per instance.  The O(n log n) sort per pair that Sec. V-D
// counts inside each bound is hoisted here: a job's position in the pair's
// order is the number of jobs that precede it under Johnson's rule.
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <unordered_map>
#include <vector>

#include "fsp_common.cuh"

struct FspHostCache {
    std::mutex mu;
    std::vector<cudaEvent_t> events;
    std::vector<void *> pinned;
    long long events_made = 0, pinned_made = 0;  // created by this instance so far
    // reserved at creation for the search that allocates nothing (fsp_solve_noalloc)
    void *rsv_pin = nullptr;
    cudaEvent_t rsv_ev[2] = {nullptr, nullptr};
    std::unordered_map<const void *, size_t> smem;
    struct OccKey {
        const void *k;
        int block;
        size_t smem;
        bool operator==(const OccKey &o) const { return k == o.k && block == o.block && smem == o.smem; }
    };
    struct OccHash {
        size_t operator()(const OccKey &o) const
        {
            return std::hash<const void *>()(o.k) ^ (std::hash<size_t>()(o.smem) * 31u) ^ (size_t)o.block;
        }
    };
    std::unordered_map<OccKey, int, OccHash> occ;
};

int fsp_event_take(fsp_instance *I, cudaEvent_t *ev)
{
    {
        std::lock_guard<std::mutex> g(I->cache->mu);
        if (!I->cache->events.empty()) {
            *ev = I->cache->events.back();
            I->cache->events.pop_back();
            return FSP_OK;
        }
    }
    FSP_CUDA(cudaEventCreate(ev));
    std::lock_guard<std::mutex> g(I->cache->mu);
    ++I->cache->events_made;
    return FSP_OK;
}

void fsp_event_give(fsp_instance *I, cudaEvent_t ev)
{
    if (!ev) return;
    std::lock_guard<std::mutex> g(I->cache->mu);
    I->cache->events.push_back(ev);
}

int fsp_pinned_take(fsp_instance *I, void **p)
{
    {
        std::lock_guard<std::mutex> g(I->cache->mu);
        if (!I->cache->pinned.empty()) {
            *p = I->cache->pinned.back();
            I->cache->pinned.pop_back();
            return FSP_OK;
        }
    }
    FSP_CUDA(cudaMallocHost(p, FSP_PINNED_BYTES));
    std::lock_guard<std::mutex> g(I->cache->mu);
    ++I->cache->pinned_made;
    return FSP_OK;
}

void fsp_noalloc_reserved(fsp_instance *I, void **pin, cudaEvent_t *ev)
{
    *pin = I->cache->rsv_pin;
    ev[0] = I->cache->rsv_ev[0];
    ev[1] = I->cache->rsv_ev[1];
}

extern "C" int fsp_instance_host_objects(const fsp_instance *I, int64_t *pinned_blocks, int64_t *events)
{
    if (!I) { fsp_set_error("fsp_instance_host_objects: inst is NULL"); return FSP_ERR_ARG; }
    std::lock_guard<std::mutex> g(I->cache->mu);
    if (pinned_blocks) *pinned_blocks = I->cache->pinned_made;
    if (events) *events = I->cache->events_made;
    return FSP_OK;
}

const void *fsp_device_view(const void *p, int align)
{
    if (!p || ((uintptr_t)p % (uintptr_t)align) != 0) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    if (a.type == cudaMemoryTypeDevice) return a.device == dev ? p : nullptr;
    if (a.type == cudaMemoryTypeHost && a.devicePointer &&
        ((uintptr_t)a.devicePointer % (uintptr_t)align) == 0)
        return a.devicePointer;
    return nullptr;
}

void fsp_pinned_give(fsp_instance *I, void *p)
{
    if (!p) return;
    std::lock_guard<std::mutex> g(I->cache->mu);
    I->cache->pinned.push_back(p);
}

int fsp_blocks_per_sm(fsp_instance *I, const void *kernel, int block, size_t smem, int *per_sm)
{
    const FspHostCache::OccKey key{kernel, block, smem};
    {
        std::lock_guard<std::mutex> g(I->cache->mu);
        auto it = I->cache->occ.find(key);
        if (it != I->cache->occ.end()) { *per_sm = it->second; return FSP_OK; }
    }
    int n = 0;
    FSP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, block, smem));
    if (n < 1) n = 1;
    std::lock_guard<std::mutex> g(I->cache->mu);
    I->cache->occ[key] = n;
    *per_sm = n;
    return FSP_OK;
}

int fsp_allow_smem(fsp_instance *I, const void *kernel, size_t bytes)
{
    std::lock_guard<std::mutex> g(I->cache->mu);
    auto it = I->cache->smem.find(kernel);
    if (it != I->cache->smem.end() && it->second >= bytes) return FSP_OK;
    FSP_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    I->cache->smem[kernel] = bytes;
    return FSP_OK;
}

static thread_local char g_err[512];

void fsp_set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

int fsp_cuda_fail(cudaError_t e, const char *what)
{
    fsp_set_error("CUDA error %s (%s) in %s", cudaGetErrorName(e), cudaGetErrorString(e), what);
    return e == cudaErrorMemoryAllocation ? FSP_ERR_OOM : FSP_ERR_CUDA;
}

extern "C" const char *fsp_last_error(void) { return g_err; }

extern "C" int fsp_node_stride(int n) { return (n + 1 + 15) / 16 * 16; }

extern "C" int fsp_default_options(fsp_options *opt)
{
    if (!opt) { fsp_set_error("fsp_default_options: opt is NULL"); return FSP_ERR_ARG; }
    memset(opt, 0, sizeof *opt);
    opt->pool_size = 1024;
    return FSP_OK;
}

// Tails q[j][k] = sum over h > k of p[j][h].
__global__ void k_tails(int n, int m, const int32_t *__restrict__ p, int32_t *__restrict__ q)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * m) return;
    const int j = i / m, k = i - j * m;
    int32_t s = 0;
    for (int h = k + 1; h < m; ++h) s += p[j * m + h];
    q[i] = s;
}

// Johnson's rule with lags: does job i (a_i, b_i, lag_i) go before job j?
// Jobs with a <= b first, by increasing a + lag; then the others by
// decreasing b + lag; equal keys by job index.
__device__ __forceinline__ bool johnson_precedes(int i, int32_t ai, int32_t bi, int32_t li, int j,
                                                 int32_t aj, int32_t bj, int32_t lj)
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

// One block per machine pair, one thread per job.
__global__ void k_pair_tables(int n, int m, int P, const int32_t *__restrict__ p, int32_t *__restrict__ lag,
                              uint8_t *__restrict__ order, FspEntry *__restrict__ ent, int2 *__restrict__ we,
                              uint8_t *__restrict__ rank_of)
{
    __shared__ int32_t a_s[FSP_MAX_JOBS + 1], b_s[FSP_MAX_JOBS + 1], l_s[FSP_MAX_JOBS + 1];
    const int kl = blockIdx.x;
    int k = 0, rem = kl;
    while (rem >= m - 1 - k) { rem -= m - 1 - k; ++k; }
    const int l = k + 1 + rem;
    const int j = threadIdx.x;
    if (j < n) {
        int32_t lg = 0;
        for (int h = k + 1; h < l; ++h) lg += p[j * m + h];
        a_s[j] = p[j * m + k];
        b_s[j] = p[j * m + l];
        l_s[j] = lg;
        lag[(size_t)kl * n + j] = lg;
    }
    __syncthreads();
    if (j < n) {
        const int32_t aj = a_s[j], bj = b_s[j], lj = l_s[j];
        int rank = 0;
        for (int i = 0; i < n; ++i)
            rank += (i != j) && johnson_precedes(i, a_s[i], b_s[i], l_s[i], j, aj, bj, lj);
        order[(size_t)kl * n + rank] = (uint8_t)j;
        FspEntry e;
        e.w = aj + lj;
        e.e = aj - bj;
        e.bit = 1u << (j & 31);
        e.widx = j >> 5;
        ent[(size_t)kl * n + rank] = e;
        we[(size_t)rank * P + kl] = make_int2(e.w, e.e);
        rank_of[(size_t)kl * n + j] = (uint8_t)rank;
    }
}

static void free_instance(fsp_instance *I)
{
    if (!I) return;
    cudaFree(I->d_p);
    cudaFree(I->d_q);
    cudaFree(I->d_lag);
    cudaFree(I->d_order);
    cudaFree(I->d_ent);
    cudaFree(I->d_we);
    cudaFree(I->d_rank);
    cudaFree(I->d_status);
    cudaFree(I->d_p16);
    if (I->cache) {
        for (cudaEvent_t ev : I->cache->events) cudaEventDestroy(ev);
        for (void *p : I->cache->pinned) cudaFreeHost(p);
        for (cudaEvent_t ev : I->cache->rsv_ev)
            if (ev) cudaEventDestroy(ev);
        if (I->cache->rsv_pin) cudaFreeHost(I->cache->rsv_pin);
        delete I->cache;
    }
    free(I);
}

extern "C" int fsp_create_instance(int n, int m, const int32_t *p, fsp_instance **out)
{
    if (!out) { fsp_set_error("fsp_create_instance: out is NULL"); return FSP_ERR_ARG; }
    *out = nullptr;
    if (n < 1 || n > FSP_MAX_JOBS || m < 2 || m > FSP_MAX_MACHINES || !p) {
        fsp_set_error("fsp_create_instance: need 1 <= n <= %d, 2 <= m <= %d and p (n=%d, m=%d)",
                      FSP_MAX_JOBS, FSP_MAX_MACHINES, n, m);
        return FSP_ERR_ARG;
    }
    for (long i = 0; i < (long)n * m; ++i)
        if (p[i] < 1 || p[i] > 32767) {
            fsp_set_error("fsp_create_instance: p[%ld] = %d outside 1..32767", i, p[i]);
            return FSP_ERR_ARG;
        }
    fsp_instance *I = (fsp_instance *)calloc(1, sizeof(fsp_instance));
    if (!I) { fsp_set_error("fsp_create_instance: out of host memory"); return FSP_ERR_OOM; }
    I->cache = new FspHostCache();
    I->n = n;
    I->m = m;
    I->P = m * (m - 1) / 2;
    I->stride = fsp_node_stride(n);
    I->mp = (m % 2 == 0) ? m + 1 : m;
    for (long i = 0; i < (long)n * m; ++i) {
        I->total += p[i];
        if (p[i] > I->pmax) I->pmax = p[i];
    }
    int rc = FSP_OK;
    cudaError_t e;
#define TRY(call)                                              \
    do {                                                       \
        e = (call);                                            \
        if (e != cudaSuccess) { rc = fsp_cuda_fail(e, #call); goto fail; } \
    } while (0)
    TRY(cudaGetDevice(&I->device));
    TRY(cudaDeviceGetAttribute(&I->sm_count, cudaDevAttrMultiProcessorCount, I->device));
    TRY(cudaDeviceGetAttribute(&I->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, I->device));
    TRY(cudaMalloc(&I->d_p, sizeof(int32_t) * n * m));
    TRY(cudaMalloc(&I->d_q, sizeof(int32_t) * n * m));
    TRY(cudaMalloc(&I->d_lag, sizeof(int32_t) * (size_t)I->P * n));
    TRY(cudaMalloc(&I->d_order, (size_t)I->P * n));
    TRY(cudaMalloc(&I->d_ent, sizeof(FspEntry) * (size_t)I->P * n));
    TRY(cudaMalloc(&I->d_we, sizeof(int2) * (size_t)I->P * n));
    TRY(cudaMalloc(&I->d_rank, (size_t)I->P * n));
    TRY(cudaMalloc(&I->d_status, sizeof(int)));
    // the read-back block and events of fsp_solve_noalloc, which must not create them
    TRY(cudaMallocHost(&I->cache->rsv_pin, FSP_PINNED_BYTES));
    TRY(cudaEventCreateWithFlags(&I->cache->rsv_ev[0], cudaEventDisableTiming));
    TRY(cudaEventCreateWithFlags(&I->cache->rsv_ev[1], cudaEventDisableTiming));
    I->cache->pinned_made = 1;
    I->cache->events_made = 2;
    TRY(cudaMemcpy(I->d_p, p, sizeof(int32_t) * n * m, cudaMemcpyHostToDevice));
    TRY(cudaMemset(I->d_status, 0, sizeof(int)));
    k_tails<<<(n * m + 255) / 256, 256>>>(n, m, I->d_p, I->d_q);
    TRY(cudaGetLastError());
    k_pair_tables<<<I->P, 256>>>(n, m, I->P, I->d_p, I->d_lag, I->d_order, I->d_ent, I->d_we, I->d_rank);
    TRY(cudaGetLastError());
    if ((rc = pool16_build(I)) != FSP_OK) goto fail;
    TRY(cudaDeviceSynchronize());
#undef TRY
    *out = I;
    return FSP_OK;
fail:
    free_instance(I);
    return rc;
}

extern "C" int fsp_set_bound(fsp_instance *inst, int variant)
{
    if (!inst || (variant != FSP_BOUND_BASE && variant != FSP_BOUND_HEADS)) {
        fsp_set_error("fsp_set_bound: NULL instance or unknown variant %d", variant);
        return FSP_ERR_ARG;
    }
    inst->var = variant;
    return FSP_OK;
}

extern "C" void fsp_destroy_instance(fsp_instance *inst)
{
    if (!inst) return;
    int cur = -1;
    const int dev = inst->device;
    cudaGetDevice(&cur);
    if (cur != dev) cudaSetDevice(dev);
    cudaDeviceSynchronize();
    free_instance(inst);
    if (cur >= 0 && cur != dev) cudaSetDevice(cur);
}

extern "C" int fsp_instance_tables(const fsp_instance *I, int32_t *q, int32_t *lag, uint8_t *order)
{
    if (!I) { fsp_set_error("fsp_instance_tables: inst is NULL"); return FSP_ERR_ARG; }
    if (q) FSP_CUDA(cudaMemcpy(q, I->d_q, sizeof(int32_t) * I->n * I->m, cudaMemcpyDeviceToHost));
    if (lag)
        FSP_CUDA(cudaMemcpy(lag, I->d_lag, sizeof(int32_t) * (size_t)I->P * I->n, cudaMemcpyDeviceToHost));
    if (order) FSP_CUDA(cudaMemcpy(order, I->d_order, (size_t)I->P * I->n, cudaMemcpyDeviceToHost));
    return FSP_OK;
}
