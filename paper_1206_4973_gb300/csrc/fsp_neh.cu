// fsp_neh.cu -- NEH insertion heuristic on the device, the initial upper
// bound of the larger searches (the paper starts from a given UB; NEH is
// the classic constructive heuristic for the permutation flow shop).
//
// One CTA: the jobs are ranked by decreasing total time (ties: smaller
// index first) with one thread per job; then, job after job, every thread
// evaluates the partial makespan of one insertion position and a 64-bit
// atomicMin on (makespan, position) picks the smallest, earliest on ties.
#include "fsp_common.cuh"

#define NEH_B 256

__global__ void __launch_bounds__(NEH_B) k_neh(const int32_t *__restrict__ p, int n, int m, int32_t *out)
{
    __shared__ int32_t tot[FSP_MAX_JOBS + 1];
    __shared__ uint8_t order[FSP_MAX_JOBS + 1];
    __shared__ uint8_t seq[FSP_MAX_JOBS + 1];
    __shared__ unsigned long long best;
    const int tid = threadIdx.x;
    for (int j = tid; j < n; j += NEH_B) {
        int32_t s = 0;
        for (int k = 0; k < m; ++k) s += p[j * m + k];
        tot[j] = s;
    }
    __syncthreads();
    for (int j = tid; j < n; j += NEH_B) {
        int rank = 0;
        for (int i = 0; i < n; ++i) rank += (tot[i] > tot[j]) || (tot[i] == tot[j] && i < j);
        order[rank] = (uint8_t)j;
    }
    __syncthreads();
    int32_t C[FSP_MAX_MACHINES];
    for (int len = 0; len < n; ++len) {
        const int job = order[len];
        if (tid == 0) best = ~0ull;
        __syncthreads();
        for (int pos = tid; pos <= len; pos += NEH_B) {
            for (int k = 0; k < m; ++k) C[k] = 0;
            for (int i = 0; i <= len; ++i) {
                const int j = i < pos ? seq[i] : (i == pos ? job : seq[i - 1]);
                const int32_t *row = p + j * m;
                C[0] += row[0];
                for (int k = 1; k < m; ++k) C[k] = max(C[k], C[k - 1]) + row[k];
            }
            atomicMin(&best, ((unsigned long long)(uint32_t)C[m - 1] << 32) | (unsigned)pos);
        }
        __syncthreads();
        const int at = (int)(best & 0xffffffffu);
        if (tid == 0) {
            for (int i = len; i > at; --i) seq[i] = seq[i - 1];
            seq[at] = (uint8_t)job;
        }
        __syncthreads();
    }
    if (tid == 0) {
        out[0] = (int32_t)(best >> 32);
        for (int i = 0; i < n; ++i) out[1 + i] = seq[i];
    }
}

extern "C" int fsp_neh(fsp_instance *I, int32_t *cmax, int32_t *perm)
{
    if (!I || !cmax || !perm) { fsp_set_error("fsp_neh: NULL argument"); return FSP_ERR_ARG; }
    int32_t *d_out = nullptr;
    int32_t h[FSP_MAX_JOBS + 1];
    int rc = FSP_OK;
    cudaError_t e = cudaMalloc(&d_out, sizeof(int32_t) * (I->n + 1));
    if (e != cudaSuccess) return fsp_cuda_fail(e, "cudaMalloc(neh)");
    k_neh<<<1, NEH_B>>>(I->d_p, I->n, I->m, d_out);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(h, d_out, sizeof(int32_t) * (I->n + 1), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        rc = fsp_cuda_fail(e, "fsp_neh");
    } else {
        *cmax = h[0];
        for (int i = 0; i < I->n; ++i) perm[i] = h[1 + i];
    }
    cudaFree(d_out);
    return rc;
}
