// fsp_mlp.cu -- the learned pair-ordering network (not in the paper): node
// features and labels, a small MLP (F -> H -> H -> P, ReLU) with BF16
// weights and FP32 accumulation on the tensor cores, its backward pass and
// an Adam step, and the top-K pairs per node.
//
// Every matrix product goes through gemm_bf16: a 64 x 64 output tile per CTA
// (4 warps of 32 x 32), K staged 32 at a time in shared memory as bf16, and
// mma.sync.m16n8k16 (bf16 x bf16 -> fp32).  Operands stored as fp32 are
// rounded to bf16 (nearest even) when staged, which is where the oracle
// rounds them too.
#include <cuda_bf16.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "fsp_common.cuh"

typedef __nv_bfloat16 bf16_t;

// ------------------------------------------------------------------ GEMM --

#define G_BM 64
#define G_BN 64
#define G_BK 32
#define G_PAD 8

template <typename T>
__device__ __forceinline__ bf16_t to_bf16(T v);
template <>
__device__ __forceinline__ bf16_t to_bf16<float>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ bf16_t to_bf16<bf16_t>(bf16_t v) { return v; }

// C[i][j] = sum_k A(i,k) B(k,j) over i < M, j < N, k < K, then epi(i, j, c).
// A(i,k) = TA ? A[k*lda + i] : A[i*lda + k];  B(k,j) = TB ? B[j*ldb + k] : B[k*ldb + j].
template <typename TAt, bool TA, typename TBt, bool TB, class Epi>
__global__ void __launch_bounds__(128) k_gemm(const TAt *__restrict__ A, int lda, const TBt *__restrict__ B, int ldb,
                                              int M, int N, int K, Epi epi, const long long *Mdev)
{
    if (Mdev && *Mdev < M) M = (int)*Mdev;  // rows known on the device only
    if ((int)(blockIdx.y * G_BM) >= M) return;
    __shared__ __align__(16) bf16_t As[G_BM][G_BK + G_PAD];
    __shared__ __align__(16) bf16_t Bs[G_BN][G_BK + G_PAD];  // n-major: k contiguous
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int i0 = blockIdx.y * G_BM, j0 = blockIdx.x * G_BN;
    const int wi = (warp >> 1) * 32, wj = (warp & 1) * 32;
    const int g = lane >> 2, t = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
    for (int k0 = 0; k0 < K; k0 += G_BK) {
        for (int e = tid; e < G_BM * G_BK; e += 128) {
            const int r = TA ? (e % G_BM) : (e / G_BK), c = TA ? (e / G_BM) : (e % G_BK);
            const int i = i0 + r, k = k0 + c;
            bf16_t v = __float2bfloat16_rn(0.f);
            if (i < M && k < K) v = to_bf16<TAt>(TA ? A[(size_t)k * lda + i] : A[(size_t)i * lda + k]);
            As[r][c] = v;
        }
        for (int e = tid; e < G_BN * G_BK; e += 128) {
            const int nn = TB ? (e / G_BK) : (e % G_BN), c = TB ? (e % G_BK) : (e / G_BN);
            const int j = j0 + nn, k = k0 + c;
            bf16_t v = __float2bfloat16_rn(0.f);
            if (j < N && k < K) v = to_bf16<TBt>(TB ? B[(size_t)j * ldb + k] : B[(size_t)k * ldb + j]);
            Bs[nn][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < G_BK; kk += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const int r = wi + a * 16 + g;
                af[a][0] = *reinterpret_cast<const uint32_t *>(&As[r][kk + 2 * t]);
                af[a][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + 2 * t]);
                af[a][2] = *reinterpret_cast<const uint32_t *>(&As[r][kk + 8 + 2 * t]);
                af[a][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + 8 + 2 * t]);
            }
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int nn = wj + b * 8 + g;
                bfr[b][0] = *reinterpret_cast<const uint32_t *>(&Bs[nn][kk + 2 * t]);
                bfr[b][1] = *reinterpret_cast<const uint32_t *>(&Bs[nn][kk + 8 + 2 * t]);
            }
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                        "{%8,%9}, {%0,%1,%2,%3};\n"
                        : "+f"(acc[a][b][0]), "+f"(acc[a][b][1]), "+f"(acc[a][b][2]), "+f"(acc[a][b][3])
                        : "r"(af[a][0]), "r"(af[a][1]), "r"(af[a][2]), "r"(af[a][3]), "r"(bfr[b][0]),
                          "r"(bfr[b][1]));
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int i = i0 + wi + a * 16 + g + (c >= 2 ? 8 : 0);
                const int j = j0 + wj + b * 8 + 2 * t + (c & 1);
                if (i < M && j < N) epi(i, j, acc[a][b][c]);
            }
}

// Epilogues.
struct EpiBiasReluBf16 {  // out = bf16(relu(v + bias[j]))
    const float *bias;
    bf16_t *out;
    int ld;
    __device__ void operator()(int i, int j, float v) const
    {
        out[(size_t)i * ld + j] = __float2bfloat16_rn(fmaxf(v + bias[j], 0.f));
    }
};
struct EpiBiasF32 {  // out = v + bias[j]
    const float *bias;
    float *out;
    int ld;
    __device__ void operator()(int i, int j, float v) const { out[(size_t)i * ld + j] = v + bias[j]; }
};
struct EpiStoreF32 {  // out = v
    float *out;
    int ld;
    __device__ void operator()(int i, int j, float v) const { out[(size_t)i * ld + j] = v; }
};
struct EpiReluMaskF32 {  // out = v where the stored activation h > 0, else 0
    const bf16_t *h;
    float *out;
    int ld;
    __device__ void operator()(int i, int j, float v) const
    {
        out[(size_t)i * ld + j] = __bfloat162float(h[(size_t)i * ld + j]) > 0.f ? v : 0.f;
    }
};

template <typename TAt, bool TA, typename TBt, bool TB, class Epi>
static cudaError_t gemm(const TAt *A, int lda, const TBt *B, int ldb, int M, int N, int K, Epi epi, cudaStream_t st,
                        const long long *Mdev = nullptr)
{
    dim3 grid((N + G_BN - 1) / G_BN, (M + G_BM - 1) / G_BM);
    k_gemm<TAt, TA, TBt, TB, Epi><<<grid, 128, 0, st>>>(A, lda, B, ldb, M, N, K, epi, Mdev);
    return cudaGetLastError();
}

// ------------------------------------------------------------ the network --

struct fsp_mlp {
    int F, H, P;
    int device;
    int64_t np;                // number of parameters
    int64_t oW1, ob1, oW2, ob2, oW3, ob3;  // offsets in the flat fp32 arrays
    float *w, *g, *m1, *m2;    // master weights, gradients, Adam moments (device)
    bf16_t *wb;                // bf16 weights W1 | W2 | W3 (device)
    bf16_t *wt;                // transposed bf16 weights W1^T | W2^T | W3^T (n-major, k contiguous)
    bf16_t *w1p;               // W1^T zero-padded to [H][48] rows (16-byte copies), when F <= 48
    int64_t step;
    int64_t cap;               // rows the activation buffers hold
    bf16_t *h1, *h2;           // [cap][H]
    float *L, *dL, *dz2, *dz1; // [cap][P], [cap][P], [cap][H], [cap][H]
    float *loss;               // [1] device
};

static void mlp_offsets(fsp_mlp *M)
{
    const int64_t F = M->F, H = M->H, P = M->P;
    M->oW1 = 0;
    M->ob1 = M->oW1 + F * H;
    M->oW2 = M->ob1 + H;
    M->ob2 = M->oW2 + H * H;
    M->oW3 = M->ob2 + H;
    M->ob3 = M->oW3 + H * P;
    M->np = M->ob3 + P;
}

__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Glorot-uniform weights from a counter-based hash of (seed, index); zero biases.
__global__ void k_mlp_init(float *w, int64_t np, int64_t oW1, int64_t ob1, int64_t oW2, int64_t ob2, int64_t oW3,
                           int64_t ob3, int F, int H, int P, uint64_t seed)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    float a = 0.f;
    if (i < ob1) a = sqrtf(6.f / (F + H));
    else if (i >= oW2 && i < ob2) a = sqrtf(6.f / (H + H));
    else if (i >= oW3 && i < ob3) a = sqrtf(6.f / (H + P));
    const double u = (double)(mix64(seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1)) >> 11) * (1.0 / 9007199254740992.0);
    w[i] = (float)((2.0 * u - 1.0) * a);
}

// bf16 copies of W1, W2, W3 (packed back to back), row-major and transposed.
__global__ void k_mlp_to_bf16(const float *w, bf16_t *wb, bf16_t *wt, bf16_t *w1p, int64_t oW1, int64_t nW1,
                              int64_t oW2, int64_t nW2, int64_t oW3, int64_t nW3, int F, int H, int P)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t o, base;
    int rows, cols;  // the matrix is rows x cols, row-major
    if (i < nW1) { o = oW1; base = 0; rows = F; cols = H; }
    else if (i < nW1 + nW2) { o = oW2; base = nW1; rows = H; cols = H; }
    else if (i < nW1 + nW2 + nW3) { o = oW3; base = nW1 + nW2; rows = H; cols = P; }
    else return;
    const int64_t e = i - base;
    const bf16_t v = __float2bfloat16_rn(w[o + e]);
    wb[i] = v;
    const int r = (int)(e / cols), c = (int)(e - (int64_t)r * cols);
    wt[base + (int64_t)c * rows + r] = v;
    if (w1p && i < nW1) w1p[(int64_t)c * 48 + r] = v;  // padding columns stay zero
}

// Row-wise softmax cross-entropy: loss (summed / B) and dL = (softmax - onehot) / B.
__global__ void k_xent(const float *L, const int32_t *y, int64_t B, int P, float *dL, float *loss)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= B) return;
    const float *l = L + r * P;
    float mx = l[0];
    for (int j = 1; j < P; ++j) mx = fmaxf(mx, l[j]);
    float s = 0.f;
    for (int j = 0; j < P; ++j) s += expf(l[j] - mx);
    const float inv = 1.f / s;
    const int yr = y[r];
    for (int j = 0; j < P; ++j) dL[r * P + j] = (expf(l[j] - mx) * inv - (j == yr ? 1.f : 0.f)) / (float)B;
    atomicAdd(loss, (logf(s) + mx - l[yr]) / (float)B);
}

// Column sums of a [B][N] fp32 matrix into out[N].
__global__ void k_colsum(const float *X, int64_t B, int N, float *out)
{
    const int j = blockIdx.x;
    float s = 0.f;
    for (int64_t r = threadIdx.x; r < B; r += blockDim.x) s += X[r * N + j];
    __shared__ float red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[j] = red[0];
}

__global__ void k_adam(float *w, const float *g, float *m1, float *m2, int64_t np, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    w[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
}

static int mlp_reserve(fsp_mlp *M, int64_t B)
{
    if (B <= M->cap) return FSP_OK;
    cudaFree(M->h1); cudaFree(M->h2); cudaFree(M->L); cudaFree(M->dL); cudaFree(M->dz2); cudaFree(M->dz1);
    M->h1 = M->h2 = nullptr;
    M->L = M->dL = M->dz2 = M->dz1 = nullptr;
    M->cap = 0;
    const size_t H = M->H, P = M->P;
    FSP_CUDA(cudaMalloc(&M->h1, B * H * sizeof(bf16_t)));
    FSP_CUDA(cudaMalloc(&M->h2, B * H * sizeof(bf16_t)));
    FSP_CUDA(cudaMalloc(&M->L, B * P * sizeof(float)));
    FSP_CUDA(cudaMalloc(&M->dL, B * P * sizeof(float)));
    FSP_CUDA(cudaMalloc(&M->dz2, B * H * sizeof(float)));
    FSP_CUDA(cudaMalloc(&M->dz1, B * H * sizeof(float)));
    M->cap = B;
    return FSP_OK;
}

static int mlp_refresh_bf16(fsp_mlp *M, cudaStream_t st)
{
    const int64_t nW1 = (int64_t)M->F * M->H, nW2 = (int64_t)M->H * M->H, nW3 = (int64_t)M->H * M->P;
    const int64_t tot = nW1 + nW2 + nW3;
    k_mlp_to_bf16<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(M->w, M->wb, M->wt, M->w1p, M->oW1, nW1, M->oW2,
                                                                  nW2, M->oW3, nW3, M->F, M->H, M->P);
    FSP_CUDA(cudaGetLastError());
    return FSP_OK;
}

static void mlp_free(fsp_mlp *M)
{
    if (!M) return;
    cudaFree(M->w); cudaFree(M->g); cudaFree(M->m1); cudaFree(M->m2); cudaFree(M->wb); cudaFree(M->wt);
    cudaFree(M->w1p);
    cudaFree(M->h1); cudaFree(M->h2); cudaFree(M->L); cudaFree(M->dL); cudaFree(M->dz2); cudaFree(M->dz1);
    cudaFree(M->loss);
    free(M);
}

extern "C" int fsp_mlp_create(int in_dim, int hidden, int out_dim, uint64_t seed, fsp_mlp **out)
{
    if (!out || in_dim < 1 || hidden < 1 || out_dim < 1 || in_dim > 4096 || hidden > 4096 || out_dim > 4096) {
        fsp_set_error("fsp_mlp_create: invalid dimensions");
        return FSP_ERR_ARG;
    }
    fsp_mlp *M = (fsp_mlp *)calloc(1, sizeof(fsp_mlp));
    if (!M) { fsp_set_error("fsp_mlp_create: out of host memory"); return FSP_ERR_OOM; }
    M->F = in_dim; M->H = hidden; M->P = out_dim;
    mlp_offsets(M);
    int rc = FSP_OK;
    cudaError_t e;
    const size_t nb = (size_t)M->np * sizeof(float);
    const size_t nwb = ((size_t)M->F * M->H + (size_t)M->H * M->H + (size_t)M->H * M->P) * sizeof(bf16_t);
#define TRYM(call) do { e = (call); if (e != cudaSuccess) { rc = fsp_cuda_fail(e, #call); goto fail; } } while (0)
    TRYM(cudaGetDevice(&M->device));
    TRYM(cudaMalloc(&M->w, nb));
    TRYM(cudaMalloc(&M->g, nb));
    TRYM(cudaMalloc(&M->m1, nb));
    TRYM(cudaMalloc(&M->m2, nb));
    TRYM(cudaMalloc(&M->wb, nwb));
    TRYM(cudaMalloc(&M->wt, nwb));
    if (M->F <= 48) {
        TRYM(cudaMalloc(&M->w1p, (size_t)M->H * 48 * sizeof(bf16_t)));
        TRYM(cudaMemset(M->w1p, 0, (size_t)M->H * 48 * sizeof(bf16_t)));
    }
    TRYM(cudaMalloc(&M->loss, sizeof(float)));
    TRYM(cudaMemset(M->m1, 0, nb));
    TRYM(cudaMemset(M->m2, 0, nb));
    TRYM(cudaMemset(M->g, 0, nb));
    k_mlp_init<<<(unsigned)((M->np + 255) / 256), 256>>>(M->w, M->np, M->oW1, M->ob1, M->oW2, M->ob2, M->oW3,
                                                          M->ob3, M->F, M->H, M->P, seed);
    TRYM(cudaGetLastError());
    if ((rc = mlp_refresh_bf16(M, 0)) != FSP_OK) goto fail;
    TRYM(cudaDeviceSynchronize());
#undef TRYM
    *out = M;
    return FSP_OK;
fail:
    mlp_free(M);
    return rc;
}

extern "C" void fsp_mlp_destroy(fsp_mlp *M)
{
    if (!M) return;
    cudaDeviceSynchronize();
    mlp_free(M);
}

extern "C" int64_t fsp_mlp_num_params(const fsp_mlp *M) { return M ? M->np : FSP_ERR_ARG; }

extern "C" int fsp_mlp_get_params(const fsp_mlp *M, float *host)
{
    if (!M || !host) { fsp_set_error("fsp_mlp_get_params: NULL argument"); return FSP_ERR_ARG; }
    FSP_CUDA(cudaMemcpy(host, M->w, (size_t)M->np * sizeof(float), cudaMemcpyDeviceToHost));
    return FSP_OK;
}

extern "C" int fsp_mlp_set_params(fsp_mlp *M, const float *host)
{
    if (!M || !host) { fsp_set_error("fsp_mlp_set_params: NULL argument"); return FSP_ERR_ARG; }
    const size_t nb = (size_t)M->np * sizeof(float);
    FSP_CUDA(cudaMemcpy(M->w, host, nb, cudaMemcpyHostToDevice));
    FSP_CUDA(cudaMemset(M->m1, 0, nb));
    FSP_CUDA(cudaMemset(M->m2, 0, nb));
    M->step = 0;
    int rc = mlp_refresh_bf16(M, 0);
    if (rc != FSP_OK) return rc;
    FSP_CUDA(cudaDeviceSynchronize());
    return FSP_OK;
}

// Forward pass into M->h1, M->h2 and `scores` ([B][P] fp32); Bdev (device,
// may be NULL) caps the rows at a count only the device knows.
static int mlp_forward(fsp_mlp *M, const float *X, int64_t B, float *scores, cudaStream_t st,
                       const long long *Bdev = nullptr)
{
    const bf16_t *W1 = M->wb, *W2 = M->wb + (size_t)M->F * M->H, *W3 = W2 + (size_t)M->H * M->H;
    const int F = M->F, H = M->H, P = M->P;
    const int Bi = (int)B;
    FSP_CUDA((gemm<float, false, bf16_t, false>(X, F, W1, H, Bi, H, F, EpiBiasReluBf16{M->w + M->ob1, M->h1, H}, st, Bdev)));
    FSP_CUDA((gemm<bf16_t, false, bf16_t, false>(M->h1, H, W2, H, Bi, H, H, EpiBiasReluBf16{M->w + M->ob2, M->h2, H}, st, Bdev)));
    FSP_CUDA((gemm<bf16_t, false, bf16_t, false>(M->h2, H, W3, P, Bi, P, H, EpiBiasF32{M->w + M->ob3, scores, P}, st, Bdev)));
    return FSP_OK;
}

int fsp_mlp_dims(const fsp_mlp *M, int *F, int *H, int *P)
{
    if (!M) return FSP_ERR_ARG;
    *F = M->F; *H = M->H; *P = M->P;
    return FSP_OK;
}

// Scores of up to Bmax rows (the first *Bdev of them) for the search.
int fsp_mlp_forward_dev(fsp_mlp *M, const float *X, const long long *Bdev, int64_t Bmax, float *scores,
                        cudaStream_t st)
{
    int rc = mlp_reserve(M, Bmax);
    if (rc != FSP_OK) return rc;
    return mlp_forward(M, X, Bmax, scores, st, Bdev);
}

extern "C" int fsp_mlp_forward(fsp_mlp *M, const float *X, int64_t B, float *scores, void *stream)
{
    if (!M || B < 0 || (B > 0 && (!X || !scores))) { fsp_set_error("fsp_mlp_forward: invalid argument"); return FSP_ERR_ARG; }
    if (B == 0) return FSP_OK;
    if (B > (1LL << 30)) { fsp_set_error("fsp_mlp_forward: batch too large"); return FSP_ERR_ARG; }
    int rc = mlp_reserve(M, B);
    if (rc != FSP_OK) return rc;
    return mlp_forward(M, X, B, scores, (cudaStream_t)stream);
}

// Loss and gradients of the mean cross-entropy into M->g (layout of the parameters).
static int mlp_loss_grad(fsp_mlp *M, const float *X, const int32_t *y, int64_t B, cudaStream_t st)
{
    const int F = M->F, H = M->H, P = M->P, Bi = (int)B;
    const bf16_t *W2 = M->wb + (size_t)F * H, *W3 = W2 + (size_t)H * H;
    int rc = mlp_forward(M, X, B, M->L, st);
    if (rc != FSP_OK) return rc;
    FSP_CUDA(cudaMemsetAsync(M->loss, 0, sizeof(float), st));
    k_xent<<<(unsigned)((B + 127) / 128), 128, 0, st>>>(M->L, y, B, P, M->dL, M->loss);
    FSP_CUDA(cudaGetLastError());
    // layer 3: dW3 = H2^T dL, db3 = colsum dL, dZ2 = (dL W3^T) masked by H2 > 0
    FSP_CUDA((gemm<bf16_t, true, float, false>(M->h2, H, M->dL, P, H, P, Bi, EpiStoreF32{M->g + M->oW3, P}, st)));
    k_colsum<<<P, 256, 0, st>>>(M->dL, B, P, M->g + M->ob3);
    FSP_CUDA((gemm<float, false, bf16_t, true>(M->dL, P, W3, P, Bi, H, P, EpiReluMaskF32{M->h2, M->dz2, H}, st)));
    // layer 2
    FSP_CUDA((gemm<bf16_t, true, float, false>(M->h1, H, M->dz2, H, H, H, Bi, EpiStoreF32{M->g + M->oW2, H}, st)));
    k_colsum<<<H, 256, 0, st>>>(M->dz2, B, H, M->g + M->ob2);
    FSP_CUDA((gemm<float, false, bf16_t, true>(M->dz2, H, W2, H, Bi, H, H, EpiReluMaskF32{M->h1, M->dz1, H}, st)));
    // layer 1
    FSP_CUDA((gemm<float, true, float, false>(X, F, M->dz1, H, F, H, Bi, EpiStoreF32{M->g + M->oW1, H}, st)));
    k_colsum<<<H, 256, 0, st>>>(M->dz1, B, H, M->g + M->ob1);
    FSP_CUDA(cudaGetLastError());
    return FSP_OK;
}

extern "C" int fsp_mlp_loss_grad(fsp_mlp *M, const float *X, const int32_t *labels, int64_t B, float *loss,
                                 float *grad, void *stream)
{
    if (!M || B < 1 || !X || !labels) { fsp_set_error("fsp_mlp_loss_grad: invalid argument"); return FSP_ERR_ARG; }
    if (B > (1LL << 30)) { fsp_set_error("fsp_mlp_loss_grad: batch too large"); return FSP_ERR_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    int rc = mlp_reserve(M, B);
    if (rc != FSP_OK) return rc;
    if ((rc = mlp_loss_grad(M, X, labels, B, st)) != FSP_OK) return rc;
    if (grad) FSP_CUDA(cudaMemcpyAsync(grad, M->g, (size_t)M->np * sizeof(float), cudaMemcpyDefault, st));
    if (loss) {
        FSP_CUDA(cudaMemcpyAsync(loss, M->loss, sizeof(float), cudaMemcpyDeviceToHost, st));
        FSP_CUDA(cudaStreamSynchronize(st));
    }
    return FSP_OK;
}

extern "C" int fsp_mlp_train_step(fsp_mlp *M, const float *X, const int32_t *labels, int64_t B, float lr,
                                  float *loss, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    int rc = fsp_mlp_loss_grad(M, X, labels, B, nullptr, nullptr, stream);
    if (rc != FSP_OK) return rc;
    M->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)M->step), c2 = 1.f - powf(b2, (float)M->step);
    k_adam<<<(unsigned)((M->np + 255) / 256), 256, 0, st>>>(M->w, M->g, M->m1, M->m2, M->np, lr, b1, b2, 1e-8f, c1, c2);
    FSP_CUDA(cudaGetLastError());
    if ((rc = mlp_refresh_bf16(M, st)) != FSP_OK) return rc;
    if (loss) {
        FSP_CUDA(cudaMemcpyAsync(loss, M->loss, sizeof(float), cudaMemcpyDeviceToHost, st));
        FSP_CUDA(cudaStreamSynchronize(st));
    }
    return FSP_OK;
}

// ---------------------------------------------------- features and top-K --

// Features of a node: C_k / T, S_k / T (k < m), d / n, T = total time / m;
// label: first pair (k-major) with the largest two-machine bound.  One
// thread per node; general n and m (this runs on logged nodes, off the
// bounding path).
__global__ void k_node_features(DevInst I, const uint8_t *__restrict__ nodes, long long count, float T,
                                float *__restrict__ x, int32_t *__restrict__ label)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const int n = I.n, m = I.m;
    int32_t C[FSP_MAX_MACHINES], S[FSP_MAX_MACHINES], Q[FSP_MAX_MACHINES];
    uint32_t U[8];
    fsp_features(I, nodes + t * I.stride, T, x + t * (2 * m + 1), U, C, S, Q);
    if (!label) return;
    int best = 0, bestv = 0, kl = 0;
    for (int k = 0; k < m - 1; ++k)
        for (int l = k + 1; l < m; ++l, ++kl) {
            const FspEntry *e = I.ent + (size_t)kl * n;
            int32_t E = 0, M = FSP_NEG;
            for (int pos = 0; pos < n; ++pos) {
                const FspEntry en = e[pos];
                if (U[en.widx] & en.bit) {
                    M = max(M, E + en.w);
                    E += en.e;
                }
            }
            const int32_t ql = Q[l] == 0x7fffffff ? 0 : Q[l];
            const int32_t v = S[l] + ql + max(C[l], C[k] + M);
            if (kl == 0 || v > bestv) { bestv = v; best = kl; }
        }
    if (label) label[t] = best;
}

extern "C" int fsp_node_features(fsp_instance *I, const uint8_t *nodes, int64_t count, float *x, int32_t *label,
                                 void *stream)
{
    if (!I || count < 0 || (count > 0 && (!nodes || !x))) { fsp_set_error("fsp_node_features: invalid argument"); return FSP_ERR_ARG; }
    if (count == 0) return FSP_OK;
    const float T = (float)I->total / (float)I->m;  // float32 total over float32 m, nearest
    k_node_features<<<(unsigned)((count + 127) / 128), 128, 0, (cudaStream_t)stream>>>(dev_view(I), nodes, count, T,
                                                                                       x, label);
    FSP_CUDA(cudaGetLastError());
    return FSP_OK;
}


// ------------------------------------------- fused inference for the search --
// One CTA scores RM parents: their features, the three layers on the tensor
// cores with the (transposed, bf16) weights and the activations in shared
// memory, and the K best pairs of each parent.  Each warp owns 16 rows end
// to end, so layers only need a warp barrier.  H = 128, P <= 192, F <= 48.
#define FM_RM 128  // rows (parents) per CTA round: 8 warps x 16
#define FM_T 256   // threads
#define FM_H 128
#define FM_KP 48   // padded input width
#define FM_NP 192  // padded output width
#define FM_S 8     // row padding (bf16) against bank conflicts
#define FM_TKR 4   // rows whose top-K reductions run together
#define FM_SCS (FM_NP + 2)  // score row stride (bf16): an odd word count, rows in distinct banks

struct FusedSmem {
    size_t w1, w2, w3, act, sc, pq, bytes;
};

static inline FusedSmem fused_layout(const fsp_instance *I)
{
    FusedSmem L;
    size_t o = 0;
    L.w1 = o; o += (size_t)FM_H * (FM_KP + FM_S) * 2;
    L.w2 = o; o += (size_t)FM_H * (FM_H + FM_S) * 2;
    L.w3 = o; o += (size_t)FM_NP * (FM_H + FM_S) * 2;
    L.act = o; o += (size_t)FM_RM * (FM_H + FM_S) * 2;  // X, then H1, then H2 (per warp strip)
    L.sc = o; o += (size_t)FM_RM * FM_SCS * 2;           // scores (bf16) for the top-K
    L.pq = o; o += (size_t)I->n * I->mp * 8;
    L.bytes = o;
    return L;
}


// acc[nt][4] += A(16 x K, rows r0.., stride lda) x Bt(n-major, stride ldb) for NT n-tiles of 8.
template <int NT, int K>
__device__ __forceinline__ void fm_warp_gemm(const bf16_t *A, int lda, const bf16_t *Bt, int ldb, float (&acc)[NT][4],
                                             int g, int t)
{
#pragma unroll
    for (int k0 = 0; k0 < K; k0 += 16) {
        uint32_t a[4];
        a[0] = *reinterpret_cast<const uint32_t *>(A + g * lda + k0 + 2 * t);
        a[1] = *reinterpret_cast<const uint32_t *>(A + (g + 8) * lda + k0 + 2 * t);
        a[2] = *reinterpret_cast<const uint32_t *>(A + g * lda + k0 + 8 + 2 * t);
        a[3] = *reinterpret_cast<const uint32_t *>(A + (g + 8) * lda + k0 + 8 + 2 * t);
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const bf16_t *b = Bt + (nt * 8 + g) * ldb + k0 + 2 * t;
            const uint32_t b0 = *reinterpret_cast<const uint32_t *>(b);
            const uint32_t b1 = *reinterpret_cast<const uint32_t *>(b + 8);
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};\n"
                : "+f"(acc[nt][0]), "+f"(acc[nt][1]), "+f"(acc[nt][2]), "+f"(acc[nt][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
        }
    }
}

__device__ __forceinline__ void fm_cp16(void *dst_smem, const void *src_gmem)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src_gmem));
}

// Half of a node's features as bf16 into xr (the machine count known at
// compile time, p from the shared {p, q} rows of odd stride mp): part 0 the
// release times over T (columns 0..MT-1), the depth over n (2 MT) and the
// zero padding; part 1 the remaining work over T (MT..2 MT-1).  Same values
// as fsp_features.
template <int MT>
__device__ __forceinline__ void fm_features_part(const uint8_t *r, int n, const int2 *pq, int mp, float T, int part,
                                                 bf16_t *xr)
{
    const int d = r[n] <= n ? r[n] : n;
    int32_t A[MT];
#pragma unroll
    for (int k = 0; k < MT; ++k) A[k] = 0;
    if (part == 0) {
        for (int i = 0; i < d; ++i) {
            const int j = r[i] < n ? r[i] : 0;
            const int2 *row = pq + j * mp;
            A[0] += row[0].x;
#pragma unroll
            for (int k = 1; k < MT; ++k) A[k] = max(A[k], A[k - 1]) + row[k].x;
        }
#pragma unroll
        for (int k = 0; k < MT; ++k) xr[k] = __float2bfloat16_rn(__fdiv_rn((float)A[k], T));
        xr[2 * MT] = __float2bfloat16_rn(__fdiv_rn((float)d, (float)n));
        for (int k = 2 * MT + 1; k < FM_KP; ++k) xr[k] = __float2bfloat16_rn(0.f);
    } else {
        for (int i = d; i < n; ++i) {
            const int j = r[i] < n ? r[i] : 0;
            const int2 *row = pq + j * mp;
#pragma unroll
            for (int k = 0; k < MT; ++k) A[k] += row[k].x;
        }
#pragma unroll
        for (int k = 0; k < MT; ++k) xr[MT + k] = __float2bfloat16_rn(__fdiv_rn((float)A[k], T));
    }
}

template <int MT>
__global__ void __launch_bounds__(FM_T) k_mlp_topk_parents(DevInst I, const uint8_t *__restrict__ stack,
                                                           const long long *__restrict__ s_pop,
                                                           const long long *__restrict__ n_parents, float T,
                                                           const bf16_t *__restrict__ wt, const bf16_t *__restrict__ w1p,
                                                           const float *__restrict__ w, int64_t ob1, int64_t ob2,
                                                           int64_t ob3, int F, int P, int K,
                                                           int16_t *__restrict__ topk, FusedSmem L, int reversed)
{
    const long long np = *n_parents;
    if ((long long)blockIdx.x * FM_RM >= np) return;
    extern __shared__ __align__(16) unsigned char smem[];
    bf16_t *w1s = reinterpret_cast<bf16_t *>(smem + L.w1);
    bf16_t *w2s = reinterpret_cast<bf16_t *>(smem + L.w2);
    bf16_t *w3s = reinterpret_cast<bf16_t *>(smem + L.w3);
    bf16_t *act = reinterpret_cast<bf16_t *>(smem + L.act);
    int2 *pq = reinterpret_cast<int2 *>(smem + L.pq);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, g = lane >> 2, t = lane & 3;
    // weights, once per CTA, as 16-byte asynchronous copies
    const bf16_t *g2 = wt + (size_t)F * FM_H, *g3 = g2 + (size_t)FM_H * FM_H;
    for (int e = tid; e < FM_H * (FM_KP / 8); e += FM_T) {
        const int nn = e / (FM_KP / 8), q = e - nn * (FM_KP / 8);
        fm_cp16(w1s + nn * (FM_KP + FM_S) + q * 8, w1p + (size_t)nn * FM_KP + q * 8);
    }
    for (int e = tid; e < FM_H * 16; e += FM_T) {
        const int nn = e >> 4, q = e & 15;
        fm_cp16(w2s + nn * (FM_H + FM_S) + q * 8, g2 + (size_t)nn * FM_H + q * 8);
    }
    for (int e = tid; e < FM_NP * 16; e += FM_T) {
        const int nn = e >> 4, q = e & 15;
        if (nn < P) fm_cp16(w3s + nn * (FM_H + FM_S) + q * 8, g3 + (size_t)nn * FM_H + q * 8);
        else *reinterpret_cast<uint4 *>(w3s + nn * (FM_H + FM_S) + q * 8) = make_uint4(0u, 0u, 0u, 0u);
    }
    asm volatile("cp.async.commit_group;\n" ::);
    for (int i = tid; i < I.n * MT; i += FM_T) {
        const int j = i / MT, k = i - j * MT;
        pq[j * I.mp + k] = make_int2(__ldg(I.p + i), __ldg(I.q + i));
    }
    asm volatile("cp.async.wait_all;\n" ::);
    const long long S = *s_pop + np;
    const int rw = warp * 16;                        // the warp's rows
    bf16_t *strip = act + rw * (FM_H + FM_S);        // X (stride FM_KP + FM_S), then H1, H2 (stride FM_H + FM_S)
    for (long long r0 = (long long)blockIdx.x * FM_RM; r0 < np; r0 += (long long)gridDim.x * FM_RM) {
        __syncthreads();  // weights staged / previous rows done
        {   // features: row tid % FM_RM (warp row/16's strip, row row%16); the first
            // half of the threads writes the release-time columns and the depth,
            // the second half the remaining-work columns
            const int row = tid % FM_RM, part = tid / FM_RM;
            const long long r = r0 + row;
            bf16_t *xr = act + (row >> 4) * 16 * (FM_H + FM_S) + (row & 15) * (FM_KP + FM_S);
            if (r < np) {
                const long long at = reversed ? S - 1 - r : r;  // the search's parents sit top down
                fm_features_part<MT>(stack + at * I.stride, I.n, pq, I.mp, T, part, xr);
            } else {
                for (int k = part; k < FM_KP; k += 2) xr[k] = __float2bfloat16_rn(0.f);
            }
        }
        __syncthreads();
        {   // layer 1: X (16 x 48) -> H1 (16 x 128), written over the strip once X is consumed
            float acc[16][4];
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
            fm_warp_gemm<16, FM_KP>(strip, FM_KP + FM_S, w1s, FM_KP + FM_S, acc, g, t);
            __syncwarp();
#pragma unroll
            for (int nt = 0; nt < 16; ++nt)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int row = g + (c >= 2 ? 8 : 0), col = nt * 8 + 2 * t + (c & 1);
                    strip[row * (FM_H + FM_S) + col] = __float2bfloat16_rn(fmaxf(acc[nt][c] + w[ob1 + col], 0.f));
                }
        }
        __syncwarp();
        {   // layer 2: H1 -> H2 in place
            float acc[16][4];
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
            fm_warp_gemm<16, FM_H>(strip, FM_H + FM_S, w2s, FM_H + FM_S, acc, g, t);
            __syncwarp();
#pragma unroll
            for (int nt = 0; nt < 16; ++nt)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int row = g + (c >= 2 ? 8 : 0), col = nt * 8 + 2 * t + (c & 1);
                    strip[row * (FM_H + FM_S) + col] = __float2bfloat16_rn(fmaxf(acc[nt][c] + w[ob2 + col], 0.f));
                }
        }
        __syncwarp();
        // layer 3 in two halves of 96 columns, scores to shared memory (bf16: the
        // order is a heuristic, the search stays exact whatever it is)
        bf16_t *sc = reinterpret_cast<bf16_t *>(smem + L.sc) + rw * FM_SCS;
        for (int half = 0; half < 2; ++half) {
            float acc[12][4];
#pragma unroll
            for (int i = 0; i < 12; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
            fm_warp_gemm<12, FM_H>(strip, FM_H + FM_S, w3s + half * 96 * (FM_H + FM_S), FM_H + FM_S, acc, g, t);
#pragma unroll
            for (int nt = 0; nt < 12; ++nt)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int row = g + (c >= 2 ? 8 : 0), col = half * 96 + nt * 8 + 2 * t + (c & 1);
                    sc[row * FM_SCS + col] = __float2bfloat16_rn(col < P ? acc[nt][c] + w[ob3 + col] : -INFINITY);
                }
        }
        __syncwarp();
        // top-K of each of the warp's 16 rows across the warp: best first, ties to
        // the lower pair; FM_TKR rows at a time so their reduction chains overlap
#pragma unroll 1
        for (int rr = 0; rr < 16; rr += FM_TKR) {
            float v6[FM_TKR][FM_NP / 32];
            uint32_t taken[FM_TKR];
#pragma unroll
            for (int u = 0; u < FM_TKR; ++u) {
                const bf16_t *sr = sc + (rr + u) * FM_SCS;
                taken[u] = 0u;
#pragma unroll
                for (int q = 0; q < FM_NP / 32; ++q)
                    v6[u][q] = lane + 32 * q < P ? __bfloat162float(sr[lane + 32 * q]) : -INFINITY;
            }
#pragma unroll 1
            for (int j = 0; j < K; ++j) {
                float bv[FM_TKR];
                int bq[FM_TKR];
#pragma unroll
                for (int u = 0; u < FM_TKR; ++u) {
                    bv[u] = -INFINITY;
                    bq[u] = 0x7fffffff;
#pragma unroll
                    for (int q = 0; q < FM_NP / 32; ++q) {
                        const int pq2 = lane + 32 * q;
                        if (pq2 < P && !(taken[u] & (1u << q)) && (v6[u][q] > bv[u] || (v6[u][q] == bv[u] && pq2 < bq[u]))) {
                            bv[u] = v6[u][q];
                            bq[u] = pq2;
                        }
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                    for (int u = 0; u < FM_TKR; ++u) {
                        const float ov = __shfl_xor_sync(0xffffffffu, bv[u], o);
                        const int oq = __shfl_xor_sync(0xffffffffu, bq[u], o);
                        if (ov > bv[u] || (ov == bv[u] && oq < bq[u])) { bv[u] = ov; bq[u] = oq; }
                    }
                }
#pragma unroll
                for (int u = 0; u < FM_TKR; ++u) {
                    const long long r = r0 + rw + rr + u;
                    int q = bq[u] == 0x7fffffff ? 0 : bq[u];
                    if ((q & 31) == lane) taken[u] |= 1u << (q >> 5);
                    if (lane == 0 && r < np) topk[r * K + j] = (int16_t)q;
                }
            }
        }
    }
}

// Scores and top-K pairs of the search's parents with the fused kernel
// (H = 128, P <= 192, F <= 48); returns FSP_ERR_ARG for other shapes.
static int mlp_topk(fsp_mlp *M, const fsp_instance *I, const uint8_t *stack, const long long *s_pop,
                    const long long *n_parents, long long max_parents, int K, int16_t *topk, cudaStream_t st,
                    int reversed)
{
    if (M->H != FM_H || M->P > FM_NP || M->F > FM_KP || !M->w1p) return FSP_ERR_ARG;
    typedef void (*Fn)(DevInst, const uint8_t *, const long long *, const long long *, float, const bf16_t *,
                       const bf16_t *, const float *, int64_t, int64_t, int64_t, int, int, int, int16_t *, FusedSmem,
                       int);
    Fn fn = I->m == 5 ? (Fn)k_mlp_topk_parents<5> : I->m == 10 ? (Fn)k_mlp_topk_parents<10>
          : I->m == 20 ? (Fn)k_mlp_topk_parents<20> : nullptr;
    if (!fn) return FSP_ERR_ARG;
    const FusedSmem L = fused_layout(I);
    if ((int)L.bytes > I->smem_optin) return FSP_ERR_ARG;
    FSP_CUDA(cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.bytes));
    const float T = (float)I->total / (float)I->m;
    unsigned grid = (unsigned)((max_parents + FM_RM - 1) / FM_RM);
    if (grid > (unsigned)I->sm_count) grid = (unsigned)I->sm_count;  // persistent: weights staged once per CTA
    fn<<<grid, FM_T, L.bytes, st>>>(dev_view(I), stack, s_pop, n_parents, T, M->wt, M->w1p, M->w, M->ob1, M->ob2,
                                    M->ob3, M->F, M->P, K, topk, L, reversed);
    FSP_CUDA(cudaGetLastError());
    return FSP_OK;
}

int fsp_mlp_topk_parents(fsp_mlp *M, const fsp_instance *I, const uint8_t *stack, const long long *s_pop,
                         const long long *n_parents, long long max_parents, int K, int16_t *topk, cudaStream_t st)
{
    return mlp_topk(M, I, stack, s_pop, n_parents, max_parents, K, topk, st, 1);
}

extern "C" int fsp_pair_order(fsp_instance *I, fsp_mlp *M, const uint8_t *nodes, int64_t count, int k,
                              int16_t *topk, void *stream)
{
    if (!I || !M || count < 0 || k < 1 || k > 8 || (count > 0 && (!nodes || !topk))) {
        fsp_set_error("fsp_pair_order: invalid argument");
        return FSP_ERR_ARG;
    }
    if (M->F != 2 * I->m + 1 || M->P != I->P) {
        fsp_set_error("fsp_pair_order: the network does not match the instance");
        return FSP_ERR_ARG;
    }
    if (M->H != FM_H || (I->m != 5 && I->m != 10 && I->m != 20)) {
        fsp_set_error("fsp_pair_order: needs 128 hidden units and m in {5, 10, 20}");
        return FSP_ERR_ARG;
    }
    if (count == 0) return FSP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    long long *d = nullptr;  // {0, count}: the records play the stack with nothing below them
    const long long h[2] = {0, count};
    FSP_CUDA(cudaMalloc(&d, sizeof h));
    cudaError_t e = cudaMemcpyAsync(d, h, sizeof h, cudaMemcpyHostToDevice, st);
    int rc = e == cudaSuccess ? mlp_topk(M, I, nodes, d, d + 1, count, k, topk, st, 0) : fsp_cuda_fail(e, "fsp_pair_order");
    if (rc == FSP_OK) {
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = fsp_cuda_fail(e, "fsp_pair_order");
    }
    cudaFree(d);
    return rc;
}
