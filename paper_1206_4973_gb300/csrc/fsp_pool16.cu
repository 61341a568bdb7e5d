// fsp_pool16.cu -- parallel bounding of a pool of arbitrary node records
// (the paper's Type 1 model, Sec. III: one bound per subproblem) with two
// nodes per 32-bit register.
//
// The two-machine term of pair (k,l) over the remaining set U in the pair's
// Johnson order (Sec. V-D bound, as read in fsp.h) is
//     M = max_{i in U} (E_{<i} + w_i),  w = a + lag, e = a - b, E_{<i} = sum of e
// over the members before i.  Read from the back of the order it is one
// add-max per member:  G <- max(G + e_i, w_i),  M = G after the first member.
// Every quantity of the bound is the length of a path through the n x m grid
// of processing times (C_k, S_l + qmin_l, M + S_l, the bound itself), so it is
// at most (n + m - 1) * pmax; when (n + m) * pmax <= 16383 every value and
// every intermediate sum fits a signed 16-bit lane and the packed instructions
// add.s16x2 / max.s16x2 evaluate two nodes at once, exactly.
//
// The node bound is LB1 + max(0, max_{k<l} (C_k - LB1 + SQ_l + M_kl)) with
// SQ = S + qmin: the pair value SQ_l + max(C_l, C_k + M) never falls below
// its C_l + SQ_l <= LB1 part, so only the C_k + M branch can raise the bound.
//
// Work split: one warp bounds 32 nodes at a time.  Lane v first computes node
// v's release times, remaining sums, smallest tails and LB1 (one thread per
// node), and writes into the warp's tables, in 16-bit half v of each row,
//   - row j < n:       0xFFFF if job j is in node v's remaining set, else 0,
//   - row n + k:       C_k - LB1,
//   - row n + MT + l:  SQ_l.
// Then the lanes own machine pairs (32 at a time; 190 pairs = 6 passes at m =
// 20) and scan their pair's Johnson order for all 16 node pairs: per position
// one broadcast-free read of the entry {w,w | e,e} and of the job's table row
// (a row stride of 17 words makes the 32 lanes' rows fall in distinct banks),
// then per node pair one add-max and one select that keeps G where the job is
// not in the remaining set.  A butterfly over the lanes leaves lane v with
// node v's maximum, and lane v writes its bound.
#include "fsp_bound.cuh"

#define P16_TS 17           // words per table row: 16 node pairs + 1 (odd: distinct banks)
#define P16_MAX_WARPS 16
#define P16_NEG 0xC000C000u  // -16384 in both halves: "no member yet"
#define P16_QMAX 0x7FFF7FFFu // "no remaining job" for the smallest tails

// The instance image every CTA copies into shared memory (built once per
// instance by k_pool16_image, in this order, each part 16-byte aligned):
//   rows [n][RS] words: p[j][k] (k < MT), then the pairs {p[j][2h], p[j][2h+1]}
//        and the pairs {q[j][2h], q[j][2h+1]} as 16-bit halves (h < H = ceil(MT/2));
//        RS = MT + 2H rounded up to odd, so lanes reading different jobs' rows
//        hit different banks;
//   ej   [n][P] {w | e << 16, byte offset of the job's table row}: position-major;
//   klm  [P] k | l << 8.
template <int MT>
struct P16Dims {
    static constexpr int H = (MT + 1) / 2;
    static constexpr int RS = (MT + 2 * H) | 1;
};

// Two signed 16-bit lanes: max(a + b, c) per lane (the add wraps; the
// callers keep every sum inside the 16-bit range).
__device__ __forceinline__ uint32_t p16_addmax(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t r;
    asm("{.reg .b32 t;\n\tadd.s16x2 t, %1, %2;\n\tmax.s16x2 %0, t, %3;\n\t}" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}

__device__ __forceinline__ uint32_t p16_add(uint32_t a, uint32_t b)
{
    uint32_t r;
    asm("add.s16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

__device__ __forceinline__ uint32_t p16_max(uint32_t a, uint32_t b)
{
    uint32_t r;
    asm("max.s16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

__device__ __forceinline__ uint32_t p16_min(uint32_t a, uint32_t b)
{
    uint32_t r;
    asm("min.s16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

__device__ __forceinline__ int p16_rs_dev(int m)
{
    const int H = (m + 1) / 2;
    return (m + 2 * H) | 1;
}

struct Pool16Smem {
    size_t rows_off, ej_off, klm_off, img_bytes, tab_off, tab_bytes, red_off, bytes;
    int warps, slices;
};

static inline int p16_rs(int m)
{
    const int H = (m + 1) / 2;
    return (m + 2 * H) | 1;
}

static inline Pool16Smem pool16_layout(const fsp_instance *I, int warps, int slices = 1)
{
    Pool16Smem L;
    size_t o = 0;
    L.rows_off = o; o += fsp_align16((size_t)I->n * p16_rs(I->m) * 4);
    L.ej_off = o; o += fsp_align16((size_t)I->n * I->P * 8);
    L.klm_off = o; o += fsp_align16((size_t)I->P * 2);
    L.img_bytes = o;
    L.tab_off = o;
    L.tab_bytes = fsp_align16((size_t)(I->n + 2 * I->m) * P16_TS * 4);
    o += L.tab_bytes * warps;
    L.red_off = o;
    if (slices > 1) o += (size_t)warps * 32 * 4;
    L.bytes = o;
    L.warps = warps;
    L.slices = slices;
    return L;
}

// Build the image (one thread per word of it).
__global__ void k_pool16_image(int n, int m, int P, const int32_t *__restrict__ p, const int32_t *__restrict__ q,
                               const int2 *__restrict__ we, const uint8_t *__restrict__ order, Pool16Smem L,
                               uint8_t *__restrict__ img)
{
    const int H = (m + 1) / 2, RS = p16_rs_dev(m);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n * RS) {
        const int j = i / RS, c = i - j * RS;
        uint32_t v = 0;
        if (c < m) {
            v = (uint32_t)p[j * m + c];
        } else if (c < m + H) {
            const int k = 2 * (c - m);
            v = (uint32_t)p[j * m + k] | (k + 1 < m ? (uint32_t)p[j * m + k + 1] << 16 : 0u);
        } else if (c < m + 2 * H) {
            const int k = 2 * (c - m - H);
            v = (uint32_t)q[j * m + k] | (k + 1 < m ? (uint32_t)q[j * m + k + 1] << 16 : 0u);
        }
        reinterpret_cast<uint32_t *>(img + L.rows_off)[i] = v;
    }
    if (i < n * P) {
        const int pos = i / P, kl = i - pos * P;
        const int2 x = we[i];
        reinterpret_cast<uint2 *>(img + L.ej_off)[i] =
            make_uint2(((uint32_t)x.x & 0xFFFFu) | ((uint32_t)x.y << 16), (uint32_t)order[kl * n + pos] * (P16_TS * 4));
    }
    if (i < P) {
        int k = 0, rem = i;
        while (rem >= m - 1 - k) { rem -= m - 1 - k; ++k; }
        reinterpret_cast<uint16_t *>(img + L.klm_off)[i] = (uint16_t)(k | ((k + 1 + rem) << 8));
    }
}

// a1-a3 of one node from the image rows: release times (32-bit chain over
// the prefix), remaining sums, smallest tails and, for the heads variant,
// smallest processing times as 16-bit machine pairs; the remaining set Um
// and the validity of the record, as fsp_prologue.
template <int MT, int NV, bool BIDIR>
__device__ __forceinline__ void p16_prologue(const FspRec<NV> &r, int d, int d2, int n,
                                             const uint32_t *__restrict__ rows, uint32_t &Um, int32_t (&C)[MT],
                                             int32_t (&SQ)[MT], int32_t &lb1, bool &bad, int var)
{
    constexpr int H = P16Dims<MT>::H, RS = P16Dims<MT>::RS;
    if (!BIDIR) d2 = 0;
    bad = d + d2 > n;
    const int mid_end = n - d2;  // positions [d, mid_end) hold the remaining set
    const bool heads = !BIDIR && var == FSP_BOUND_HEADS;
    uint32_t Am = 0u, S2[H], Q2[H], Pm2[H];
    Um = 0u;
#pragma unroll
    for (int k = 0; k < MT; ++k) C[k] = 0;
#pragma unroll
    for (int h = 0; h < H; ++h) { S2[h] = 0u; Q2[h] = P16_QMAX; Pm2[h] = P16_QMAX; }
    // word by word (the record stays in registers: no byte of it is indexed
    // at run time); positions past n are skipped
    uint32_t rw[4 * NV];
#pragma unroll
    for (int q = 0; q < 4 * NV; ++q) rw[q] = r.w[q];
#pragma unroll 1
    for (int wq = 0; wq < 4 * NV; ++wq) {
        const uint32_t wd = rw[0];
#pragma unroll
        for (int q = 0; q + 1 < 4 * NV; ++q) rw[q] = rw[q + 1];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = 4 * wq + b;
            if (i < n) {
                uint32_t j = (wd >> (8 * b)) & 0xFFu;
                if (j >= (uint32_t)n) { bad = true; j = 0; }
                const uint32_t bit = 1u << j;
                if (Am & bit) bad = true;
                Am |= bit;
                const uint32_t *row = rows + j * RS;
                if (i < d) {
                    C[0] += (int32_t)row[0];
#pragma unroll
                    for (int k = 1; k < MT; ++k) C[k] = max(C[k], C[k - 1]) + (int32_t)row[k];
                } else if (BIDIR && i >= mid_end) {
                    // suffix job: its delivery times follow in a second pass
                } else {
                    Um |= bit;
#pragma unroll
                    for (int h = 0; h < H; ++h) {
                        S2[h] = p16_add(S2[h], row[MT + h]);
                        Q2[h] = p16_min(Q2[h], row[MT + H + h]);
                    }
                    if (heads) {
#pragma unroll
                        for (int h = 0; h < H; ++h) Pm2[h] = p16_min(Pm2[h], row[MT + h]);
                    }
                }
            }
        }
    }
    if (heads && d < n && !bad) {  // R_k = max(C_k, R_{k-1} + min over U of p[j][k-1])
#pragma unroll
        for (int k = 1; k < MT; ++k) {
            const int32_t pm = (int32_t)((Pm2[(k - 1) >> 1] >> (((k - 1) & 1) * 16)) & 0xFFFFu);
            C[k] = max(C[k], C[k - 1] + pm);
        }
    }
    // bidirectional nodes: delivery times of the suffix, its jobs from the
    // last back (words from the top, rotated the other way), machines from
    // m-1 down: D_k = max(D_k, D_{k+1}) + p
    int32_t D[MT];
#pragma unroll
    for (int k = 0; k < MT; ++k) D[k] = 0;
    if (BIDIR && d2 > 0) {
        uint32_t rw[4 * NV];
#pragma unroll
        for (int q = 0; q < 4 * NV; ++q) rw[q] = r.w[q];
#pragma unroll 1
        for (int wq = 4 * NV - 1; wq >= 0; --wq) {
            const uint32_t wd = rw[4 * NV - 1];
#pragma unroll
            for (int q = 4 * NV - 1; q > 0; --q) rw[q] = rw[q - 1];
#pragma unroll
            for (int b = 3; b >= 0; --b) {
                const int i = 4 * wq + b;
                if (i < n && i >= mid_end) {
                    uint32_t j = (wd >> (8 * b)) & 0xFFu;
                    if (j >= (uint32_t)n) j = 0;
                    const uint32_t *row = rows + j * RS;
                    D[MT - 1] += (int32_t)row[MT - 1];
#pragma unroll
                    for (int k = MT - 2; k >= 0; --k) D[k] = max(D[k], D[k + 1]) + (int32_t)row[k];
                }
            }
        }
    }
    lb1 = 0;
#pragma unroll
    for (int k = 0; k < MT; ++k) {
        const int32_t sk = (int32_t)((S2[k >> 1] >> ((k & 1) * 16)) & 0xFFFFu);
        const int32_t qk = (int32_t)((Q2[k >> 1] >> ((k & 1) * 16)) & 0xFFFFu);
        const int32_t qm = qk == 0x7FFF ? 0 : qk;
        SQ[k] = sk + (BIDIR ? max(D[k], qm) : qm);  // the tail after machine k
        lb1 = max(lb1, C[k] + SQ[k]);
    }
}

// S > 1 (small pools, which leave SMs idle at one warp per 32 nodes): a team
// of S consecutive warps takes each group of 32 nodes, every warp computes the
// group's tables itself and scans NPASS / S of the passes over the pairs, and
// the team combines its maxima through shared memory (a named barrier per
// team; S divides NPASS and the warps per CTA).
template <int MT, int NV, bool BIDIR>
__global__ void __launch_bounds__(P16_MAX_WARPS * 32, 1) k_bound_pool16(DevInst I, const uint8_t *__restrict__ img,
                                                                      const uint8_t *__restrict__ nodes,
                                                                      long long count, const long long *dcount,
                                                                      int stride, int32_t *__restrict__ lb_out,
                                                                      Pool16Smem L)
{
    if (dcount) count = *dcount;  // a pool whose size only the device knows (the search's children)
    constexpr int P = MT * (MT - 1) / 2;
    constexpr int NPASS = (P + 31) / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t *rows_s = reinterpret_cast<const uint32_t *>(smem + L.rows_off);
    const uint2 *ej_s = reinterpret_cast<const uint2 *>(smem + L.ej_off);
    const uint16_t *klm_s = reinterpret_cast<const uint16_t *>(smem + L.klm_off);
    const int n = I.n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
    const int S = L.slices, team = warp / S, slice = warp - team * S, TEAMS = W / S;
    const int pass0 = slice * (NPASS / S), pass1 = pass0 + NPASS / S;
    uint32_t *tw = reinterpret_cast<uint32_t *>(smem + L.tab_off + warp * L.tab_bytes);
    uint16_t *th = reinterpret_cast<uint16_t *>(tw);
    int32_t *raise_s = reinterpret_cast<int32_t *>(smem + L.red_off);  // [W][32]: each warp's raises

    // stage the image: 16-byte asynchronous copies, all in flight at once
    for (int c = threadIdx.x; c < (int)(L.img_bytes >> 4); c += blockDim.x) {
        const unsigned dst = (unsigned)__cvta_generic_to_shared(smem + 16 * c);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(img + 16 * c));
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();

    const long long groups = (count + 31) >> 5;
    for (long long g = (long long)blockIdx.x * TEAMS + team; g < groups; g += (long long)gridDim.x * TEAMS) {
        // -- lane v: node g*32 + v, its one-machine quantities into the tables
        const long long node = (g << 5) + lane;
        FspRec<NV> r;
        int d = 0, d2 = 0;
        if (node < count) {
            fsp_load_rec(r, nodes + node * stride);
            d = __ldg(nodes + node * stride + n);  // the depth bytes (same sector: no second fetch)
            if (BIDIR) d2 = __ldg(nodes + node * stride + n + 1);
        } else {
#pragma unroll
            for (int q = 0; q < 4 * NV; ++q) r.w[q] = 0u;
        }
        uint32_t Um;
        int32_t C[MT], SQ[MT], lb1;
        bool bad;
        p16_prologue<MT, NV, BIDIR>(r, d, d2, n, rows_s, Um, C, SQ, lb1, bad, I.var);
        for (int j = 0; j < n; ++j) th[j * (2 * P16_TS) + lane] = ((Um >> j) & 1u) ? 0xFFFFu : 0u;
#pragma unroll
        for (int k = 0; k < MT; ++k) {
            th[(n + k) * (2 * P16_TS) + lane] = (uint16_t)(C[k] - lb1);
            th[(n + MT + k) * (2 * P16_TS) + lane] = (uint16_t)SQ[k];
        }
        __syncwarp();

        // -- lanes own pairs: the backward add-max scan of 16 node pairs
        uint32_t acc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = 0u;
#pragma unroll 1
        for (int pass = pass0; pass < pass1; ++pass) {
            const int kl_raw = pass * 32 + lane;
            const bool live = kl_raw < P;
            const int kl = live ? kl_raw : P - 1;
            uint32_t G[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) G[q] = P16_NEG;
            const uint2 *ep = ej_s + kl;
#pragma unroll 2
            for (int pos = n - 1; pos >= 0; --pos) {
                const uint2 x = ep[pos * P];
                const uint32_t w2 = __byte_perm(x.x, 0u, 0x1010), e2 = __byte_perm(x.x, 0u, 0x3232);
                const uint32_t *row =
                    reinterpret_cast<const uint32_t *>(reinterpret_cast<const unsigned char *>(tw) + x.y);
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const uint32_t msk = row[q];
                    const uint32_t t = p16_addmax(G[q], e2, w2);
                    G[q] = (t & msk) | (G[q] & ~msk);
                }
            }
            const int km = klm_s[kl];
            const uint32_t *ckr = tw + (n + (km & 255)) * P16_TS;
            const uint32_t *sqr = tw + (n + MT + (km >> 8)) * P16_TS;
            if (live) {
#pragma unroll
                for (int q = 0; q < 16; ++q) acc[q] = p16_addmax(G[q], p16_add(ckr[q], sqr[q]), acc[q]);
            }
        }

        // -- maximum over the lanes: lane v ends with node pair v >> 1
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int b = 16 >> s, h = 8 >> s;
            const bool up = (lane & b) != 0;
#pragma unroll
            for (int i = 0; i < h; ++i) {
                const uint32_t send = up ? acc[i] : acc[i + h];
                const uint32_t keep = up ? acc[i + h] : acc[i];
                acc[i] = p16_max(keep, __shfl_xor_sync(0xffffffffu, send, b));
            }
        }
        const uint32_t v = p16_max(acc[0], __shfl_xor_sync(0xffffffffu, acc[0], 1));
        int32_t raise = (int32_t)((lane & 1) ? (v >> 16) : (v & 0xFFFFu));
        if (S > 1) {  // the team's maximum over its slices of the pairs
            raise_s[warp * 32 + lane] = raise;
            asm volatile("bar.sync %0, %1;" ::"r"(1 + team), "r"(S * 32) : "memory");
            if (slice == 0)
                for (int w = 1; w < S; ++w) raise = max(raise, raise_s[(warp + w) * 32 + lane]);
            asm volatile("bar.sync %0, %1;" ::"r"(1 + team), "r"(S * 32) : "memory");  // raise_s reused next
        }
        if (node < count && slice == 0) {
            int32_t lb = lb1 + raise;
            if (bad) {
                lb = FSP_LB_INVALID;
                atomicOr(I.status, 1);
            }
            lb_out[node] = lb;
        }
        __syncwarp();  // the tables are rewritten for the next 32 nodes
    }
}

typedef void (*Pool16Fn)(DevInst, const uint8_t *, const uint8_t *, long long, const long long *, int, int32_t *,
                         Pool16Smem);

static Pool16Fn pick_pool16(int mt, int nv, bool bidir)
{
#define FSP_CASE16(MT_, NV_) \
    if (mt == MT_ && nv == NV_) return bidir ? &k_bound_pool16<MT_, NV_, true> : &k_bound_pool16<MT_, NV_, false>;
    FSP_CASE16(5, 1) FSP_CASE16(5, 2) FSP_CASE16(10, 1) FSP_CASE16(10, 2) FSP_CASE16(20, 1) FSP_CASE16(20, 2)
#undef FSP_CASE16
    if (bidir && nv == 3) {  // bidirectional records of 30 and 31 jobs: 48 bytes
        if (mt == 5) return &k_bound_pool16<5, 3, true>;
        if (mt == 10) return &k_bound_pool16<10, 3, true>;
        if (mt == 20) return &k_bound_pool16<20, 3, true>;
    }
    return nullptr;
}

// Whether the packed kernel bounds this instance exactly: n <= 31 (one mask
// word, records of at most 32 bytes), m in {5, 10, 20}, and every grid path
// plus one processing time within 16 bits.
int pool16_eligible(const fsp_instance *I)
{
    return I->n <= 31 && fsp_mt(I->m) != 0 && (long long)(I->n + I->m) * I->pmax <= 16383;
}

// Build the instance's image when the packed kernel applies (called by
// fsp_create_instance, on its stream 0, before it synchronises).
int pool16_build(fsp_instance *I)
{
    if (!pool16_eligible(I)) return FSP_OK;
    const Pool16Smem L = pool16_layout(I, 1);
    FSP_CUDA(cudaMalloc(&I->d_p16, L.img_bytes));
    FSP_CUDA(cudaMemset(I->d_p16, 0, L.img_bytes));
    const int words = I->n * p16_rs(I->m) > I->n * I->P ? I->n * p16_rs(I->m) : I->n * I->P;
    k_pool16_image<<<(words + 255) / 256, 256>>>(I->n, I->m, I->P, I->d_p, I->d_q, I->d_we, I->d_order, L,
                                                 I->d_p16);
    FSP_CUDA(cudaGetLastError());
    return FSP_OK;
}

// Launch on a pool of count nodes; FSP_ERR_ARG (nothing launched) when the
// instance is not eligible or its tables do not fit.  warps = 0: the default
// CTA shape: 8 warps, fewer when the pool has fewer than 8 groups of 32 nodes
// per SM, so that a small pool still spreads over every SM; and when even one
// warp per group leaves most of the GPU's 16 warps per SM idle, teams of S
// warps per group (the largest divisor S of the passes over the pairs that
// keeps groups x S within SMs x 16).  FSP_POOL16_SLICES sets S (tests).
int pool16_bound(fsp_instance *I, const uint8_t *nodes, long long count, int32_t *lb_out, cudaStream_t st,
                 int warps)
{
    return pool16_bound_ex(I, nodes, count, nullptr, false, lb_out, st, warps);
}

// count: the number of records, or (dcount non-NULL) an upper bound on it,
// the exact number being read by the kernel from device memory.  bidir:
// bidirectional records (fsp_node_stride_bidir bytes: perm, d1, d2).
int pool16_bound_ex(fsp_instance *I, const uint8_t *nodes, long long count, const long long *dcount, bool bidir,
                    int32_t *lb_out, cudaStream_t st, int warps)
{
    if (!pool16_eligible(I) || !I->d_p16) return FSP_ERR_ARG;
    const int stride = bidir ? fsp_node_stride_bidir(I->n) : I->stride;
    Pool16Fn fn = pick_pool16(fsp_mt(I->m), stride / 16, bidir);
    if (!fn) return FSP_ERR_ARG;
    const long long groups = (count + 31) / 32;
    const int npass = (I->P + 31) / 32;
    int slices = 1;
    const char *es = getenv("FSP_POOL16_SLICES");
    if (es) {
        slices = atoi(es);
        if (slices < 1 || npass % slices != 0) slices = 1;
    } else if (warps <= 0) {
        for (int sl = npass; sl > 1; --sl)
            if (npass % sl == 0 && groups * sl <= (long long)I->sm_count * 16) { slices = sl; break; }
    }
    if (slices > 1) {
        warps = slices * (8 / slices > 1 ? 8 / slices : 1);
    } else if (warps <= 0) {
        const long long per_sm = (groups + I->sm_count - 1) / I->sm_count;
        warps = per_sm >= 16 ? 8 : per_sm >= 2 ? (int)((per_sm + 1) / 2) : 1;
    }
    if (warps > P16_MAX_WARPS) warps = P16_MAX_WARPS;
    Pool16Smem L = pool16_layout(I, warps, slices);
    while (warps > slices && (int)L.bytes > I->smem_optin) {
        warps -= slices;
        L = pool16_layout(I, warps, slices);
    }
    if ((int)L.bytes > I->smem_optin) return FSP_ERR_ARG;
    int rc = fsp_allow_smem(I, (const void *)fn, L.bytes);
    if (rc != FSP_OK) return rc;
    int per_sm = 1;
    if ((rc = fsp_blocks_per_sm(I, (const void *)fn, warps * 32, L.bytes, &per_sm)) != FSP_OK) return rc;
    long long grid = (long long)I->sm_count * per_sm;
    const long long teams = warps / slices;
    const long long need = (groups + teams - 1) / teams;
    if (need < grid) grid = need;
    fn<<<(unsigned)grid, warps * 32, L.bytes, st>>>(dev_view(I), I->d_p16, nodes, count, dcount, stride, lb_out, L);
    FSP_CUDA(cudaGetLastError());
    return FSP_OK;
}
