// fsp_bound.cu -- K1: parallel bounding of a pool of node records (the
// paper's Type 1 model, Sec. II-A / III: one lower-bound evaluation per
// subproblem, all subproblems of the pool in parallel).
//
// Layout: one thread per node; the CTA stages the instance tables (p, tails,
// and the P x n Johnson entries) into shared memory once, so every table read
// of the pair loop is a broadcast (all lanes read the same entry).  The grid
// is persistent (SMs x resident CTAs) and strides over the pool.
#include <stdlib.h>

#include "fsp_family.cuh"

template <int NW, int MT, bool ES>
__global__ void __launch_bounds__(256) k_bound_pool(DevInst I, const uint8_t *__restrict__ nodes,
                                                    long long count, int32_t *__restrict__ lb_out,
                                                    BoundSmem L)
{
    extern __shared__ __align__(16) unsigned char smem[];
    FspEntry *ent_s = ES ? reinterpret_cast<FspEntry *>(smem + L.ent_off) : nullptr;
    int32_t *p_s = reinterpret_cast<int32_t *>(smem + L.p_off);
    int32_t *q_s = reinterpret_cast<int32_t *>(smem + L.q_off);
    const int B = blockDim.x, tid = threadIdx.x;
    uint32_t *rec = reinterpret_cast<uint32_t *>(smem + L.rec_off) + tid;
    int32_t *cs = reinterpret_cast<int32_t *>(smem + L.cs_off) + tid;
    int32_t *sq = reinterpret_cast<int32_t *>(smem + L.sq_off) + tid;
    int32_t *ss = reinterpret_cast<int32_t *>(smem + L.ss_off) + tid;
    fsp_stage_tables(I, ent_s, p_s, q_s);
    const FspEntry *ent = ES ? ent_s : I.ent;
    const int nvec = I.stride >> 4;
    for (long long base = (long long)blockIdx.x * B; base < count; base += (long long)gridDim.x * B) {
        const long long node = base + tid;
        if (node < count) {
            const uint4 *src = reinterpret_cast<const uint4 *>(nodes + node * I.stride);
            for (int c = 0; c < nvec; ++c) {
                const uint4 v = __ldg(src + c);
                rec[(4 * c + 0) * B] = v.x;
                rec[(4 * c + 1) * B] = v.y;
                rec[(4 * c + 2) * B] = v.z;
                rec[(4 * c + 3) * B] = v.w;
            }
            bool bad;
            int32_t lb = fsp_node_bound<NW, MT, ES>(I, ent, p_s, q_s, rec, cs, sq, ss, B, bad);
            if (bad) {
                lb = FSP_LB_INVALID;
                atomicOr(I.status, 1);
            }
            lb_out[node] = lb;
        }
    }
}

// Fast path: NPT nodes per thread, registers, DPX add-max (fsp_bound2.cuh).
template <int MT, int NV, int NW>
__global__ void __launch_bounds__(FSP_B2) k_bound_pool2(DevInst I, const uint8_t *__restrict__ nodes,
                                                        long long count, int32_t *__restrict__ lb_out,
                                                        Bound2Smem L)
{
    constexpr int NPT = FSP_NPT;
    extern __shared__ __align__(16) unsigned char smem[];
    FspEntry *ent_s = reinterpret_cast<FspEntry *>(smem + L.ent_off);
    int2 *pq_s = reinterpret_cast<int2 *>(smem + L.pq_off);
    int32_t *cs = reinterpret_cast<int32_t *>(smem + L.cs_off);
    int32_t *sq = reinterpret_cast<int32_t *>(smem + L.sq_off);
    fsp_stage_pq(I, ent_s, pq_s);
    const int B = blockDim.x, tid = threadIdx.x, SB = B * NPT;
    int slot[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) slot[j] = tid + j * B;
    for (long long base = (long long)blockIdx.x * SB; base < count; base += (long long)gridDim.x * SB) {
        uint32_t Um[NPT][NW];
        int32_t lb[NPT];
        bool bad[NPT];
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            const long long node = base + slot[j];
            FspRec<NV> r;
            if (node < count) {
                fsp_load_rec(r, nodes + node * I.stride);
            } else {
#pragma unroll
                for (int q = 0; q < 4 * NV; ++q) r.w[q] = 0u;
            }
            int32_t C[MT], SQ[MT];
            fsp_prologue<MT, NV, NW>(r, I.n, pq_s, I.mp, Um[j], C, SQ, lb[j], bad[j], I.var);
#pragma unroll
            for (int k = 0; k < MT; ++k) {
                cs[k * SB + slot[j]] = C[k];
                sq[k * SB + slot[j]] = SQ[k];
            }
        }
        fsp_pair_scan<MT, NPT, NW>(I.n, ent_s, cs, sq, SB, slot, Um, lb);
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            const long long node = base + slot[j];
            if (node < count) {
                int32_t v = lb[j];
                if (bad[j]) {
                    v = FSP_LB_INVALID;
                    atomicOr(I.status, 1);
                }
                lb_out[node] = v;
            }
        }
    }
}

typedef void (*BoundPool2Fn)(DevInst, const uint8_t *, long long, int32_t *, Bound2Smem);

static BoundPool2Fn pick_bound_pool2(int mt, int nv, int nw)
{
#define FSP_CASE2(MT_, NV_, NW_) \
    if (mt == MT_ && nv == NV_ && nw == NW_) return &k_bound_pool2<MT_, NV_, NW_>;
    FSP_SHAPES2(FSP_CASE2)
#undef FSP_CASE2
    return nullptr;
}

typedef void (*BoundPoolFn)(DevInst, const uint8_t *, long long, int32_t *, BoundSmem);

static BoundPoolFn pick_bound_pool(int nw, int mt, bool es)
{
#define FSP_CASE(NW_, MT_, ES_) \
    if (nw == NW_ && mt == MT_ && es == ES_) return &k_bound_pool<NW_, MT_, ES_>;
    FSP_SHAPES(FSP_CASE)
#undef FSP_CASE
    return nullptr;
}

int fsp_bound_shape(const fsp_instance *I, BoundShape *s)
{
    int nw = fsp_nw(I->n), mt = fsp_mt(I->m);
    s->nv = I->stride / 16;
    if (mt != 0 && nw <= 2 && s->nv <= 4 && !getenv("FSP_BOUND_V1")) {
        Bound2Smem L2 = bound2_smem_layout(I, FSP_B2, FSP_NPT, mt);
        if ((int)L2.bytes <= I->smem_optin) {
            s->ver = 2; s->nw = nw; s->mt = mt; s->es = false; s->B = FSP_B2; s->L2 = L2;
            return FSP_OK;
        }
    }
    s->ver = 1;
    if (nw == 8) mt = 0;
    const int blocks[4] = {256, 128, 64, 32};
    for (int t = 0; t < 4; ++t) {
        const int B = blocks[t];
        BoundSmem L = bound_smem_layout(I, B, true, mt);
        if ((int)L.bytes <= I->smem_optin) {
            s->nw = nw; s->mt = mt; s->es = true; s->B = B; s->L = L;
            return FSP_OK;
        }
        L = bound_smem_layout(I, B, false, 0);
        if ((int)L.bytes <= I->smem_optin) {
            s->nw = nw; s->mt = 0; s->es = false; s->B = B; s->L = L;
            return FSP_OK;
        }
    }
    fsp_set_error("instance %dx%d does not fit in shared memory", I->n, I->m);
    return FSP_ERR_ARG;
}

extern "C" int fsp_bound_pool(fsp_instance *I, const uint8_t *nodes, int64_t count, int32_t ub,
                              int32_t *lb_out, void *stream)
{
    (void)ub;
    if (!I) { fsp_set_error("fsp_bound_pool: inst is NULL"); return FSP_ERR_ARG; }
    if (count < 0) { fsp_set_error("fsp_bound_pool: count < 0"); return FSP_ERR_ARG; }
    if (count == 0) return FSP_OK;
    if (!nodes || !lb_out) { fsp_set_error("fsp_bound_pool: NULL buffer"); return FSP_ERR_ARG; }
    if (((uintptr_t)nodes & 15) != 0) {
        fsp_set_error("fsp_bound_pool: nodes must be 16-byte aligned");
        return FSP_ERR_ARG;
    }
    if (pool16_eligible(I) && !getenv("FSP_BOUND_V1") && !getenv("FSP_BOUND_V2")) {
        const char *w = getenv("FSP_POOL16_WARPS");
        return pool16_bound(I, nodes, count, lb_out, (cudaStream_t)stream, w ? atoi(w) : 0);
    }
    BoundShape s;
    int rc = fsp_bound_shape(I, &s);
    if (rc != FSP_OK) return rc;
    if (s.ver == 2 && count <= FAM_POOL_SMALL && !getenv("FSP_FAMILY_POOL0")) {
        // a pool too small to fill the GPU one node per thread: one warp per node
        rc = fam_bound_pool(I, s.mt, s.nv, nodes, count, lb_out, (cudaStream_t)stream);
        if (rc != FSP_ERR_ARG) return rc;
        rc = FSP_OK;
    }
    if (s.ver == 2) {
        BoundPool2Fn fn2 = pick_bound_pool2(s.mt, s.nv, s.nw);
        if (!fn2) { fsp_set_error("fsp_bound_pool: no kernel for this shape"); return FSP_ERR_ARG; }
        if ((rc = fsp_allow_smem(I, (const void *)fn2, s.L2.bytes)) != FSP_OK) return rc;
        int per_sm = 1;
        if ((rc = fsp_blocks_per_sm(I, (const void *)fn2, s.B, s.L2.bytes, &per_sm)) != FSP_OK) return rc;
        const long long per_block = (long long)s.B * FSP_NPT;
        long long need = (count + per_block - 1) / per_block;
        long long grid = (long long)I->sm_count * per_sm;
        if (need < grid) grid = need;
        fn2<<<(unsigned)grid, s.B, s.L2.bytes, (cudaStream_t)stream>>>(dev_view(I), nodes, (long long)count,
                                                                       lb_out, s.L2);
        FSP_CUDA(cudaGetLastError());
        return FSP_OK;
    }
    BoundPoolFn fn = pick_bound_pool(s.nw, s.mt, s.es);
    if (!fn) { fsp_set_error("fsp_bound_pool: no kernel for this shape"); return FSP_ERR_ARG; }
    if ((rc = fsp_allow_smem(I, (const void *)fn, s.L.bytes)) != FSP_OK) return rc;
    int per_sm = 1;
    if ((rc = fsp_blocks_per_sm(I, (const void *)fn, s.B, s.L.bytes, &per_sm)) != FSP_OK) return rc;
    long long need = (count + s.B - 1) / s.B;
    long long grid = (long long)I->sm_count * per_sm;
    if (need < grid) grid = need;
    fn<<<(unsigned)grid, s.B, s.L.bytes, (cudaStream_t)stream>>>(dev_view(I), nodes, (long long)count,
                                                                 lb_out, s.L);
    FSP_CUDA(cudaGetLastError());
    return FSP_OK;
}

extern "C" int fsp_check_status(fsp_instance *I, void *stream)
{
    if (!I) { fsp_set_error("fsp_check_status: inst is NULL"); return FSP_ERR_ARG; }
    FSP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int h = 0;
    FSP_CUDA(cudaMemcpy(&h, I->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        FSP_CUDA(cudaMemset(I->d_status, 0, sizeof(int)));
        fsp_set_error("malformed node record (depth > n, job id >= n or repeated job)");
        return FSP_ERR_ARG;
    }
    return FSP_OK;
}
