// fsp_bound.cuh -- kernel shape selection shared by the bounding and search
// kernels.
#pragma once

#include "fsp_bound2.cuh"

// Shapes compiled: mask words NW (n <= 32, 64, 128, 255) x machine template
// MT (5, 10, 20, or 0 = any m) with the Johnson entries in shared memory
// (ES), plus the any-m path reading entries from global memory.
#define FSP_SHAPES(X)                                                              \
    X(1, 5, true) X(1, 10, true) X(1, 20, true) X(1, 0, true) X(1, 0, false)        \
    X(2, 5, true) X(2, 10, true) X(2, 20, true) X(2, 0, true) X(2, 0, false)        \
    X(4, 5, true) X(4, 10, true) X(4, 20, true) X(4, 0, true) X(4, 0, false)        \
    X(8, 0, true) X(8, 0, false)

// Fast-path shapes (fsp_bound2.cuh): machines MT x record vectors NV
// (stride 16 * NV bytes) x mask words NW, two nodes per thread.
#define FSP_SHAPES2(X)                                                   \
    X(5, 1, 1) X(5, 2, 1) X(5, 3, 1) X(5, 3, 2) X(5, 4, 2)                \
    X(10, 1, 1) X(10, 2, 1) X(10, 3, 1) X(10, 3, 2) X(10, 4, 2)           \
    X(20, 1, 1) X(20, 2, 1) X(20, 3, 1) X(20, 3, 2) X(20, 4, 2)
#define FSP_NPT 2
#define FSP_B2 128

struct BoundShape {
    int ver;  // 2: fast path (fsp_bound2.cuh), 1: any shape (fsp_common.cuh)
    int nw, mt, nv;
    bool es;
    int B;
    BoundSmem L;
    Bound2Smem L2;
};

// Pick the kernel shape and CTA size whose shared memory fits the device.
int fsp_bound_shape(const fsp_instance *I, BoundShape *s);

// Packed kernel (fsp_pool16.cu): two nodes per register, one warp per 32
// nodes; for n <= 31, m in {5, 10, 20} and (n + m) * max p <= 16383.
int pool16_eligible(const fsp_instance *I);
int pool16_bound(fsp_instance *I, const uint8_t *nodes, long long count, int32_t *lb_out, cudaStream_t st,
                 int warps);
int pool16_bound_ex(fsp_instance *I, const uint8_t *nodes, long long count, const long long *dcount, bool bidir,
                    int32_t *lb_out, cudaStream_t st, int warps);
