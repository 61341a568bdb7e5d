// fsp_bound.cuh -- kernel shape selection shared by the bounding and search
// kernels.
#pragma once

#include "fsp_common.cuh"

// Shapes compiled: mask words NW (n <= 32, 64, 128, 255) x machine template
// MT (5, 10, 20, or 0 = any m) with the Johnson entries in shared memory
// (ES), plus the any-m path reading entries from global memory.
#define FSP_SHAPES(X)                                                              \
    X(1, 5, true) X(1, 10, true) X(1, 20, true) X(1, 0, true) X(1, 0, false)        \
    X(2, 5, true) X(2, 10, true) X(2, 20, true) X(2, 0, true) X(2, 0, false)        \
    X(4, 5, true) X(4, 10, true) X(4, 20, true) X(4, 0, true) X(4, 0, false)        \
    X(8, 0, true) X(8, 0, false)

struct BoundShape {
    int nw, mt;
    bool es;
    int B;
    BoundSmem L;
};

// Pick the kernel shape and CTA size whose shared memory fits the device.
int fsp_bound_shape(const fsp_instance *I, BoundShape *s);
