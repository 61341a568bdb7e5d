// fsp_family.cuh -- the family kernel (fsp_family.cu): a parent's children
// branched and bounded together, one warp per parent.
#pragma once

#include "fsp_solve.cuh"

#define FAM_MAX_WARPS 16  // warps per CTA at most (one parent per warp at a time)
#define FAM_MIN_WARPS 4   // below this the per-child kernel is used
#define FAM_TS 33         // row stride of the per-warp scan table (32 pairs + 1)

// Compiled shapes: machines MT x record vectors NV (n <= 16 NV - 1).
#define FSP_SHAPES_FAMILY(X) \
    X(5, 1) X(5, 2) X(5, 3) X(5, 4) X(10, 1) X(10, 2) X(10, 3) X(10, 4) X(20, 1) X(20, 2) X(20, 3) X(20, 4)

// Position masks: n <= 31 jobs fit 32 bits (records of up to 32 bytes).
template <int NV>
struct FamMask {
    typedef unsigned long long type;
};
template <>
struct FamMask<1> {
    typedef uint32_t type;
};
template <>
struct FamMask<2> {
    typedef uint32_t type;
};

// Shared memory of a family CTA.  Instance tables: the Johnson entries
// position-major (we), each job's position per pair (rk8), max(0, -e) per
// job and pair (en) and its maximum over the jobs (gam), each pair's
// machines (klm), the {p, q} rows (pq).  Then per warp (offsets w_*): the
// parent state, the record buffers, the children's release times, S + qmin
// and running bounds (rows of mtp words), the scan table T [n][FAM_TS] and
// the list of pairs still to evaluate.
struct FamSmem {
    size_t we_off, rk8_off, en_off, gam_off, klm_off, pq_off, warp_off, warp_bytes, bytes;
    size_t w_ps, w_psa, w_ab, w_rec, w_pofs, w_cc, w_sq, w_lb, w_T, w_lkl, w_lm;
    int rks8, mtp, warps;
    int K;  // learned order: predicted pairs per parent
};

FamSmem family_smem_layout(const fsp_instance *I, int MT, int NV, int warps);
int family_warps(const fsp_instance *I, int MT, int NV);

typedef void (*BranchFamilyFn)(DevInst, SolveWs, FamSmem);
BranchFamilyFn pick_branch_family(int mt, int nv, bool learned);
