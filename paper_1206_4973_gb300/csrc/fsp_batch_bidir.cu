// fsp_batch_bidir.cu -- the batch kernels with bidirectional branching (a
// translation unit of their own: the template instantiations compile in
// parallel with the forward ones of fsp_batch.cu).
#include "fsp_batch.cuh"

typedef void (*BatchFn)(const BatchDesc *, const int *, int, const int32_t *, BatchOut *, uint8_t *, int *, BatchWs);
typedef void (*BatchSplitFn)(const BatchDesc *, const int *, int, const int32_t *, int *, BatchWs, BatchSplit);

BatchFn batch_kernel_bidir() { return &k_batch<true>; }
BatchSplitFn batch_split_kernel_bidir() { return &k_batch_split<true>; }
