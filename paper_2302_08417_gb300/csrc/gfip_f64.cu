// FP64 instantiation of the fused-in-packing GEMM kernels (DFMA tile core).
#include "gfip_kernels.cuh"

GFIP_INSTANTIATE(double)
