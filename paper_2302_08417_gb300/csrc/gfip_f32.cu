// FP32 instantiation of the fused-in-packing GEMM kernels (FFMA tile core).
#include "gfip_kernels.cuh"

GFIP_INSTANTIATE(float)
