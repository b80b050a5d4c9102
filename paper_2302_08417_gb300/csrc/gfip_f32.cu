// FP32 instantiation of the fused-in-packing GEMM kernels (FFMA tile core).  The TRMM
// (triangular-operand) instantiations come from gfip_f32_tmask.cu.
#include "gfip_kernels.cuh"

GFIP_TMASK_LAUNCHERS(extern, float)
GFIP_INSTANTIATE(float)
