// FP64 instantiation of the fused-in-packing GEMM kernels (DFMA tile core).  The TRMM
// (triangular-operand) instantiations come from gfip_f64_tmask.cu.
#include "gfip_kernels.cuh"

GFIP_TMASK_LAUNCHERS(extern, double)
GFIP_INSTANTIATE(double)
