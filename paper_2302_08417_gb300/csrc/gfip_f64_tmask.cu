// FP64 GEMM kernels with triangular-operand masks (TRMM), compiled apart from the others.
#include "gfip_kernels.cuh"

GFIP_TMASK_LAUNCHERS(, double)
