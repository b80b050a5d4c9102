// gfip_trsm.cu -- the diagonal-block solves of the blocked triangular solve (TRSM).
//
// TRSM runs as a sequence over the diagonal blocks of op(A) (see gfip_api.cu): each step
// solves one block of at most TRSM_NB unknowns for every right-hand side with the kernel
// below, then the fused GEMM kernel subtracts that block's contribution from the unknowns
// still to be solved.  The block's triangle is staged in shared memory (only the entries a
// triangular solve reads: never the other triangle, nor a unit diagonal); one thread runs the
// substitution for one right-hand side, in place in B.
#include <cstdint>

#include "gfip_internal.h"

namespace gfip {

template <typename T>
__global__ void __launch_bounds__(128)
    trsm_diag_kernel(T *B, int64_t vstride, int64_t estride, int nvec, const T *A, int64_t lda,
                     int a_trans, int k0, int nb, int lower_t, int transpose_t, int unit)
{
    __shared__ T t[TRSM_NB][TRSM_NB + 1];
    // t(r, c) = op(A)[k0 + r, k0 + c] (side 'L') or op(A)[k0 + c, k0 + r] (side 'R'),
    // op(A)[i, j] = A[i + j lda] ('N') or A[j + i lda] ('T')
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int r = e % nb, c = e / nb;
        const bool need = (lower_t ? r > c : r < c) || (r == c && !unit);
        T v = T(0);
        if (need) {
            const int oi = k0 + (transpose_t ? c : r), oj = k0 + (transpose_t ? r : c);
            v = a_trans ? A[oj + (int64_t)oi * lda] : A[oi + (int64_t)oj * lda];
        }
        t[r][c] = v;
    }
    __syncthreads();
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvec) return;
    T *x = B + (int64_t)v * vstride;
    for (int q = 0; q < nb; ++q) {
        const int i = lower_t ? q : nb - 1 - q;
        T s = x[(int64_t)i * estride];
        for (int d = 0; d < q; ++d) {
            const int c = lower_t ? d : nb - 1 - d;
            s -= t[i][c] * x[(int64_t)c * estride];
        }
        if (!unit) s = s / t[i][i];
        x[(int64_t)i * estride] = s;
    }
}

template <typename T>
cudaError_t launch_trsm_diag_impl(T *B, int64_t vstride, int64_t estride, int nvec, const T *A,
                                  int64_t lda, int a_trans, int k0, int nb, int lower_t,
                                  int transpose_t, int unit, cudaStream_t s)
{
    if (nvec <= 0 || nb <= 0) return cudaSuccess;
    const int threads = 128;
    trsm_diag_kernel<T><<<(nvec + threads - 1) / threads, threads, 0, s>>>(
        B, vstride, estride, nvec, A, lda, a_trans, k0, nb, lower_t, transpose_t, unit);
    return cudaGetLastError();
}

template <>
cudaError_t launch_trsm_diag<double>(double *B, int64_t vstride, int64_t estride, int nvec,
                                     const double *A, int64_t lda, int a_trans, int k0, int nb,
                                     int lower_t, int transpose_t, int unit, cudaStream_t s)
{
    return launch_trsm_diag_impl<double>(B, vstride, estride, nvec, A, lda, a_trans, k0, nb,
                                         lower_t, transpose_t, unit, s);
}

template <>
cudaError_t launch_trsm_diag<float>(float *B, int64_t vstride, int64_t estride, int nvec,
                                    const float *A, int64_t lda, int a_trans, int k0, int nb,
                                    int lower_t, int transpose_t, int unit, cudaStream_t s)
{
    return launch_trsm_diag_impl<float>(B, vstride, estride, nvec, A, lda, a_trans, k0, nb,
                                        lower_t, transpose_t, unit, s);
}

}  // namespace gfip
