// gfip_trsm.cu -- the diagonal-block solves of the blocked triangular solve (TRSM).
//
// TRSM runs as a sequence over the diagonal blocks of op(A) (see gfip_api.cu): each step
// solves one block of at most TRSM_NB unknowns for every right-hand side with the kernel
// below, then the fused GEMM kernel subtracts that block's contribution from the unknowns
// still to be solved.  The block's triangle is staged in shared memory (only the entries a
// triangular solve reads: never the other triangle, nor a unit diagonal); one thread runs the
// substitution for one right-hand side, on a copy of the block's rows of it in shared memory.
#include <cstdint>

#include "gfip_internal.h"

namespace gfip {

// Right-hand sides per CTA (one warp): the block's rows of them are staged in shared memory
// with coalesced loads (the unit-stride direction of B runs across the threads), solved
// there, and written back the same way.
constexpr int TRSM_VPC = 32;

template <typename T> constexpr size_t trsm_diag_smem()
{
    return sizeof(T) * (size_t)TRSM_NB * TRSM_NB + sizeof(T) * (size_t)TRSM_NB * (TRSM_VPC + 1);
}

template <typename T>
__global__ void __launch_bounds__(TRSM_VPC)
    trsm_diag_kernel(T *B, int64_t vstride, int64_t estride, int nvec, const T *A, int64_t lda,
                     int a_trans, int k0, int nb, int lower_t, int transpose_t, int unit)
{
    extern __shared__ __align__(16) unsigned char smem[];
    // t(r, c) = op(A)[k0 + r, k0 + c] (side 'L') or op(A)[k0 + c, k0 + r] (side 'R'),
    // op(A)[i, j] = A[i + j lda] ('N') or A[j + i lda] ('T'); read by all threads at once
    T(*t)[TRSM_NB] = reinterpret_cast<T(*)[TRSM_NB]>(smem);
    // xs(i, v) = element i of right-hand side v0 + v (padded: conflict-free along i and v)
    T(*xs)[TRSM_VPC + 1] =
        reinterpret_cast<T(*)[TRSM_VPC + 1]>(smem + sizeof(T) * TRSM_NB * TRSM_NB);
    const int tid = threadIdx.x;
    const int v0 = blockIdx.x * TRSM_VPC;
    const int nv = min(TRSM_VPC, nvec - v0);
    for (int e = tid; e < nb * nb; e += TRSM_VPC) {
        const int r = e / nb, c = e % nb;
        const bool need = (lower_t ? r > c : r < c) || (r == c && !unit);
        T v = T(0);
        if (need) {
            const int oi = k0 + (transpose_t ? c : r), oj = k0 + (transpose_t ? r : c);
            v = a_trans ? A[oj + (int64_t)oi * lda] : A[oi + (int64_t)oj * lda];
        }
        t[r][c] = v;
    }
    // element i of vector v sits at B[v vstride + i estride]; one of the strides is 1
    const bool along_i = (estride == 1);
    for (int e = tid; e < nb * nv; e += TRSM_VPC) {
        const int i = along_i ? e % nb : e / nv, v = along_i ? e / nb : e % nv;
        xs[i][v] = B[(int64_t)(v0 + v) * vstride + (int64_t)i * estride];
    }
    __syncthreads();
    if (tid < nv) {
        for (int q = 0; q < nb; ++q) {
            const int i = lower_t ? q : nb - 1 - q;
            T s = xs[i][tid];
            for (int d = 0; d < q; ++d) {
                const int c = lower_t ? d : nb - 1 - d;
                s -= t[i][c] * xs[c][tid];
            }
            if (!unit) s = s / t[i][i];
            xs[i][tid] = s;
        }
    }
    __syncthreads();
    for (int e = tid; e < nb * nv; e += TRSM_VPC) {
        const int i = along_i ? e % nb : e / nv, v = along_i ? e / nb : e % nv;
        B[(int64_t)(v0 + v) * vstride + (int64_t)i * estride] = xs[i][v];
    }
}

template <typename T>
cudaError_t launch_trsm_diag_impl(T *B, int64_t vstride, int64_t estride, int nvec, const T *A,
                                  int64_t lda, int a_trans, int k0, int nb, int lower_t,
                                  int transpose_t, int unit, cudaStream_t s)
{
    if (nvec <= 0 || nb <= 0) return cudaSuccess;
    if (nb > TRSM_NB) return cudaErrorInvalidValue;
    static bool configured = false;
    if (!configured) {
        const cudaError_t e = cudaFuncSetAttribute(trsm_diag_kernel<T>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   static_cast<int>(trsm_diag_smem<T>()));
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int blocks = (nvec + TRSM_VPC - 1) / TRSM_VPC;
    trsm_diag_kernel<T><<<blocks, TRSM_VPC, trsm_diag_smem<T>(), s>>>(
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
