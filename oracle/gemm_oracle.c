/*
 * gemm_oracle.c -- plain FP64 GEMM oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline / reference arm load this file's library.  It shares no code, header,
 * table or helper with the CUDA path, and the CUDA path never calls it.
 *
 * What it computes (GEMMFIP, Sec. 2.1: the prototypical gemm C := A B + C with A m x k,
 * B k x n, C m x n; extended to the BLAS dgemm semantics C := alpha op(A) op(B) + beta C,
 * op(X) = X or X^T, on column-major operands with leading dimensions, Sec. 1):
 *
 *     C[i,j] <- alpha * S[i,j] + beta * C[i,j],   S[i,j] = sum_{p=0}^{k-1} op(A)[i,p] * op(B)[p,j]
 *
 * with op(A)[i,p] = A[i + p*lda] for transa = 'N' and A[p + i*lda] for 'T'/'C', and
 * op(B)[p,j] = B[p + j*ldb] for 'N' and B[j + p*ldb] for 'T'/'C'.
 *
 * Arithmetic order: S[i,j] is accumulated in a double temporary starting from +0.0 with p
 * increasing, then scaled: alpha*S first, beta*C second, one addition.  Compiled with
 * -ffp-contract=off so no multiply-add is fused.  The loop nest is j, then p, then i (the
 * axpy form): for each element that is the same sequence of roundings as the dot form.
 * No blocking, no reordering, no SIMD intrinsics.
 *
 * BLAS rules kept: beta == 0 means C is not read (a NaN there does not propagate);
 * alpha == 0 or k == 0 means A and B are not read; m == 0, n == 0, or
 * ((alpha == 0 or k == 0) and beta == 1) return without touching C.  Rows m..ldc-1 of C
 * are never written.
 *
 * FIP (Sec. 3.2) changes only where the operands are read from, and the paper's kernels
 * compute the same C with or without packing (Sec. 3.1: the microkernel is used without
 * modification), so this single definition is the oracle for the fused, the pack-then-
 * compute and the direct variants alike.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Reference-BLAS argument check: returns 0, or minus the 1-based position of the first
 * bad argument in (transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc). */
static int oracle_check(char transa, char transb, int64_t m, int64_t n, int64_t k,
                        int64_t lda, int64_t ldb, int64_t ldc)
{
    int ta_ok = (transa == 'N' || transa == 'n' || transa == 'T' || transa == 't' ||
                 transa == 'C' || transa == 'c');
    int tb_ok = (transb == 'N' || transb == 'n' || transb == 'T' || transb == 't' ||
                 transb == 'C' || transb == 'c');
    int a_notrans = (transa == 'N' || transa == 'n');
    int b_notrans = (transb == 'N' || transb == 'n');
    int64_t rows_a = a_notrans ? m : k;
    int64_t rows_b = b_notrans ? k : n;
    if (!ta_ok) return -1;
    if (!tb_ok) return -2;
    if (m < 0) return -3;
    if (n < 0) return -4;
    if (k < 0) return -5;
    if (lda < (rows_a > 1 ? rows_a : 1)) return -8;
    if (ldb < (rows_b > 1 ? rows_b : 1)) return -10;
    if (ldc < (m > 1 ? m : 1)) return -13;
    return 0;
}

static double op_a(const double *A, int64_t lda, int a_notrans, int64_t i, int64_t p)
{
    return a_notrans ? A[i + p * lda] : A[p + i * lda];
}

static double op_b(const double *B, int64_t ldb, int b_notrans, int64_t p, int64_t j)
{
    return b_notrans ? B[p + j * ldb] : B[j + p * ldb];
}

/*
 * C := alpha*op(A)*op(B) + beta*C, in place, column-major, FP64.
 * nthreads > 1 splits the j loop (columns of C) over OpenMP threads; every element is
 * still produced by the same sequence of operations, so the result does not depend on
 * nthreads.  Returns 0, a negative BLAS argument position, or 1 if the temporary could not
 * be allocated.
 */
int oracle_gemm(char transa, char transb, int64_t m, int64_t n, int64_t k,
                double alpha, const double *A, int64_t lda,
                const double *B, int64_t ldb,
                double beta, double *C, int64_t ldc, int nthreads)
{
    int info = oracle_check(transa, transb, m, n, k, lda, ldb, ldc);
    if (info != 0) return info;
    if (m == 0 || n == 0) return 0;
    if ((alpha == 0.0 || k == 0) && beta == 1.0) return 0;

    int a_notrans = (transa == 'N' || transa == 'n');
    int b_notrans = (transb == 'N' || transb == 'n');
    int use_ab = !(alpha == 0.0 || k == 0);
    int failed = 0;
    if (nthreads < 1) nthreads = 1;

#pragma omp parallel num_threads(nthreads)
    {
        double *s = (double *)malloc((size_t)m * sizeof(double));
        if (s == NULL) {
#pragma omp atomic write
            failed = 1;
        } else {
#pragma omp for schedule(static)
            for (int64_t j = 0; j < n; ++j) {
                for (int64_t i = 0; i < m; ++i) s[i] = 0.0;
                if (use_ab) {
                    for (int64_t p = 0; p < k; ++p) {
                        double b = op_b(B, ldb, b_notrans, p, j);
                        for (int64_t i = 0; i < m; ++i) {
                            double prod = op_a(A, lda, a_notrans, i, p) * b;
                            s[i] = s[i] + prod;
                        }
                    }
                }
                double *c = C + j * ldc;
                for (int64_t i = 0; i < m; ++i) {
                    double t;
                    if (use_ab) {
                        t = alpha * s[i];
                        if (beta != 0.0) t = t + beta * c[i];
                    } else {
                        t = (beta != 0.0) ? beta * c[i] : 0.0;
                    }
                    c[i] = t;
                }
            }
            free(s);
        }
    }
    return failed ? 1 : 0;
}

/*
 * Selected entries of the same definition, for checks at sizes where the full product is
 * too slow on the CPU:  out[t] = alpha * S[ii[t], jj[t]] + beta * C0[ii[t], jj[t]], with S
 * summed over p in increasing order exactly as in oracle_gemm (same roundings, same result
 * bits).  C0 is the input C (read only; not read when beta == 0).
 *
 * With absval != 0 it returns instead the magnitude term of the error bound,
 *     |alpha| * sum_p |op(A)[i,p]| * |op(B)[p,j]| + |beta| * |C0[i,j]|,
 * used by the tests' tolerance.  Returns 0, a negative BLAS position, or -14 for an entry
 * index outside the m x n result.
 */
int oracle_gemm_entries(char transa, char transb, int64_t m, int64_t n, int64_t k,
                        double alpha, const double *A, int64_t lda,
                        const double *B, int64_t ldb,
                        double beta, const double *C0, int64_t ldc,
                        int64_t count, const int64_t *ii, const int64_t *jj,
                        double *out, int absval, int nthreads)
{
    int info = oracle_check(transa, transb, m, n, k, lda, ldb, ldc);
    if (info != 0) return info;
    for (int64_t t = 0; t < count; ++t)
        if (ii[t] < 0 || ii[t] >= m || jj[t] < 0 || jj[t] >= n) return -14;

    int a_notrans = (transa == 'N' || transa == 'n');
    int b_notrans = (transb == 'N' || transb == 'n');
    int use_ab = !(alpha == 0.0 || k == 0);
    if (nthreads < 1) nthreads = 1;

#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (int64_t t = 0; t < count; ++t) {
        int64_t i = ii[t], j = jj[t];
        double s = 0.0;
        if (use_ab) {
            for (int64_t p = 0; p < k; ++p) {
                double a = op_a(A, lda, a_notrans, i, p);
                double b = op_b(B, ldb, b_notrans, p, j);
                double prod = absval ? fabs(a) * fabs(b) : a * b;
                s = s + prod;
            }
        }
        double r;
        if (absval) {
            r = use_ab ? fabs(alpha) * s : 0.0;
            if (beta != 0.0) r = r + fabs(beta) * fabs(C0[i + j * ldc]);
        } else {
            if (use_ab) {
                r = alpha * s;
                if (beta != 0.0) r = r + beta * C0[i + j * ldc];
            } else if (beta == 1.0) {
                r = C0[i + j * ldc];
            } else {
                r = (beta != 0.0) ? beta * C0[i + j * ldc] : 0.0;
            }
        }
        out[t] = r;
    }
    return 0;
}

/* Number of OpenMP threads the library would use by default (1 without OpenMP). */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
