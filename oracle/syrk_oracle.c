/*
 * syrk_oracle.c -- plain FP64 symmetric rank-k update oracle.
 *
 * TEST INFRASTRUCTURE ONLY (see gemm_oracle.c): loaded by tests/ and nothing in the product.
 *
 * What it computes: the level-3 operation the GEMMFIP paper lists among the other
 * operations its technique carries over to (Sec. 1 and Sec. 5: the rest of the level-3
 * BLAS), with the reference-BLAS dsyrk semantics on column-major storage:
 *
 *     trans = 'N':  C := alpha * A * A^T + beta * C,   A is n x k
 *     trans = 'T':  C := alpha * A^T * A + beta * C,   A is k x n
 *
 * only the triangle uplo ('L' lower: i >= j, 'U' upper: i <= j) of the n x n matrix C is
 * read or written; the other triangle and rows n..ldc-1 are never touched.  Entry (i, j)
 * of the triangle is S = sum_{p=0}^{k-1} a(i,p) a(j,p) with a(i,p) = A[i + p*lda] ('N') or
 * A[p + i*lda] ('T'/'C'), accumulated in a double from +0.0 with p increasing, then
 * alpha*S + beta*C (beta*C not formed when beta == 0, so C is not read).  alpha == 0 or
 * k == 0: A is not read, C := beta*C on the triangle; n == 0 or (alpha == 0 or k == 0) and
 * beta == 1: C untouched.  Compiled with -ffp-contract=off.
 */
#include <stdint.h>

int oracle_syrk(char uplo, char trans, int64_t n, int64_t k, double alpha, const double *A,
                int64_t lda, double beta, double *C, int64_t ldc)
{
    int lower = (uplo == 'L' || uplo == 'l');
    int upper = (uplo == 'U' || uplo == 'u');
    int notrans = (trans == 'N' || trans == 'n');
    int tr = (trans == 'T' || trans == 't' || trans == 'C' || trans == 'c');
    int64_t rows_a = notrans ? n : k;
    if (!lower && !upper) return -1;
    if (!notrans && !tr) return -2;
    if (n < 0) return -3;
    if (k < 0) return -4;
    if (lda < (rows_a > 1 ? rows_a : 1)) return -7;
    if (ldc < (n > 1 ? n : 1)) return -10;
    if (n == 0 || ((alpha == 0.0 || k == 0) && beta == 1.0)) return 0;
    for (int64_t j = 0; j < n; ++j) {
        int64_t i0 = lower ? j : 0, i1 = lower ? n : j + 1;
        for (int64_t i = i0; i < i1; ++i) {
            double *c = C + i + j * ldc;
            if (alpha == 0.0 || k == 0) {
                *c = (beta == 0.0) ? 0.0 : beta * *c;
                continue;
            }
            double s = 0.0;
            for (int64_t p = 0; p < k; ++p) {
                double ai = notrans ? A[i + p * lda] : A[p + i * lda];
                double aj = notrans ? A[j + p * lda] : A[p + j * lda];
                s += ai * aj;
            }
            double v = alpha * s;
            if (beta != 0.0) v += beta * *c;
            *c = v;
        }
    }
    return 0;
}
