/*
 * trmm_oracle.c -- plain FP64 triangular matrix-matrix product oracle.
 *
 * TEST INFRASTRUCTURE ONLY (see gemm_oracle.c): loaded by tests/ and nothing in the product.
 *
 * What it computes: the level-3 operation TRMM with the reference-BLAS dtrmm semantics on
 * column-major storage (one of the other level-3 operations GEMMFIP carries over to, Sec. 1
 * and Sec. 5):
 *
 *     side = 'L':  B := alpha * op(A) * B,   A is m x m
 *     side = 'R':  B := alpha * B * op(A),   A is n x n
 *
 * with B m x n, op(A) = A ('N') or A^T ('T'/'C'), A triangular: only its uplo triangle
 * ('L' lower, 'U' upper) is read; with diag = 'U' its diagonal is not read either and taken
 * as 1.  op(A) is lower triangular when (uplo = 'L') xor (transa != 'N').
 *
 * Entry (i, j) of the result is alpha * S with S the sum, over the indices p where op(A) may
 * be nonzero, in increasing p, accumulated in a double from +0.0:
 *     side 'L':  S = sum_p opA(i, p) * B(p, j)
 *     side 'R':  S = sum_p B(i, p) * opA(p, j)
 * opA(p, p) = 1 for a unit diagonal.  The product is formed out of place (a column or row of
 * the old B at a time), then written to B.  alpha == 0: B := 0 without reading A or B.
 * m == 0 or n == 0: nothing.  Compiled with -ffp-contract=off.
 */
#include <stdint.h>
#include <stdlib.h>

static double opa(const double *A, int64_t lda, int trans, int lower_op, int unit, int64_t r,
                  int64_t c, int *nz)
{
    /* element (r, c) of op(A); *nz = 0 outside op(A)'s triangle */
    *nz = lower_op ? (r >= c) : (r <= c);
    if (!*nz) return 0.0;
    if (r == c && unit) return 1.0;
    return trans ? A[c + r * lda] : A[r + c * lda];
}

int oracle_trmm(char side, char uplo, char transa, char diag, int64_t m, int64_t n,
                double alpha, const double *A, int64_t lda, double *B, int64_t ldb)
{
    int left = (side == 'L' || side == 'l'), right = (side == 'R' || side == 'r');
    int lo = (uplo == 'L' || uplo == 'l'), up = (uplo == 'U' || uplo == 'u');
    int tn = (transa == 'N' || transa == 'n');
    int tt = (transa == 'T' || transa == 't' || transa == 'C' || transa == 'c');
    int unit = (diag == 'U' || diag == 'u'), nonunit = (diag == 'N' || diag == 'n');
    int64_t nrowa = left ? m : n;
    if (!left && !right) return -1;
    if (!lo && !up) return -2;
    if (!tn && !tt) return -3;
    if (!unit && !nonunit) return -4;
    if (m < 0) return -5;
    if (n < 0) return -6;
    if (lda < (nrowa > 1 ? nrowa : 1)) return -9;
    if (ldb < (m > 1 ? m : 1)) return -11;
    if (m == 0 || n == 0) return 0;
    if (alpha == 0.0) {
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = 0; i < m; ++i) B[i + j * ldb] = 0.0;
        return 0;
    }
    int lower_op = lo ^ tt;
    if (left) {
        double *col = (double *)malloc((size_t)m * sizeof(double));
        if (!col) return 1;
        for (int64_t j = 0; j < n; ++j) {
            for (int64_t i = 0; i < m; ++i) col[i] = B[i + j * ldb];
            for (int64_t i = 0; i < m; ++i) {
                double s = 0.0;
                for (int64_t p = 0; p < m; ++p) {
                    int nz;
                    double a = opa(A, lda, tt, lower_op, unit, i, p, &nz);
                    if (nz) s += a * col[p];
                }
                B[i + j * ldb] = alpha * s;
            }
        }
        free(col);
    } else {
        double *row = (double *)malloc((size_t)n * sizeof(double));
        if (!row) return 1;
        for (int64_t i = 0; i < m; ++i) {
            for (int64_t j = 0; j < n; ++j) row[j] = B[i + j * ldb];
            for (int64_t j = 0; j < n; ++j) {
                double s = 0.0;
                for (int64_t p = 0; p < n; ++p) {
                    int nz;
                    double a = opa(A, lda, tt, lower_op, unit, p, j, &nz);
                    if (nz) s += row[p] * a;
                }
                B[i + j * ldb] = alpha * s;
            }
        }
        free(row);
    }
    return 0;
}
