/*
 * trsm_oracle.c -- plain FP64 triangular solve with many right-hand sides.
 *
 * TEST INFRASTRUCTURE ONLY (see gemm_oracle.c): loaded by tests/ and nothing in the product.
 *
 * What it computes: the level-3 operation TRSM with the reference-BLAS dtrsm semantics on
 * column-major storage (one of the other level-3 operations GEMMFIP carries over to, Sec. 1
 * and Sec. 5):
 *
 *     side = 'L':  solve op(A) * X = alpha * B,   A is m x m
 *     side = 'R':  solve X * op(A) = alpha * B,   A is n x n
 *
 * and overwrite B (m x n) with X; op(A), uplo and diag as in trmm_oracle.c (only the uplo
 * triangle of A is read, and not its diagonal when diag = 'U', taken as 1).
 *
 * Method: B := alpha * B first, then plain substitution, one right-hand side at a time:
 * side 'L' solves each column x of X from op(A) x = b, side 'R' each row y of X from
 * y op(A) = b, i.e. op(A)^T y^T = b^T.  For a lower triangular system the unknowns are found
 * in increasing index order (forward substitution), for an upper one in decreasing order:
 *     x_i = (b_i - sum_{c before i} t(i, c) x_c) / t(i, i),
 * the sum accumulated in a double from b_i, c in increasing distance order from the start
 * (increasing c for forward, decreasing c for backward substitution), no division for a
 * unit diagonal.  alpha == 0: B := 0 without reading A or B.  Compiled -ffp-contract=off.
 */
#include <stdint.h>

static double opa_el(const double *A, int64_t lda, int trans, int64_t r, int64_t c)
{
    return trans ? A[c + r * lda] : A[r + c * lda];
}

int oracle_trsm(char side, char uplo, char transa, char diag, int64_t m, int64_t n,
                double alpha, const double *A, int64_t lda, double *B, int64_t ldb)
{
    int left = (side == 'L' || side == 'l'), right = (side == 'R' || side == 'r');
    int lo = (uplo == 'L' || uplo == 'l'), up = (uplo == 'U' || uplo == 'u');
    int tn = (transa == 'N' || transa == 'n');
    int tt = (transa == 'T' || transa == 't' || transa == 'C' || transa == 'c');
    int unit = (diag == 'U' || diag == 'u'), nonunit = (diag == 'N' || diag == 'n');
    int64_t na = left ? m : n;
    if (!left && !right) return -1;
    if (!lo && !up) return -2;
    if (!tn && !tt) return -3;
    if (!unit && !nonunit) return -4;
    if (m < 0) return -5;
    if (n < 0) return -6;
    if (lda < (na > 1 ? na : 1)) return -9;
    if (ldb < (m > 1 ? m : 1)) return -11;
    if (m == 0 || n == 0) return 0;
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i)
            B[i + j * ldb] = (alpha == 0.0) ? 0.0 : alpha * B[i + j * ldb];
    if (alpha == 0.0) return 0;
    int lower_op = lo ^ tt;
    /* t(r, c): the system matrix -- op(A) for side L, op(A)^T for side R */
    int lower_t = left ? lower_op : !lower_op;
    int64_t nvec = left ? n : m;
    for (int64_t v = 0; v < nvec; ++v) {
        /* element i of right-hand side v */
        double *base = left ? B + v * ldb : B + v;
        int64_t step = left ? 1 : ldb;
        for (int64_t q = 0; q < na; ++q) {
            int64_t i = lower_t ? q : na - 1 - q;
            double s = base[i * step];
            for (int64_t d = 0; d < q; ++d) {
                int64_t c = lower_t ? d : na - 1 - d;
                double t = left ? opa_el(A, lda, tt, i, c) : opa_el(A, lda, tt, c, i);
                s -= t * base[c * step];
            }
            if (!unit) {
                double t = left ? opa_el(A, lda, tt, i, i) : opa_el(A, lda, tt, i, i);
                s = s / t;
            }
            base[i * step] = s;
        }
    }
    return 0;
}
