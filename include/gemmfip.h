/*
 * gemmfip.h -- C ABI of the GB300 (sm_103a) fused-in-packing GEMM library.
 *
 * Operation (GEMMFIP, Sec. 2.1: the gemm C := A B + C, with A m x k, B k x n, C m x n;
 * extended to the BLAS dgemm/sgemm interface of Sec. 1):
 *
 *     C := alpha * op(A) * op(B) + beta * C,      op(X) = X ('N') or X^T ('T', 'C')
 *
 * All matrices are column-major with leading dimensions (element (i, j) of a matrix with
 * leading dimension ld sits at index i + j*ld).  op(A) is m x k, op(B) is k x n.
 *
 * Method (Sec. 3.1-3.2, Alg. 1): every operand panel that is reused is packed into a
 * contiguous tile layout the first time a CTA computes with it, in the same pass ("fused-in
 * packing"); later CTAs load the packed copy.  Which operands are worth packing follows the
 * option table of Sec. 3.3 (pack A only if the result has more than one tile column, pack
 * B only if it has more than one tile row); one scheme serves every size, and a tile reads a
 * k-block packed whenever its producer has already published it.  The two comparison
 * variants of Sec. 2.3-2.4 are exported as well: a direct-strided kernel that never packs (the
 * SUP path) and a pack-then-compute pair of launches (the conventional path).  All three
 * produce bit-identical results for the same arguments on the same GPU.
 *
 * Pointers: A, B and C are DEVICE pointers owned by the caller; A and B are only read;
 * only the m x n logical region of C is written (rows m..ldc-1 are never touched).  Calls
 * are asynchronous on the handle's stream.
 *
 * Return codes: 0 on success; a negative value -p names the first invalid argument by its
 * 1-based position in the reference-BLAS argument list
 *     (transa=1, transb=2, m=3, n=4, k=5, alpha=6, A=7, lda=8, B=9, ldb=10, beta=11, C=12,
 *      ldc=13),
 * exactly as xerbla would report it; positive values are the GFIP_ERR_* runtime errors.
 * A negative return, or a GFIP_ERR_HANDLE / GFIP_ERR_WORKSPACE / GFIP_ERR_NULLPTR /
 * GFIP_ERR_SIZE / GFIP_ERR_ARG / GFIP_ERR_CAPTURE return, happens before anything is
 * launched: C (B for TRMM and TRSM) is unchanged.  GFIP_ERR_CUDA means a launch or copy
 * failed; a call that enqueues several kernels (pack-then-compute, TRMM, TRSM) may then
 * have enqueued the earlier ones, and the output operand is undefined.
 *
 * Quick returns (reference-BLAS rules): m == 0 or n == 0, or (alpha == 0 or k == 0) and
 * beta == 1, return 0 with nothing launched; alpha == 0 or k == 0 scales C by beta
 * without reading A or B; beta == 0 never reads C, so NaN/Inf in C do not propagate.
 *
 * Threading: a handle is used by one host thread at a time.  A workspace belongs to one
 * handle; two handles must not share one.
 */
#ifndef GEMMFIP_H
#define GEMMFIP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gfip_handle_s *gfip_handle_t;

/* Runtime error codes (positive). */
#define GFIP_OK 0
#define GFIP_ERR_HANDLE 1       /* null or destroyed handle                                */
#define GFIP_ERR_CUDA 2         /* a CUDA runtime call failed (launch, memset, query)      */
#define GFIP_ERR_WORKSPACE 3    /* no workspace set, or smaller than gfip_workspace_size() */
#define GFIP_ERR_NULLPTR 4      /* A, B or C is NULL although it would be accessed         */
#define GFIP_ERR_DEVICE 5       /* the current device is not an sm_103 GPU                 */
#define GFIP_ERR_SIZE 6         /* a dimension or leading dimension exceeds 2^31 - 1       */
#define GFIP_ERR_ARG 7          /* an invalid value for a non-BLAS argument                */
#define GFIP_ERR_SCRATCH_LIMIT 8 /* gfip_dgemm_noalloc: the problem needs more scratch than
                                    GFIP_NOALLOC_SCRATCH_BYTES                               */
#define GFIP_ERR_CAPTURE 9      /* the call would first clear control words of the workspace
                                   (the first call after gfip_set_workspace, or a call needing
                                   more control words than any before) while its stream is
                                   capturing a CUDA graph; make one such call eagerly first    */

/* Device status bits, reported by gfip_get_status(). */
#define GFIP_STATUS_BAD_SEGMENT 0x1u   /* a split tile saw more partial sums than planned */
#define GFIP_STATUS_MMA_TIMEOUT 0x2u   /* gfip_dgemm_ozaki: a pipeline wait gave up (result invalid) */
#define GFIP_STATUS_BAD_PROBLEM 0x4u   /* grouped GEMM: a problem had invalid arguments (skipped)  */
#define GFIP_STATUS_WAIT_TIMEOUT 0x8u  /* FP32 GEMM: a pipeline wait of the warp-specialised tile
                                          core gave up (result invalid)                          */

/* Pack policies for gfip_set_pack_policy(). */
#define GFIP_PACK_AUTO 0        /* Sec. 3.3 option table: pack A iff > 1 tile column, B iff > 1 tile
                                   row (whether a tile finds a k-block already packed is decided
                                   at run time, per k-block)                                        */
#define GFIP_PACK_NONE 1        /* never pack (the fused kernel then equals the direct variant)          */
#define GFIP_PACK_A 2           /* pack A panels only                                                   */
#define GFIP_PACK_B 3           /* pack B panels only                                                   */
#define GFIP_PACK_BOTH 4        /* pack both operands regardless of reuse                               */

/* Packers for gfip_set_packer(): which CTAs write the packed copies in the fused routines. */
#define GFIP_PACKER_AUTO 0      /* LINE, at every size                                       */
#define GFIP_PACKER_LINE 1      /* the first tile column packs A, the first tile row B, while
                                   computing their own tiles (Alg. 1, Sec. 3.2)                   */
#define GFIP_PACKER_SHARED 2    /* every CTA first packs an equal share of all packed tiles,
                                   k-block by k-block over the panels, then runs its tiles
                                   (the collaborative packing of Sec. 3.5).  Only for dense
                                   operands and a full C: SYRK and TRMM always use LINE      */

/* Creates a handle bound to the CURRENT CUDA device; its stream is the legacy default
 * stream until gfip_set_stream().  Returns GFIP_ERR_DEVICE if that device is not sm_103,
 * GFIP_ERR_CUDA if the device cannot be queried. */
int gfip_create(gfip_handle_t *handle);

/* Destroys a handle.  Does not free the caller's workspace.  Pending work is not waited for. */
int gfip_destroy(gfip_handle_t handle);

/* Sets the stream (a cudaStream_t passed as void*; NULL = legacy default stream) on which
 * every later call of this handle is enqueued. */
int gfip_set_stream(gfip_handle_t handle, void *stream);

/* Bytes of device workspace a call with these arguments needs on this handle
 * (elem_bytes: 8 for the d-routines, 4 for the s-routines).  The figure includes the packed
 * copies of both operands (Sec. 2.1, "packed memory"), the per-panel ready words and the
 * partial sums of split tiles.  Returns 0 for invalid arguments. */
size_t gfip_workspace_size(gfip_handle_t handle, char transa, char transb, int64_t m, int64_t n,
                           int64_t k, int elem_bytes);

/* Hands the handle a caller-owned device buffer (16-byte aligned) of `bytes` bytes.  The
 * library never allocates device memory itself.  The buffer must stay valid, and must not be
 * used by anything else, until the last call that uses it has completed on the stream.  The
 * first call after this one clears the buffer's control words (an asynchronous memset on the
 * handle's stream). */
int gfip_set_workspace(gfip_handle_t handle, void *dev_ptr, size_t bytes);

/* Chooses which operands the fused routines pack (GFIP_PACK_*); testing and tuning aid.
 * The result bits do not depend on the policy. */
int gfip_set_pack_policy(gfip_handle_t handle, int policy);

/* Chooses who packs in the fused routines (GFIP_PACKER_*); testing and tuning aid.
 * GFIP_ERR_ARG for an unknown value.  The result bits do not depend on the packer. */
int gfip_set_packer(gfip_handle_t handle, int packer);

/* Fused-in-packing GEMM (the method of Sec. 3.2), FP64 and FP32. */
int gfip_dgemm(gfip_handle_t handle, char transa, char transb, int64_t m, int64_t n, int64_t k,
               double alpha, const double *A, int64_t lda, const double *B, int64_t ldb,
               double beta, double *C, int64_t ldc);
int gfip_sgemm(gfip_handle_t handle, char transa, char transb, int64_t m, int64_t n, int64_t k,
               float alpha, const float *A, int64_t lda, const float *B, int64_t ldb,
               float beta, float *C, int64_t ldc);

/* Direct-strided comparison variant: never packs; every CTA reads the raw strided operands
 * (the SUP path of Sec. 2.3).  Needs a workspace only for split-tile partial sums. */
int gfip_dgemm_direct(gfip_handle_t handle, char transa, char transb, int64_t m, int64_t n,
                      int64_t k, double alpha, const double *A, int64_t lda, const double *B,
                      int64_t ldb, double beta, double *C, int64_t ldc);
int gfip_sgemm_direct(gfip_handle_t handle, char transa, char transb, int64_t m, int64_t n,
                      int64_t k, float alpha, const float *A, int64_t lda, const float *B,
                      int64_t ldb, float beta, float *C, int64_t ldc);

/* Pack-then-compute comparison variant: a pack kernel copies both operands into the packed
 * layout, then the GEMM kernel reads only packed tiles (the conventional path of Sec. 2.1,
 * Fig. 1).  Two launches on the handle's stream. */
int gfip_dgemm_pack_then_compute(gfip_handle_t handle, char transa, char transb, int64_t m,
                                 int64_t n, int64_t k, double alpha, const double *A,
                                 int64_t lda, const double *B, int64_t ldb, double beta,
                                 double *C, int64_t ldc);
int gfip_sgemm_pack_then_compute(gfip_handle_t handle, char transa, char transb, int64_t m,
                                 int64_t n, int64_t k, float alpha, const float *A,
                                 int64_t lda, const float *B, int64_t ldb, float beta,
                                 float *C, int64_t ldc);

/* ---- FP64 GEMM emulated on the tensor cores ------------------------------------------------
 * Extension of the method (Sec. 5 lists other precisions as future work; the slicing is a
 * pack-time transform like the 1m method of Sec. 5): C := alpha*op(A)*op(B) + beta*C in FP64,
 * computed from exact BF16 digit products on the tcgen05 tensor cores (Ozaki splitting).
 * Every row of op(A) and column of op(B) is scaled by a power of two and split into `slices`
 * 6-bit integer digits (1 <= slices <= 10); the digit pairs (s, t) with s + t <= slices + 1 are
 * multiplied on the tensor cores with exact FP32 accumulation over k-chunks of 16384, and
 * recombined in FP64.  The result is NOT the IEEE FP64 product: its error against the exact
 * product is bounded by about k * 2^(e_i + f_j) * 2^(-6*slices) * (slices + 2) * |alpha|
 * plus FP64 rounding, where 2^e_i and 2^f_j are the powers of two just above the largest
 * magnitude in row i of op(A) and column j of op(B); slices = 9 reaches FP64-level accuracy
 * for data of uniform magnitude.
 * Same argument conventions, quick returns and error codes as gfip_dgemm, plus
 * GFIP_ERR_ARG for a slice count out of range.  Needs gfip_ozaki_workspace_size() bytes of
 * workspace.  A timeout inside the kernel raises GFIP_STATUS_MMA_TIMEOUT. */
size_t gfip_ozaki_workspace_size(gfip_handle_t handle, int64_t m, int64_t n, int64_t k,
                                 int slices);
int gfip_dgemm_ozaki(gfip_handle_t handle, char transa, char transb, int64_t m, int64_t n,
                     int64_t k, double alpha, const double *A, int64_t lda, const double *B,
                     int64_t ldb, double beta, double *C, int64_t ldc, int slices);

/* ---- SYRK on the fused kernel (one of the other level-3 operations, Sec. 1 and Sec. 5) ----
 *
 * C := alpha * A * A^T + beta * C   (trans 'N', A is n x k, column-major, lda >= max(1, n))
 * C := alpha * A^T * A + beta * C   (trans 'T' or 'C', A is k x n, lda >= max(1, k))
 * on the triangle uplo ('L': entries i >= j, 'U': i <= j) of the n x n column-major C
 * (ldc >= max(1, n)); the other triangle and rows n..ldc-1 are never read or written.  The
 * same fused kernel as gfip_dgemm computes only the tiles of that triangle, with A in both
 * operand roles: the first tile line packs each panel of A once and that packed copy serves
 * as row panel and as column panel.  The pack policy of the handle applies (NONE: raw
 * reads only).  BLAS rules: beta == 0 does not read C; alpha == 0 or k == 0 does not read A
 * (C := beta C on the triangle); n == 0 or ((alpha == 0 or k == 0) and beta == 1) returns at
 * once.  Errors: -1 uplo, -2 trans, -3 n < 0, -4 k < 0, -7 lda, -10 ldc (reference-BLAS
 * positions), or a GFIP_ERR_* code.  Needs gfip_syrk_workspace_size() bytes of workspace;
 * asynchronous on the handle's stream. */
size_t gfip_syrk_workspace_size(gfip_handle_t handle, char uplo, char trans, int64_t n,
                                int64_t k, int elem_bytes);
int gfip_dsyrk(gfip_handle_t handle, char uplo, char trans, int64_t n, int64_t k, double alpha,
               const double *A, int64_t lda, double beta, double *C, int64_t ldc);
int gfip_ssyrk(gfip_handle_t handle, char uplo, char trans, int64_t n, int64_t k, float alpha,
               const float *A, int64_t lda, float beta, float *C, int64_t ldc);

/* ---- TRMM on the fused kernel (one of the other level-3 operations, Sec. 1 and Sec. 5) ----
 *
 * B := alpha * op(A) * B   (side 'L', A is m x m, lda >= max(1, m))
 * B := alpha * B * op(A)   (side 'R', A is n x n, lda >= max(1, n))
 * with B m x n column-major (ldb >= max(1, m)), op(A) = A ('N') or A^T ('T', 'C'), A
 * triangular: only its uplo triangle ('L' or 'U') is read, and with diag 'U' its diagonal is
 * not read either and taken as 1.  The product runs on the fused kernel with op(A) read
 * through a triangular mask: k-blocks outside the triangle are skipped, blocks the diagonal
 * cuts are masked as they are staged, so the first tile line packs masked panels.  It is
 * formed out of place in the workspace and copied back into B (rows m..ldb-1 untouched).
 * BLAS rules: alpha == 0 sets B to zero without reading A or B; m == 0 or n == 0 returns at
 * once.  Errors: -1 side, -2 uplo, -3 transa, -4 diag, -5 m < 0, -6 n < 0, -9 lda, -11 ldb
 * (reference-BLAS positions), or a GFIP_ERR_* code.  Needs gfip_trmm_workspace_size() bytes
 * of workspace; asynchronous on the handle's stream. */
size_t gfip_trmm_workspace_size(gfip_handle_t handle, char side, char uplo, char transa,
                                char diag, int64_t m, int64_t n, int elem_bytes);
int gfip_dtrmm(gfip_handle_t handle, char side, char uplo, char transa, char diag, int64_t m,
               int64_t n, double alpha, const double *A, int64_t lda, double *B, int64_t ldb);
int gfip_strmm(gfip_handle_t handle, char side, char uplo, char transa, char diag, int64_t m,
               int64_t n, float alpha, const float *A, int64_t lda, float *B, int64_t ldb);

/* ---- TRSM on the fused kernel (one of the other level-3 operations, Sec. 1 and Sec. 5) ----
 *
 * Solves op(A) * X = alpha * B (side 'L', A m x m) or X * op(A) = alpha * B (side 'R',
 * A n x n) and overwrites B (m x n, column-major, ldb >= max(1, m)) with X; op(A), uplo,
 * diag and lda as for gfip_dtrmm (only the uplo triangle of A is read, and not its
 * diagonal for diag 'U').  Blocked on two levels: over panels of 512 unknowns in solve
 * order, and inside a panel over its diagonal blocks of 64, a substitution kernel solves the
 * block for every right-hand side and one fused GEMM (alpha -1, beta 1) removes its
 * contribution from the panel's unknowns still to be solved; after each panel one fused GEMM
 * removes the panel's contribution from all other unknowns still to be solved.
 * No singularity test is made (as in the reference BLAS): a zero on a non-unit diagonal
 * gives Inf or NaN.  BLAS rules: alpha == 0 sets B to zero without reading A or B; m == 0
 * or n == 0 returns at once.  Errors as gfip_dtrmm.  Needs gfip_trsm_workspace_size() bytes
 * of workspace; asynchronous on the handle's stream (many launches, no host read-back). */
size_t gfip_trsm_workspace_size(gfip_handle_t handle, char side, char uplo, char transa,
                                char diag, int64_t m, int64_t n, int elem_bytes);
int gfip_dtrsm(gfip_handle_t handle, char side, char uplo, char transa, char diag, int64_t m,
               int64_t n, double alpha, const double *A, int64_t lda, double *B, int64_t ldb);
int gfip_strsm(gfip_handle_t handle, char side, char uplo, char transa, char diag, int64_t m,
               int64_t n, float alpha, const float *A, int64_t lda, float *B, int64_t ldb);

/* ---- Grouped GEMM: many independent problems of uneven sizes in one launch ----------------
 * The size-unified code path of Sec. 1 and Sec. 3 applied to a batch: for g < count,
 *     C_g := alpha[g] * op(A_g) * op(B_g) + beta[g] * C_g
 * with per-problem transa[g], transb[g] ('N','T','C'), m[g], n[g], k[g], leading dimensions and
 * matrix pointers.  EVERY array argument is a DEVICE array of `count` entries (the pointer
 * arrays hold device pointers), so the call reads nothing on the host and can be captured in
 * a CUDA graph (after one eager call on the handle's workspace, see GFIP_ERR_CAPTURE): it
 * enqueues a preparation kernel, a prefix-sum kernel and one persistent GEMM kernel on the
 * handle's stream.  The unit of work is one warp computing one small tile of one problem, so
 * one launch runs problems of different tile shapes side by side.  Each problem follows the
 * reference-BLAS rules of gfip_dgemm; a problem with invalid arguments is skipped (its C
 * untouched) and raises GFIP_STATUS_BAD_PROBLEM.
 *
 * gfip_?gemm_grouped: every problem takes the warp tile `tile` (GFIP_GROUP_TILE_*), unsplit.
 * Needs gfip_grouped_workspace_size() bytes of workspace.  GFIP_ERR_ARG for count < 0 or an
 * unknown tile.
 *
 * gfip_?gemm_grouped_plan: problem g takes plan[g] = GFIP_GROUP_PLAN(tile, splits) (a device
 * array): its warp tile, and the number of k-ranges (1..8) each of its tiles is split into,
 * computed by different warps and added in k-range order by the last to finish (the result
 * bits depend on the plan, never on timing).  `order` (a device array, or NULL for 0..count-1)
 * is the processing order of the problems; warps are dealt the work units in bands of all
 * warps, alternately forwards and backwards, so an order with the costliest units first
 * (the Python Plan's: units' k-chunks weighted by tile area) ends the warps together.  split_elems is the number of
 * partial-sum elements the plan needs (the sum over split problems of tiles x splits x tile
 * area); the workspace must hold gfip_grouped_plan_workspace_size(count, split_elems) bytes,
 * and a problem whose partial sums would not fit runs unsplit.  The plan is chosen per size
 * bucket by the Python autotuner (grouped.autotune_plan). */
#define GFIP_GROUP_TILE_DEFAULT 0   /* warp tile 32 x 32                                        */
#define GFIP_GROUP_TILE_SMALL 1     /* warp tile 32 x 16                                        */
#define GFIP_GROUP_TILE_TINY 2      /* warp tile 16 x 16                                        */
#define GFIP_GROUP_TILE_16X8 3      /* warp tile 16 x 8                                         */
#define GFIP_GROUP_TILE_8X16 4      /* warp tile 8 x 16                                         */
#define GFIP_GROUP_PLAN(tile, splits) ((tile) | ((splits) << 8))
size_t gfip_grouped_workspace_size(gfip_handle_t handle, int count);
size_t gfip_grouped_plan_workspace_size(gfip_handle_t handle, int count, int64_t split_elems,
                                        int elem_bytes);
int gfip_dgemm_grouped(gfip_handle_t handle, int count, const char *transa, const char *transb,
                       const int *m, const int *n, const int *k, const double *alpha,
                       const double *const *A, const int64_t *lda, const double *const *B,
                       const int64_t *ldb, const double *beta, double *const *C,
                       const int64_t *ldc, int tile);
int gfip_sgemm_grouped(gfip_handle_t handle, int count, const char *transa, const char *transb,
                       const int *m, const int *n, const int *k, const float *alpha,
                       const float *const *A, const int64_t *lda, const float *const *B,
                       const int64_t *ldb, const float *beta, float *const *C,
                       const int64_t *ldc, int tile);
int gfip_dgemm_grouped_plan(gfip_handle_t handle, int count, const char *transa,
                            const char *transb, const int *m, const int *n, const int *k,
                            const double *alpha, const double *const *A, const int64_t *lda,
                            const double *const *B, const int64_t *ldb, const double *beta,
                            double *const *C, const int64_t *ldc, const int *plan,
                            const int *order, int64_t split_elems);
int gfip_sgemm_grouped_plan(gfip_handle_t handle, int count, const char *transa,
                            const char *transb, const int *m, const int *n, const int *k,
                            const float *alpha, const float *const *A, const int64_t *lda,
                            const float *const *B, const int64_t *ldb, const float *beta,
                            float *const *C, const int64_t *ldc, const int *plan,
                            const int *order, int64_t split_elems);

/* Waits for the handle's stream, then returns the OR of the device status bits
 * (GFIP_STATUS_*) raised since the previous call of this function, and clears them.
 * Needs a workspace. */
int gfip_get_status(gfip_handle_t handle, uint32_t *status);

/* Number of kernel launches the most recent GEMM call of this handle enqueued (0 for a quick
 * return), and the grid size of its GEMM kernel. */
int gfip_last_launch_info(gfip_handle_t handle, int *launches, int *grid);

/* Static description of a return code. */
const char *gfip_error_string(int code);

/* ---- Allocation-free entry point ----------------------------------------------------------
 * The paper has no counterpart to this routine; it exists for callers that cannot allocate
 * device memory or hand the library a workspace: code behind the plain BLAS dgemm interface
 * (which has no workspace argument), applications that own every byte of device memory
 * through their own pool, and code running where cudaMalloc is not allowed.
 *
 * gfip_dgemm_noalloc computes exactly what gfip_dgemm computes (the fused-in-packing FP64
 * GEMM, same kernel, same result bits), with the reference-BLAS argument list plus a stream
 * (a cudaStream_t passed as void*; NULL = legacy default stream).  It takes no handle and
 * allocates nothing: its scratch memory (packed panels, ready words, split-tile partial sums)
 * is one statically sized device array of GFIP_NOALLOC_SCRATCH_BYTES bytes inside this
 * library, which every GPU that loads the library holds until the process exits.
 *
 * A problem whose scratch would exceed that size is rejected with GFIP_ERR_SCRATCH_LIMIT
 * before anything is launched (square FP64 problems up to about m = n = k = 1600 fit; any
 * size fits the handle-based routines).  The first call on a device sets the array up: it
 * looks up the array's device address and clears its control words with an asynchronous
 * memset on the given stream, so make that first call before any stream capture (a call
 * that has to clear control words while its stream is capturing returns GFIP_ERR_CAPTURE
 * and enqueues nothing).  Every call looks the address up again, so after the device's
 * context is destroyed and created again (cudaDeviceReset) the next call starts over.
 *
 * All calls on a device share the one array, and it keeps the last call's contents (each call
 * tags its control words, so stale contents are never mistaken for its own).  Calls that can
 * overlap on the GPU -- on different streams, or from several host threads without ordering
 * -- race on the array and give wrong results; order them on one stream. */
#define GFIP_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)

int gfip_dgemm_noalloc(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                       const double *A, int64_t lda, const double *B, int64_t ldb, double beta,
                       double *C, int64_t ldc, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GEMMFIP_H */
