// gfip_internal.h -- host/device shared definitions of the fused-in-packing GEMM library.
// Not part of the public ABI (that is include/gemmfip.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gfip {

// Where an operand's tiles come from in one launch of the GEMM kernel.
// Part of C a launch computes: all of it (GEMM), or one triangle of a square C (SYRK).
enum Triangle : int { TRI_NONE = 0, TRI_LOWER = 1, TRI_UPPER = 2 };

// Triangular operand (TRMM): element (x, k) of op(X) (x = row of op(A) or column of op(B),
// k = the summed index) is kept when x - k >= s (KEEP_GE) or k - x >= s, s = 1 for a strictly
// triangular operand (a unit diagonal is added separately), else s = 0; the rest is zero.
enum TriMask : int { TMASK_ON = 1, TMASK_KEEP_GE = 2, TMASK_STRICT = 4 };

enum OperandMode : int {
    MODE_RAW = 0,     // always read the raw strided operand (direct variant, SUP analog)
    MODE_PACKED = 1,  // always read the packed copy, written beforehand by the pack kernel
    MODE_FIP = 2,     // fused: the first tile line packs each (panel, k-block) while
                      // computing with it, later tiles read the packed copy once it is
                      // published (Sec. 3.1 Alg. 1, Sec. 3.2)
};

// Tile shape of one element type.  The CTA computes a BM x BN tile of C, stepping through
// k in blocks of BK; each thread owns an (NCM*CH) x (NCN*CH) register micro-tile (CH =
// elements per 16 bytes).
template <typename T> struct TileCfg;

// FP64: the DFMA pipe (2 lanes per clock per SM) is the bound at every size, so small tiles
// cost no throughput and give fine-grained work units that keep all SMs busy.
#ifndef GFIP_F64_BM
#define GFIP_F64_BM 32
#endif
#ifndef GFIP_F64_BN
#define GFIP_F64_BN 32
#endif
#ifndef GFIP_F64_MIN_BLOCKS
#define GFIP_F64_MIN_BLOCKS 6
#endif
#ifndef GFIP_F64_UNROLL
#define GFIP_F64_UNROLL 2
#endif
// A CTA runs at least 4 warps, one per SM sub-partition (each has its own FP64 unit), with
// 4 x 2 micro-tiles for tiles of up to 1024 elements and 4 x 4 above.
template <> struct TileCfg<double> {
    static constexpr int BM = GFIP_F64_BM, BN = GFIP_F64_BN, BK = 16;
    static constexpr int NCM = 2;
    static constexpr int NCN = (BM * BN / 128 >= 16) ? 2 : 1;       // 4 x 4 or 4 x 2 per thread
    static constexpr int THREADS = BM * BN / (4 * 2 * NCN) < 128 ? 128 : BM * BN / (4 * 2 * NCN);
    static constexpr int STAGES = 3;
    static constexpr int MIN_BLOCKS = GFIP_F64_MIN_BLOCKS;
    static constexpr int UNROLL = GFIP_F64_UNROLL;  // k rows per unrolled compute step
};
#ifndef GFIP_F32_MIN_BLOCKS
#define GFIP_F32_MIN_BLOCKS 2
#endif
#ifndef GFIP_F32_STAGES
#define GFIP_F32_STAGES 3
#endif
#ifndef GFIP_F32_BK
#define GFIP_F32_BK 32
#endif
#ifndef GFIP_F32_NCM
#define GFIP_F32_NCM 2
#endif

// FP32: 128 x 128 tiles, 8 x 8 per thread on 256 threads (NCM = NCN = 2 chunks of 4).
// Shared memory delivers 128 bytes per clock per SM and the FFMA pipe 128 lanes, so an 8 x 8
// micro-tile, reading (8 + 8) x 4 bytes per 64 FMAs, sits at the shared-memory limit; 16 x 8
// (NCM = 4, 128 threads) reads 0.75 B/FMA and measured 4 % faster at 8192 but 5-10 % slower
// at 1024-2048, where only 8 warps per SM are left to hide latency.
#ifndef GFIP_F32_UNROLL
#define GFIP_F32_UNROLL 16
#endif
template <> struct TileCfg<float> {
    static constexpr int BM = 128, BN = 128, BK = GFIP_F32_BK, NCM = GFIP_F32_NCM, NCN = 2;
    static constexpr int THREADS = BM * BN / (NCM * 4 * NCN * 4);
    static constexpr int UNROLL = GFIP_F32_UNROLL;
    static constexpr int STAGES = GFIP_F32_STAGES, MIN_BLOCKS = GFIP_F32_MIN_BLOCKS;
};

// Everything one launch of the GEMM kernel needs.  Plain data, passed by value.
template <typename T> struct GemmParams {
    const T *A;
    const T *B;
    T *C;
    int64_t lda, ldb, ldc;
    int m, n, k;
    T alpha, beta;
    int a_contig_m;   // 1: op(A)[i,p] = A[i + p*lda] (transa 'N'); 0: A[p + i*lda]
    int b_contig_n;   // 1: op(B)[p,j] = B[j + p*ldb] (transb 'T'); 0: B[p + j*ldb]
    int mt, nt, kt;   // tile counts along m, n and k
    int tiles;        // mt * nt
    int band;         // tile rows per band of the consumer tile order (>= 1)
    int tri;          // TRI_NONE: all of C; TRI_LOWER / TRI_UPPER: that triangle (SYRK)
    int a_produces;   // the first tile column packs the A panels
    int b_produces;   // the first tile row packs the B panels
    int shared_pack;  // all CTAs pack the packed operands' tiles first (no line producers)
    int64_t pack_units;  // shared packing: (panel, k-block) tiles to pack in all
    int tmask_a;      // triangular mask of op(A) (TRMM), 0 = dense; see TriMask
    int tmask_b;      // triangular mask of op(B)
    int grid;         // persistent CTAs
    int dp_tiles;     // tiles [0, dp_tiles) are data-parallel, taken in order from tile_next
    int64_t sk_iters; // (tiles - dp_tiles) * kt iterations split evenly over the CTAs
    int mode_a, mode_b;
    unsigned long long *state_a;     // [mt * kt] epoch-tagged ready words of packed A tiles,
                                     // then [mt] words "whole panel published"
    unsigned long long *state_b;     // [nt * kt + nt] same for B
    unsigned long long *tile_count;  // [tiles] epoch-tagged arrival counters of split tiles
    T *pack_a;                       // [mt * kt] tiles of BM * BK elements
    T *pack_b;                       // [nt * kt] tiles of BN * BK elements
    T *partial;                      // [grid * 2] slots of BM * BN elements
    unsigned int *status;            // device status bits (GFIP_STATUS_*)
    unsigned int *launch_count;      // launches so far (the epoch of a launch is this + 1)
    unsigned int *done_count;        // CTAs of the current launch that have finished
    unsigned long long *pack_count;  // shared packing: epoch-tagged count of packed tiles
    unsigned long long *tile_next;   // epoch-tagged count of data-parallel tiles taken
};

// Parameters of the pack kernel of the pack-then-compute variant.
template <typename T> struct PackParams {
    const T *A;
    const T *B;
    int64_t lda, ldb;
    int m, n, k;
    int a_contig_m, b_contig_n;
    int mt, nt, kt;
    T *pack_a;
    T *pack_b;
};

// FP64 GEMM emulated with BF16 digit products on the tensor cores (gfip_ozaki.cu).
struct OzakiParams {
    const double *A;
    const double *B;
    double *C;
    int64_t lda, ldb, ldc;
    int m, n, k;
    double alpha, beta;
    int a_contig_rows;   // 1: row i of op(A) runs along memory (transa 'N')
    int b_contig_rows;   // 1: column j of op(B) = row j of its K-major form runs along memory ('T')
    int slices;          // digits per element (S)
    int mt, nt, kt;      // 128-row blocks of m and n, 64-wide k blocks
    int ks_a, ks_b;      // k-ranges the exponent reductions are split into
    int *ea;             // [ks_a][mt * 128] partial row exponents of op(A)
    int *eb;             // [ks_b][nt * 128] partial column exponents of op(B)
    uint16_t *sa;        // [S][mt][kt] digit tiles of op(A), 16 KB each
    uint16_t *sb;        // [S][nt][kt] digit tiles of op(B)
    unsigned int *status;
    unsigned long long wait_ns;  // budget of every mbarrier wait (nanoseconds)
    int inject_timeout;  // test hook: CTA 0 withholds its first operand copy
};
cudaError_t launch_ozaki(const OzakiParams &p, cudaStream_t s);
size_t ozaki_smem_bytes();

// Triangular solve (gfip_trsm.cu): one launch solves a panel of at most TRSM_PANEL unknowns
// (op(A)'s diagonal block at (k0, k0), transposed for side 'R') for every right-hand side;
// vector v's element i is B[v*vstride + i*estride].
constexpr int TRSM_PANEL = 512;
template <typename T>
cudaError_t launch_trsm_panel(T *B, int64_t vstride, int64_t estride, int nvec, const T *A,
                              int64_t lda, int a_trans, int k0, int pw, int lower_t,
                              int transpose_t, int unit, cudaStream_t s);

// Grouped GEMM (gfip_grouped.cu): many independent problems in one persistent launch, each
// problem with its own warp-tile shape and k-split factor.
template <typename T> struct GroupDesc;
template <typename T> struct GroupParams;
template <typename T> cudaError_t launch_grouped(const GroupParams<T> &gp, cudaStream_t s);
// Bytes of one grouped launch's descriptor arrays for `count` problems (element size es).
size_t grouped_desc_bytes(int count, int es);

// Launchers (defined per element type in gfip_f64.cu / gfip_f32.cu).
template <typename T> cudaError_t launch_gemm(const GemmParams<T> &p, cudaStream_t s);
template <typename T> cudaError_t launch_pack(const PackParams<T> &p, cudaStream_t s);
template <typename T>
cudaError_t launch_scale(T *C, int64_t ldc, int m, int n, T beta, int tri, cudaStream_t s);
// CTAs of the GEMM kernel that fit on one SM at once.
template <typename T> int gemm_blocks_per_sm();
// The warp-specialised FP32 tile core (gfip_f32_ws.cu): dense FP32 GEMMs over the whole of C
// (no triangle, no triangular operand) with line producers or no packing.
cudaError_t launch_ws_gemm(const GemmParams<float> &p, cudaStream_t s);
// Its pack kernel (pack-then-compute): packed tiles in the swizzled layout it reads.
cudaError_t launch_ws_pack(const PackParams<float> &p, cudaStream_t s);
int ws_blocks_per_sm();

}  // namespace gfip
