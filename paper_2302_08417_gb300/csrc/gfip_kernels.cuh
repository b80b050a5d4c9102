// gfip_kernels.cuh -- device code of the fused-in-packing GEMM (templated on FP64/FP32).
//
// One persistent kernel computes C := alpha*op(A)*op(B) + beta*C for column-major strided
// operands.  Three properties carry the paper's method onto the GPU:
//
//  * Packed layout = shared-memory image (Sec. 2.1, Fig. 2).  An operand tile (BX x BK of
//    op(A) or op(B)) is cut into 128-byte row segments along x, one row per k.  In shared
//    memory the rows sit at a pitch of 128 bytes plus 4 elements (bank-conflict-free raw loads
//    and fragment reads); the packed copy in global memory holds the same rows back to back,
//    so a CTA fetches a packed tile with contiguous 16-byte copies and no per-element address
//    arithmetic, and fringes are zero-padded once, when packing (Sec. 2.2).
//
//  * Fused-in packing (Sec. 3.1 Alg. 1, Sec. 3.2).  Tiles are ordered producers first: the
//    tiles of the first tile column come first and pack the A panels, then the rest of the
//    first tile row, which pack the B panels.  A producer reads its raw strided operand
//    k-block by k-block, computes with it, and in the same pass writes the staged tile image
//    to the packed buffer and publishes it (an epoch-tagged ready word, release order).  Every
//    other tile looks the ready word up (acquire load) a few k-blocks ahead: published tiles
//    are read packed, the rest raw.  Nothing ever waits for another CTA (the multithreaded
//    scheme of Sec. 3.5 synchronises once after a collaborative pack; here only tiles that
//    run after a producer use what it packed).
//
//  * One code path for all sizes.  Tiles run as data-parallel waves over the persistent
//    CTAs; the tiles of the last, partial wave (with one full wave more when the partial one
//    would give each CTA a short run) are split evenly along k over all CTAs ("stream-K"), and split tiles are summed in a fixed order by whichever CTA
//    finishes last.  The split points depend only on the problem shape and the grid, so every
//    variant (fused, direct, pack-then-compute) and every pack policy produces identical
//    bits: packing changes where a tile is read from, never its value.
#pragma once

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "gfip_internal.h"

namespace gfip {

constexpr unsigned int STATUS_BAD_SEGMENT = 0x1u;  // mirrors GFIP_STATUS_BAD_SEGMENT

enum Decision : int { DEC_RAW = 0, DEC_PACKED = 1, DEC_PRODUCE = 2, DEC_SKIP = 3 };

__device__ __forceinline__ bool tmask_keep(int mask, int x, int k)
{
    const int s = (mask & TMASK_STRICT) ? 1 : 0;
    return (mask & TMASK_KEEP_GE) ? (x - k >= s) : (k - x >= s);
}

// A BX x BK operand block at (x0, k0) under a mask: 0 all kept, 1 partly kept, 2 all zero.
__device__ __forceinline__ int tmask_class(int mask, int x0, int bx, int k0, int bk)
{
    if (!(mask & TMASK_ON)) return 0;
    const int s = (mask & TMASK_STRICT) ? 1 : 0;
    const int lo = (mask & TMASK_KEEP_GE) ? x0 - (k0 + bk - 1) : k0 - (x0 + bx - 1);
    const int hi = (mask & TMASK_KEEP_GE) ? (x0 + bx - 1) - k0 : (k0 + bk - 1) - x0;
    if (lo >= s) return 0;
    if (hi < s) return 2;
    return 1;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Element copy global -> shared through L1, zero-filling the destination when !ok (no
// bytes are read from src then).
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(uint32_t dst, const void *src, bool ok)
{
    const int src_bytes = ok ? BYTES : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(dst), "l"(src),
                 "n"(BYTES), "r"(src_bytes)
                 : "memory");
}

// 16-byte copy global -> shared bypassing L1 (packed tiles are written by other SMs).
__device__ __forceinline__ void cp_async_16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int N> __device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Layout of one BX x BK operand tile (x runs along m for A, along n for B; kk along k).
// The tile is cut into BX/W segments of W = 128/sizeof(T) consecutive x; a segment holds BK
// rows (one per kk) of W elements, i.e. 128 bytes.
//  * Packed copy in global memory: the rows back to back, row r = (x / W) * BK + kk
//    (ROWS rows, no padding), so a packed tile is one contiguous block of 16-byte chunks.
//  * Shared memory: the same rows with a pitch of P = W + PADE elements.  The padding moves
//    consecutive rows across banks, so the raw loads that write 8 consecutive kk of 4
//    consecutive x in one warp instruction are bank-conflict free, and a compute-loop
//    fragment is the address base + kk * P (an immediate offset).
template <typename T, int BX, int BK> struct TileLayout {
    static constexpr int W = 128 / static_cast<int>(sizeof(T));
    static constexpr int PADE = 4;                // 4 floats (16 B) or 4 doubles (32 B)
    static constexpr int P = W + PADE;            // shared-memory row pitch, elements
    static constexpr int SEG = BK * P;            // shared-memory segment pitch, elements
    static constexpr int ELEMS = (BX / W) * SEG;  // shared-memory elements per tile
    static constexpr int ROWS = (BX / W) * BK;    // 128-byte rows per tile
    static constexpr int PACKED = BX * BK;        // packed elements per tile
    static_assert(BX % W == 0, "tile must be whole 128-byte segments");
    static_assert((P * sizeof(T)) % 16 == 0, "rows must stay 16-byte aligned");
    static __device__ __forceinline__ int off(int x, int kk)
    {
        return (x / W) * SEG + kk * P + (x % W);
    }
};

// Raw strided loads of one operand's BX x BK tiles, k-block after k-block.  Element (x, kk)
// of the tile at (x0, k0) of op(X) sits at g[(x0+x) + (k0+kk)*ld] when CONTIG (x runs along
// memory) and at g[(k0+kk) + (x0+x)*ld] otherwise.  Each thread owns PER fixed elements of
// the tile; their addresses differ from one base pointer by per-element constants, so a
// k-block costs one pointer increment plus one copy per element.  Out-of-range elements are
// zero-filled (the fringe padding of Sec. 2.2).
//   CONTIG: x = tid % BX, kk = tid / BX + r * (THREADS / BX): a warp reads 32 consecutive x.
//   else:   a warp covers blocks of 4 consecutive x by 8 consecutive k (four runs of 8
//           contiguous elements); block b = warp + r * NW (NW warps) sits at
//           x = 4 * (b % XB) + lane/8, kk = 8 * (b / XB) + lane%8 with XB = BX/4.  Because NW
//           divides XB, element r is element 0 shifted by the constants DX(r), DK(r).
template <typename T, int BX, int BK, int THREADS, bool CONTIG> struct RawLoader {
    using L = TileLayout<T, BX, BK>;
    static constexpr int PER = BX * BK / THREADS;
    static constexpr int NW = THREADS / 32;
    static constexpr int XB = BX / 4;
    static_assert(PER * THREADS == BX * BK, "tile must divide over the threads");
    static_assert(!CONTIG || THREADS % BX == 0, "contiguous pattern needs THREADS % BX == 0");
    static_assert(CONTIG || (XB % NW == 0 && BK % 8 == 0 && PER * NW == XB * (BK / 8)),
                  "transposed pattern needs the warps to divide the x blocks");
    static_assert(L::W % (4 * NW) == 0 || (4 * NW) % L::W == 0,
                  "a warp's x span and a 128-byte segment must nest");
    static constexpr int NG = XB / NW;  // distinct x offsets: element r is in x group GX(r)
    static __device__ __forceinline__ constexpr int GX(int r) { return ((r * NW) % XB) / NW; }
    static __device__ __forceinline__ constexpr int DX(int r) { return 4 * NW * GX(r); }
    static __device__ __forceinline__ constexpr int DK(int r) { return 8 * ((r * NW) / XB); }

    const T *g;       // operand base (a valid address for zero-filled copies)
    const T *p;       // this thread's element 0 at the next k-block to issue
    int64_t ld;
    int xg;           // global x of element 0 (for triangular masks)
    uint32_t xok;     // bit GX(r): x of element r lies inside the operand (CONTIG: bit 0 only)
    int kk0;          // kk of element 0
    uint32_t s0;      // shared-memory byte offset (within a stage) of element 0

    __device__ __forceinline__ void init(const T *g_, int64_t ld_, int x0, int k0, int x_ext,
                                         int tid)
    {
        g = g_;
        ld = ld_;
        if (CONTIG) {
            const int x = tid % BX;
            kk0 = tid / BX;
            xg = x0 + x;
            p = g + (int64_t)(x0 + x) + (int64_t)(k0 + kk0) * ld;
            xok = (x0 + x < x_ext) ? 1u : 0u;
            s0 = 0;
        } else {
            const int lane = tid & 31, w = tid >> 5;
            const int x = 4 * w + (lane >> 3);
            kk0 = lane & 7;
            xg = x0 + x;
            p = g + (int64_t)(k0 + kk0) + (int64_t)(x0 + x) * ld;
            xok = 0;
#pragma unroll
            for (int gx = 0; gx < NG; ++gx)
                if (x0 + x + 4 * NW * gx < x_ext) xok |= 1u << gx;
            s0 = L::off(x, kk0) * sizeof(T);
        }
    }

    // Copies the next k-block's tile (kleft = rows of k still inside the operand) into the
    // stage at byte address sdst, then advances to the following k-block.
    __device__ __forceinline__ void issue(uint32_t sdst, int kleft, int tid)
    {
        if (CONTIG) {
            const int x = tid % BX;
#pragma unroll
            for (int r = 0; r < PER; ++r) {
                const int kk = kk0 + r * (THREADS / BX);
                const bool ok = xok && (kk < kleft);
                const T *src = ok ? p + (int64_t)(r * (THREADS / BX)) * ld : g;
                cp_async_elem<sizeof(T)>(sdst + L::off(x, kk) * sizeof(T), src, ok);
            }
            p += (int64_t)BK * ld;
        } else {
#pragma unroll
            for (int r = 0; r < PER; ++r) {
                const bool ok = ((xok >> GX(r)) & 1u) && (kk0 + DK(r) < kleft);
                const T *src = ok ? p + (int64_t)DX(r) * ld + DK(r) : g;
                // x and x + DX(r) lie in the same 128-byte column position when DX(r) is a
                // multiple of W, or DX(r) < W apart in the same segment: either way the
                // layout offset moves by a constant
                const uint32_t soff =
                    s0 + ((DX(r) / L::W) * L::SEG + (DX(r) % L::W) + DK(r) * L::P) * sizeof(T);
                cp_async_elem<sizeof(T)>(sdst + soff, src, ok);
            }
            p += BK;
        }
    }

    // issue() for a block that a triangular mask cuts: elements outside the triangle are
    // zero-filled, not read (kstart = k of the block's first row).
    __device__ __forceinline__ void issue_masked(uint32_t sdst, int kleft, int kstart, int mask,
                                                 int tid)
    {
        if (CONTIG) {
            const int x = tid % BX;
#pragma unroll
            for (int r = 0; r < PER; ++r) {
                const int kk = kk0 + r * (THREADS / BX);
                const bool ok = xok && (kk < kleft) && tmask_keep(mask, xg, kstart + kk);
                const T *src = ok ? p + (int64_t)(r * (THREADS / BX)) * ld : g;
                cp_async_elem<sizeof(T)>(sdst + L::off(x, kk) * sizeof(T), src, ok);
            }
            p += (int64_t)BK * ld;
        } else {
#pragma unroll
            for (int r = 0; r < PER; ++r) {
                const bool ok = ((xok >> GX(r)) & 1u) && (kk0 + DK(r) < kleft) &&
                                tmask_keep(mask, xg + DX(r), kstart + kk0 + DK(r));
                const T *src = ok ? p + (int64_t)DX(r) * ld + DK(r) : g;
                const uint32_t soff =
                    s0 + ((DX(r) / L::W) * L::SEG + (DX(r) % L::W) + DK(r) * L::P) * sizeof(T);
                cp_async_elem<sizeof(T)>(sdst + soff, src, ok);
            }
            p += BK;
        }
    }

    __device__ __forceinline__ void skip()
    {
        p += CONTIG ? (int64_t)BK * ld : (int64_t)BK;
    }
};

// Packed tile load: 16-byte chunk c of the packed tile goes to row c/8, bytes (c%8)*16 of
// the padded shared-memory tile.
template <typename T, int BX, int BK, int THREADS>
__device__ __forceinline__ void load_packed_tile(uint32_t sdst, const T *src, int tid)
{
    using L = TileLayout<T, BX, BK>;
    constexpr int CHUNKS = L::ROWS * 8;
    constexpr int PB = L::P * static_cast<int>(sizeof(T));
    const char *s = reinterpret_cast<const char *>(src);
#pragma unroll
    for (int c = tid; c < CHUNKS; c += THREADS)
        cp_async_16(sdst + (c >> 3) * PB + (c & 7) * 16, s + c * 16);
}

// Writes a staged tile to its packed slot (the fused pack store): the inverse mapping.
template <typename T, int BX, int BK, int THREADS>
__device__ __forceinline__ void store_packed_tile(T *dst, const T *stile, int tid)
{
    using L = TileLayout<T, BX, BK>;
    constexpr int CHUNKS = L::ROWS * 8;
    constexpr int PB = L::P * static_cast<int>(sizeof(T));
    const char *s = reinterpret_cast<const char *>(stile);
    uint4 *d = reinterpret_cast<uint4 *>(dst);
#pragma unroll
    for (int c = tid; c < CHUNKS; c += THREADS)
        __stcg(d + c, *reinterpret_cast<const uint4 *>(s + (c >> 3) * PB + (c & 7) * 16));
}

// Relaxed read of a ready word; pair a "published" result with fence_acquire() before the
// packed data is read (the acquire pattern of the PTX memory model).  Split from the fence so
// the load's latency overlaps a k-block of compute.
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *word)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];\n" : "=l"(v) : "l"(word) : "memory");
    return v;
}

__device__ __forceinline__ void fence_acquire()
{
    asm volatile("fence.acq_rel.gpu;\n" ::: "memory");
}

__device__ __forceinline__ unsigned long long ready_value(unsigned int epoch)
{
    return (static_cast<unsigned long long>(epoch) << 32) | 1ull;
}

// Publishes a packed tile.  Called by thread 0 after a CTA barrier that follows every
// thread's pack stores of that tile: the release store is cumulative, so the stores the
// barrier ordered before it are visible to any thread that acquires the word.
__device__ __forceinline__ void publish(unsigned long long *word, unsigned int epoch)
{
    const unsigned long long v = (static_cast<unsigned long long>(epoch) << 32) | 1ull;
    asm volatile("st.release.gpu.global.u64 [%0], %1;\n" ::"l"(word), "l"(v) : "memory");
}

// Tile order, producers first: t < mt are (t, 0) (first tile column, packs A), the next
// nt - 1 are (0, j) (rest of the first tile row, packs B), then the (mt-1) x (nt-1) others
// in bands of `band` tile rows, column-major within a band.  A wave of G concurrent tiles then
// spans about band A panels and G / band B panels (band ~ sqrt(G)), which stay in L2 while
// the wave runs, instead of every A panel of the matrix.
__device__ __forceinline__ void tile_coords(int t, int mt, int nt, int band, int &i, int &j)
{
    if (t < mt) {
        i = t;
        j = 0;
        return;
    }
    t -= mt;
    if (t < nt - 1) {
        i = 0;
        j = t + 1;
        return;
    }
    t -= nt - 1;
    const int rows = mt - 1, cols = nt - 1;
    const int b = t / (band * cols);          // band index
    const int h = min(band, rows - b * band);  // rows in this band (the last may be short)
    const int r = t - b * band * cols;
    i = 1 + b * band + r % h;
    j = 1 + r / h;
}


// Tile order of a triangle of a square tile grid (mt x mt), producers first: the first tile
// column (t < mt: (t, 0)), then the other tiles (i, j), 1 <= j <= i, column by column.  The
// upper triangle is the transpose: (j, i), whose first tile row holds the producers.
__device__ __forceinline__ void tri_coords(int t, int mt, int tri, int &i, int &j)
{
    int a, b;
    if (t < mt) {
        a = t;
        b = 0;
    } else {
        t -= mt;
        b = 1;
        while (t >= mt - b) {   // column b holds rows b .. mt-1
            t -= mt - b;
            ++b;
        }
        a = b + t;
    }
    if (tri == TRI_UPPER) {
        i = b;
        j = a;
    } else {
        i = a;
        j = b;
    }
}

// The (i, j) of tile t in the launch's order.
template <typename P> __device__ __forceinline__ void tile_of(const P &p, int t, int &i, int &j)
{
    if (p.tri != TRI_NONE)
        tri_coords(t, p.mt, p.tri, i, j);
    else
        tile_coords(t, p.mt, p.nt, p.band, i, j);
}

// Position of tile (i, j) in the launch's tile order of a whole C (inverse of tile_coords).
__device__ __forceinline__ int tile_index(int i, int j, int mt, int nt, int band)
{
    if (j == 0) return i;
    if (i == 0) return mt + j - 1;
    const int rows = mt - 1, cols = nt - 1;
    const int b = (i - 1) / band;
    const int h = min(band, rows - b * band);
    return mt + nt - 1 + b * band * cols + (j - 1) * h + (i - 1 - b * band);
}

// Round in which tile t starts: its data-parallel wave, or, for the k-split tiles, the round
// after the data-parallel waves (their segments run side by side).
template <typename P> __device__ __forceinline__ int tile_round(const P &p, int t)
{
    return min(t, p.dp_tiles) / p.grid;
}

// The run-time reuse logic of the unified method (Sec. 3.3's table, which the paper's
// conclusion has a runtime logic apply per micropanel), read in time for a GPU: a packed copy
// of a panel is only ever read by tiles that start after its producer has published it, so a
// panel is worth packing iff its last consumer tile starts in a later round than its producer
// (A panel i: producer (i, 0), consumers (i, j >= 1); B panel j: producer (0, j), consumers
// (i >= 1, j)).  Tiles of one round run side by side and read the raw operand.  Small problems
// (one round) thus pack nothing, large ones every panel, and the code path is the same.  A
// triangle (SYRK) and shared packing pack every panel the table allows.
template <typename P> __device__ __forceinline__ bool reused_a(const P &p, int i)
{
    if (p.tri != TRI_NONE || p.shared_pack) return true;
    if (p.dp_tiles == 0) return false;   // every tile is split: all run in round 0
    return p.nt > 1 && tile_round(p, tile_index(i, p.nt - 1, p.mt, p.nt, p.band)) >
                           tile_round(p, tile_index(i, 0, p.mt, p.nt, p.band));
}
template <typename P> __device__ __forceinline__ bool reused_b(const P &p, int j)
{
    if (p.tri != TRI_NONE || p.shared_pack) return true;
    if (p.dp_tiles == 0) return false;   // every tile is split: all run in round 0
    return p.mt > 1 && tile_round(p, tile_index(p.mt - 1, j, p.mt, p.nt, p.band)) >
                           tile_round(p, tile_index(0, j, p.mt, p.nt, p.band));
}

template <typename T, typename C = TileCfg<T>> struct GemmSmem {
    using Cfg = C;
    T a[Cfg::STAGES][TileLayout<T, Cfg::BM, Cfg::BK>::ELEMS];
    T b[Cfg::STAGES][TileLayout<T, Cfg::BN, Cfg::BK>::ELEMS];
    int dec_a[4 * Cfg::STAGES];
    int dec_b[4 * Cfg::STAGES];
    int part[4 * Cfg::STAGES];   // bit 0 (1): the A (B) block is cut by a triangular mask
    int full_a, full_b;  // the tile's whole A (B) panel is already published
    int mode_a, mode_b;  // the segment's operand modes after the reuse logic (reused_a/_b)
    int watch;           // shared packing: the count of packed tiles is not complete yet
    int flag;
    int next_tile;       // the data-parallel tile this CTA takes next
};

// Loads one 16-byte chunk (CH elements) from shared memory.
template <typename T> __device__ __forceinline__ void lds16(T *dst, const T *src);
template <> __device__ __forceinline__ void lds16<double>(double *dst, const double *src)
{
    const double2 v = *reinterpret_cast<const double2 *>(src);
    dst[0] = v.x;
    dst[1] = v.y;
}
template <> __device__ __forceinline__ void lds16<float>(float *dst, const float *src)
{
    const float4 v = *reinterpret_cast<const float4 *>(src);
    dst[0] = v.x;
    dst[1] = v.y;
    dst[2] = v.z;
    dst[3] = v.w;
}

// TMASK: compile the triangular-operand handling (TRMM); every other launch runs without it.
template <typename T, bool ACONTIG, bool BCONTIG, typename C = TileCfg<T>, bool TMASK = false>
struct Kernel {
    using Cfg = C;
    using Smem = GemmSmem<T, C>;
    static constexpr int BM = Cfg::BM, BN = Cfg::BN, BK = Cfg::BK;
    static constexpr int THREADS = Cfg::THREADS, STAGES = Cfg::STAGES;
    static constexpr int CH = 16 / static_cast<int>(sizeof(T));
    // register micro-tile: NCM (NCN) 16-byte chunks along m (n), chunk c at c/NCM (c/NCN)
    // of the tile
    static constexpr int NCM = Cfg::NCM, NCN = Cfg::NCN;
    static constexpr int TM = NCM * CH, TN = NCN * CH;
    static constexpr int TX = BM / TM;               // threads along m
    static_assert(TX * (BN / TN) == THREADS, "thread grid must cover the tile");
    static_assert(NCN == 1 || NCN == 2, "one or two chunks along n");
    static_assert(NCM == 2 || NCM == 4, "two or four chunks along m");
    static constexpr int DEC = 4 * STAGES;   // decision ring: STAGES ahead, PUB behind
    static constexpr int PUB = 4;            // k-blocks a producer publishes per fence
    using LoadA = RawLoader<T, BM, BK, THREADS, ACONTIG>;
    using LoadB = RawLoader<T, BN, BK, THREADS, BCONTIG>;
    using AccT = T[TM][TN];

    // Decision for one operand tile at one k-block, in two steps so the ready-word load
    // overlaps compute.  FIP with line producers: the first tile column produces A panels,
    // the first tile row produces B panels; the others read what is already published (the
    // whole panel, known at segment start, or this k-block's word).  FIP with shared packing:
    // no producers; a panel counts as whole once the count of packed tiles is complete.
    //   need_word(): does the decision need this k-block's ready word?
    //   classify():  the decision, given that word (relaxed-loaded) when needed.
    static __device__ __forceinline__ bool need_word(int mode, bool producer, int full)
    {
        return mode == MODE_FIP && !producer && !full;
    }
    static __device__ __forceinline__ int classify(int mode, bool producer, int full,
                                                   unsigned long long word, unsigned int epoch)
    {
        if (mode == MODE_RAW) return DEC_RAW;
        if (mode == MODE_PACKED) return DEC_PACKED;
        if (producer) return DEC_PRODUCE;
        if (full) return DEC_PACKED;
        return word == ready_value(epoch) ? DEC_PACKED : DEC_RAW;
    }

    // Is C[row, col] inside the part of C the launch computes (the whole of C, or a triangle)?
    static __device__ __forceinline__ bool in_tri(const GemmParams<T> &p, int row, int col)
    {
        return p.tri == TRI_NONE || (p.tri == TRI_LOWER ? row >= col : row <= col);
    }

    // Producers: the first tile column packs the A panels, the first tile row the B panels
    // (Alg. 1), unless the launch reads that operand from the other one's packed copy.
    static __device__ __forceinline__ bool prod_a(const GemmParams<T> &p, int j)
    {
        return j == 0 && p.a_produces;
    }
    static __device__ __forceinline__ bool prod_b(const GemmParams<T> &p, int i)
    {
        return i == 0 && p.b_produces;
    }

    struct Words {
        unsigned long long a, b;
    };

    static __device__ __forceinline__ Words fetch_words(const GemmParams<T> &p,
                                                        const Smem &sm, int i, int j,
                                                        int kb)
    {
        Words w{0ull, 0ull};
        if (need_word(sm.mode_a, prod_a(p, j), sm.full_a))
            w.a = ld_relaxed(p.state_a + (int64_t)i * p.kt + kb);
        if (need_word(sm.mode_b, prod_b(p, i), sm.full_b))
            w.b = ld_relaxed(p.state_b + (int64_t)j * p.kt + kb);
        return w;
    }

    // Stores the decisions for local k-block q; returns true if one of them reads a tile
    // published by another CTA (the caller then issues fence_acquire()).
    static __device__ __forceinline__ bool store_decisions(const GemmParams<T> &p,
                                                           Smem &sm, int i, int j, int kb,
                                                           Words w, int q, unsigned int epoch)
    {
        int da = classify(sm.mode_a, prod_a(p, j), sm.full_a, w.a, epoch);
        int db = classify(sm.mode_b, prod_b(p, i), sm.full_b, w.b, epoch);
        if constexpr (TMASK) {
            // triangular operands: a k-block in which either operand block lies outside its
            // triangle contributes nothing and is not computed; an operand block is then not
            // loaded either, unless this tile packs it for others (a producer packs every
            // nonzero block of its panel, so a panel published complete has no holes); a
            // block the diagonal cuts is loaded with a mask
            const int ca = tmask_class(p.tmask_a, i * BM, BM, kb * BK, BK);
            const int cb = tmask_class(p.tmask_b, j * BN, BN, kb * BK, BK);
            const bool idle = (ca == 2 || cb == 2);
            if (ca == 2 || (idle && da != DEC_PRODUCE)) da = DEC_SKIP;
            if (cb == 2 || (idle && db != DEC_PRODUCE)) db = DEC_SKIP;
            sm.part[q % DEC] = (ca == 1 ? 1 : 0) | (cb == 1 ? 2 : 0) | (idle ? 4 : 0);
        } else {
            (void)kb;
        }
        sm.dec_a[q % DEC] = da;
        sm.dec_b[q % DEC] = db;
        return (da == DEC_PACKED && sm.mode_a == MODE_FIP && !sm.full_a) ||
               (db == DEC_PACKED && sm.mode_b == MODE_FIP && !sm.full_b);
    }

    static __device__ __forceinline__ void issue(const GemmParams<T> &p, Smem &sm,
                                                 LoadA &la, LoadB &lb, int i, int j, int kb,
                                                 int q, int tid)
    {
        const int stage = q % STAGES;
        const int kleft = p.k - kb * BK;
        const uint32_t sa = smem_addr(sm.a[stage]), sb = smem_addr(sm.b[stage]);
        if constexpr (TMASK) {
            const int part = sm.part[q % DEC];
            if (sm.dec_a[q % DEC] == DEC_SKIP) {
                la.skip();
            } else if (sm.dec_a[q % DEC] == DEC_PACKED) {
                load_packed_tile<T, BM, BK, THREADS>(
                    sa, p.pack_a + ((int64_t)i * p.kt + kb) * (BM * BK), tid);
                la.skip();
            } else if (part & 1) {
                la.issue_masked(sa, kleft, kb * BK, p.tmask_a, tid);
            } else {
                la.issue(sa, kleft, tid);
            }
            if (sm.dec_b[q % DEC] == DEC_SKIP) {
                lb.skip();
            } else if (sm.dec_b[q % DEC] == DEC_PACKED) {
                load_packed_tile<T, BN, BK, THREADS>(
                    sb, p.pack_b + ((int64_t)j * p.kt + kb) * (BN * BK), tid);
                lb.skip();
            } else if (part & 2) {
                lb.issue_masked(sb, kleft, kb * BK, p.tmask_b, tid);
            } else {
                lb.issue(sb, kleft, tid);
            }
        } else {
            if (sm.dec_a[q % DEC] == DEC_PACKED) {
                load_packed_tile<T, BM, BK, THREADS>(
                    sa, p.pack_a + ((int64_t)i * p.kt + kb) * (BM * BK), tid);
                la.skip();
            } else {
                la.issue(sa, kleft, tid);
            }
            if (sm.dec_b[q % DEC] == DEC_PACKED) {
                load_packed_tile<T, BN, BK, THREADS>(
                    sb, p.pack_b + ((int64_t)j * p.kt + kb) * (BN * BK), tid);
                lb.skip();
            } else {
                lb.issue(sb, kleft, tid);
            }
        }
    }

    // acc += As^T Bs over the BK rows of one stage.  Fragment addresses are a per-thread base
    // plus kk * P; the loop is unrolled UNROLL rows at a time to bound the code size.
    static constexpr int UNROLL = BK < Cfg::UNROLL ? BK : Cfg::UNROLL;
    // Only the first NMA of the NCM row chunks and the first kext rows of k (a multiple of
    // UNROLL) are computed: a fringe tile skips rows past m and k-rows past k, which hold
    // zero padding or belong to rows that are never stored.
    template <int NMA>
    static __device__ __forceinline__ void compute(const T *As, const T *Bs, T (&acc)[TM][TN],
                                                   int tx, int ty, int kext)
    {
        using LA = TileLayout<T, BM, BK>;
        using LB = TileLayout<T, BN, BK>;
        const T *a0 = As + LA::off(tx * CH, 0);
        const T *b0 = Bs + LB::off(ty * CH, 0);
        // chunk c of a fragment sits c * BM / NCM (BN / NCN) further along x: whole 128-byte
        // segments, i.e. a constant offset in the layout
        static_assert((BM / NCM) % LA::W == 0 && (NCN == 1 || (BN / NCN) % LB::W == 0),
                      "fragment chunks must be whole segments apart");
        constexpr int DA = (BM / NCM) / LA::W * LA::SEG, DB = (BN / NCN) / LB::W * LB::SEG;
#pragma unroll 1
        for (int k0 = 0; k0 < kext; k0 += UNROLL) {
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                const int kk = k0 + u;
                T a[TM], b[TN];
#pragma unroll
                for (int c = 0; c < NMA; ++c)
                    lds16<T>(a + c * CH, a0 + c * DA + kk * LA::P);
#pragma unroll
                for (int c = 0; c < NCN; ++c)
                    lds16<T>(b + c * CH, b0 + c * DB + kk * LB::P);
                fma_block<NMA * CH>(a, b, acc);
            }
        }
    }

    // acc[ii][jj] += a[ii] * b[jj].  FP32 uses the paired FMA of sm_100+ (two lanes of
    // independent single-rounding FMAs per instruction, so the result bits equal fmaf's),
    // which halves the instructions the FFMA-bound loop issues.
    template <int TME>   // rows of the micro-tile computed (TM, or a fringe tile's first chunks)
    static __device__ __forceinline__ void fma_block(const T (&a)[TM], const T (&b)[TN],
                                                     T (&acc)[TM][TN])
    {
        if constexpr (std::is_same<T, float>::value && TM >= TN) {
            // pairs along m: {a[ii], a[ii+1]} x b[jj] (b[jj] duplicated once per jj)
#pragma unroll
            for (int jj = 0; jj < TN; ++jj) {
                const float2 bb = make_float2(b[jj], b[jj]);
#pragma unroll
                for (int ii = 0; ii < TME; ii += 2) {
                    const float2 c = __ffma2_rn(make_float2(a[ii], a[ii + 1]), bb,
                                                make_float2(acc[ii][jj], acc[ii + 1][jj]));
                    acc[ii][jj] = c.x;
                    acc[ii + 1][jj] = c.y;
                }
            }
        } else if constexpr (std::is_same<T, float>::value) {
            // pairs along n: a[ii] x {b[jj], b[jj+1]}
#pragma unroll
            for (int ii = 0; ii < TME; ++ii) {
                const float2 aa = make_float2(a[ii], a[ii]);
#pragma unroll
                for (int jj = 0; jj < TN; jj += 2) {
                    const float2 c = __ffma2_rn(aa, make_float2(b[jj], b[jj + 1]),
                                                make_float2(acc[ii][jj], acc[ii][jj + 1]));
                    acc[ii][jj] = c.x;
                    acc[ii][jj + 1] = c.y;
                }
            }
        } else {
#pragma unroll
            for (int ii = 0; ii < TME; ++ii)
#pragma unroll
                for (int jj = 0; jj < TN; ++jj) acc[ii][jj] = fma(a[ii], b[jj], acc[ii][jj]);
        }
    }

    // Value of the count of packed tiles once shared packing is complete in this launch: the
    // epoch in the upper half, twice the tiles in the lower (each tile counts 2, so a count
    // is even and never equals a ready word, which is odd).
    static __device__ __forceinline__ unsigned long long all_packed(const GemmParams<T> &p,
                                                                    unsigned int epoch)
    {
        return (static_cast<unsigned long long>(epoch) << 32) |
               (2ull * static_cast<unsigned long long>(p.pack_units));
    }

    // Publishes the tiles this CTA produced at local k-blocks it0 .. it1 - 1 (thread 0 only,
    // after a CTA barrier that follows their pack stores): one release fence for the whole
    // range, then relaxed stores of the ready words.  Batching PUB k-blocks per fence keeps
    // the fence, which stalls warp 0 until its earlier memory operations are done, off most
    // k-blocks; only tiles running beside the producer could use a finer grain.
    static __device__ __forceinline__ void publish_produced(const GemmParams<T> &p,
                                                            const Smem &sm, int i, int j,
                                                            int kb0, int it0, int it1,
                                                            unsigned int epoch)
    {
        bool any = false;
        for (int it = it0; it < it1; ++it)
            any |= sm.dec_a[it % DEC] == DEC_PRODUCE || sm.dec_b[it % DEC] == DEC_PRODUCE;
        if (!any) return;
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        const unsigned long long v = ready_value(epoch);
        for (int it = it0; it < it1; ++it) {
            if (sm.dec_a[it % DEC] == DEC_PRODUCE)
                asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(
                                 p.state_a + (int64_t)i * p.kt + kb0 + it),
                             "l"(v)
                             : "memory");
            if (sm.dec_b[it % DEC] == DEC_PRODUCE)
                asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(
                                 p.state_b + (int64_t)j * p.kt + kb0 + it),
                             "l"(v)
                             : "memory");
        }
    }

    // Accumulates op(A)[tile rows, kb0*BK : kb1*BK] * op(B)[..., tile cols] into acc, packing
    // operand tiles on the way where this tile is a producer.
    // FRINGE: compile fringe-tile shortcuts; 1: the last k-block trimmed to its rows of k and
    // idle warps skipping the FMA loop, 2: also the half-height micro-tile for tiles whose
    // lower row chunks lie past m.  They pay where most tiles are fringe tiles (grouped
    // problems); elsewhere their registers cost the full tiles more than they save.
    template <int FRINGE = 0>
    static __device__ void run_segment(const GemmParams<T> &p, Smem &sm, int i, int j,
                                       int kb0, int kb1, T (&acc)[TM][TN], unsigned int epoch)
    {
        const int tid = threadIdx.x;
        const int tx = tid % TX, ty = tid / TX;
        const int nkb = kb1 - kb0;
        // fringe tiles: a warp whose columns all lie past n has nothing to compute; if every
        // row chunk but the first lies past m, only the first is computed
        const bool warp_idle = FRINGE >= 1 && j * BN + ((tid & ~31) / TX) * CH >= p.n;
        const bool half_rows = FRINGE >= 2 && i * BM + BM / NCM >= p.m;

#pragma unroll
        for (int ii = 0; ii < TM; ++ii)
#pragma unroll
            for (int jj = 0; jj < TN; ++jj) acc[ii][jj] = T(0);

        // the segment that ends the tile's k loop will read C: warm L2 with it now
        if (kb1 == p.kt && p.beta != T(0)) {
            constexpr int LINES = 128 / static_cast<int>(sizeof(T));  // elements per line
            constexpr int PER_COL = (BM + LINES - 1) / LINES;
            for (int e = tid; e < BN * PER_COL; e += THREADS) {
                const int col = j * BN + e / PER_COL, row = i * BM + (e % PER_COL) * LINES;
                if (col < p.n && row < p.m)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(p.C + row + (int64_t)col * p.ldc));
            }
        }
        LoadA la;
        LoadB lb;
        la.init(p.A, p.lda, i * BM, kb0 * BK, p.m, tid);
        lb.init(p.B, p.ldb, j * BN, kb0 * BK, p.n, tid);

        if (tid == 0) {
            // a panel whose producer finished it whole needs no per-k-block look-ups; with
            // shared packing, every panel is whole once all CTAs have counted their tiles
            // (until then thread 0 watches the count, loaded in place of the words)
            // operands of panels that no later tile reuses are read raw here (reused_a/_b)
            sm.mode_a = (p.mode_a == MODE_FIP && !reused_a(p, i)) ? MODE_RAW : p.mode_a;
            sm.mode_b = (p.mode_b == MODE_FIP && !reused_b(p, j)) ? MODE_RAW : p.mode_b;
            const bool all = !TMASK && p.shared_pack &&
                             ld_relaxed(p.pack_count) == all_packed(p, epoch);
            sm.watch = !TMASK && p.shared_pack && !all;
            const bool fa = need_word(sm.mode_a, prod_a(p, j), 0) &&
                            (all || ld_relaxed(p.state_a + (int64_t)p.mt * p.kt + i) ==
                                        ready_value(epoch));
            const bool fb = need_word(sm.mode_b, prod_b(p, i), 0) &&
                            (all || ld_relaxed(p.state_b + (int64_t)p.nt * p.kt + j) ==
                                        ready_value(epoch));
            sm.full_a = fa;
            sm.full_b = fb;
            Words w[STAGES];
#pragma unroll
            for (int q = 0; q < STAGES; ++q)
                if (q < nkb) w[q] = fetch_words(p, sm, i, j, kb0 + q);
            bool acq = fa || fb;
#pragma unroll
            for (int q = 0; q < STAGES; ++q)
                if (q < nkb) acq |= store_decisions(p, sm, i, j, kb0 + q, w[q], q, epoch);
            if (acq) fence_acquire();
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < STAGES - 1; ++q) {
            if (q < nkb) issue(p, sm, la, lb, i, j, kb0 + q, q, tid);
            cp_async_commit();
        }

        for (int it = 0; it < nkb; ++it) {
            cp_async_wait<STAGES - 2>();
            __syncthreads();
            const int stage = it % STAGES;
            if (sm.dec_a[it % DEC] == DEC_PRODUCE)
                store_packed_tile<T, BM, BK, THREADS>(
                    p.pack_a + ((int64_t)i * p.kt + kb0 + it) * (BM * BK), sm.a[stage], tid);
            if (sm.dec_b[it % DEC] == DEC_PRODUCE)
                store_packed_tile<T, BN, BK, THREADS>(
                    p.pack_b + ((int64_t)j * p.kt + kb0 + it) * (BN * BK), sm.b[stage], tid);
            const int q = it + STAGES - 1;
            if (q < nkb) issue(p, sm, la, lb, i, j, kb0 + q, q, tid);
            cp_async_commit();
            // ready words for k-block it+STAGES: loaded now, used after this block's compute
            const bool ahead = (tid == 0) && (it + STAGES < nkb);
            Words w{0ull, 0ull};
            if (ahead) w = fetch_words(p, sm, i, j, kb0 + it + STAGES);
            // shared packing publishes no per-k-block words (they read as not ready); while
            // the count of packed tiles is incomplete it travels in A's word slot (counts are
            // even, ready words odd, so classify() never takes it for a ready word)
            if (!TMASK && ahead && p.shared_pack && sm.watch) w.a = ld_relaxed(p.pack_count);
            if (!warp_idle && !(TMASK && (sm.part[it % DEC] & 4))) {
                // the tile's last k-block computes only its rows of k that exist
                const int kin = p.k - (kb0 + it) * BK;
                const int kext =
                    (FRINGE == 0 || kin >= BK) ? BK : ((kin + UNROLL - 1) / UNROLL) * UNROLL;
                if (FRINGE >= 2 && half_rows)
                    compute<1>(sm.a[stage], sm.b[stage], acc, tx, ty, kext);
                else
                    compute<NCM>(sm.a[stage], sm.b[stage], acc, tx, ty, kext);
            }
            if (tid == 0) {
                if (!TMASK && ahead && p.shared_pack && sm.watch &&
                    w.a == all_packed(p, epoch)) {
                    // every panel is packed: k-blocks from it + STAGES on read the copies
                    sm.full_a = need_word(sm.mode_a, false, 0);
                    sm.full_b = need_word(sm.mode_b, false, 0);
                    sm.watch = 0;
                    fence_acquire();
                }
                if (ahead && store_decisions(p, sm, i, j, kb0 + it + STAGES, w, it + STAGES, epoch))
                    fence_acquire();
                // the pack stores of the previous PUB k-blocks were ordered by this
                // iteration's barrier and have drained during the compute
                if (it > 0 && it % PUB == 0) publish_produced(p, sm, i, j, kb0, it - PUB, it, epoch);
            }
        }
        cp_async_wait<0>();
        __syncthreads();
        if (tid == 0 && nkb > 0) {
            publish_produced(p, sm, i, j, kb0, ((nkb - 1) / PUB) * PUB, nkb, epoch);
            // a producer that covered its whole panel publishes the panel as complete
            if (kb0 == 0 && kb1 == p.kt) {
                if (sm.mode_a == MODE_FIP && prod_a(p, j))
                    publish(p.state_a + (int64_t)p.mt * p.kt + i, epoch);
                if (sm.mode_b == MODE_FIP && prod_b(p, i))
                    publish(p.state_b + (int64_t)p.nt * p.kt + j, epoch);
            }
        }
    }

    // C[tile] := alpha*acc + beta*C[tile]; C is not read when beta == 0.  A column's C values
    // are all loaded before any of them is stored, so their load latencies overlap instead of
    // queueing behind the stores (the stores could alias later loads as far as the compiler
    // knows).
    static __device__ void epilogue(const GemmParams<T> &p, int i, int j,
                                    const T (&acc)[TM][TN])
    {
        const int tid = threadIdx.x;
        const int tx = tid % TX, ty = tid / TX;
        const int m0 = i * BM, n0 = j * BN;
        const bool read_c = (p.beta != T(0));
#pragma unroll
        for (int jj = 0; jj < TN; ++jj) {
            const int col = n0 + ty * CH + (jj % CH) + (jj / CH) * (BN / NCN);
            if (col >= p.n) continue;
            T *ccol = p.C + (int64_t)col * p.ldc;
            T c[TM];
#pragma unroll
            for (int ii = 0; ii < TM; ++ii) {
                const int row = m0 + tx * CH + (ii % CH) + (ii / CH) * (BM / NCM);
                c[ii] = (read_c && row < p.m && in_tri(p, row, col)) ? ccol[row] : T(0);
            }
#pragma unroll
            for (int ii = 0; ii < TM; ++ii) {
                const int row = m0 + tx * CH + (ii % CH) + (ii / CH) * (BM / NCM);
                if (row >= p.m || !in_tri(p, row, col)) continue;
                T v = p.alpha * acc[ii][jj];
                if (read_c) v = fma(p.beta, c[ii], v);
                ccol[row] = v;
            }
        }
    }

    // Stream-K bookkeeping: the CTA whose iteration range contains split iteration q.
    static __device__ __forceinline__ int cta_of(int64_t q, int64_t S, int G)
    {
        return static_cast<int>(((q + 1) * G - 1) / S);
    }

    // A split tile's partial sum: store it, count arrivals, and let the last arrival add the
    // partials of all segments in k order and write C.
    static __device__ void fixup(const GemmParams<T> &p, Smem &sm, int t, int i, int j,
                                 int g, int slot, T (&acc)[TM][TN], unsigned int epoch)
    {
        const int tid = threadIdx.x;
        const int64_t S = p.sk_iters;
        const int G = p.grid;
        const int u = t - p.dp_tiles;
        const int g0 = cta_of((int64_t)u * p.kt, S, G);
        const int g1 = cta_of((int64_t)(u + 1) * p.kt - 1, S, G);
        const int nseg = g1 - g0 + 1;

        T *mine = p.partial + (int64_t)(2 * g + slot) * (BM * BN);
#pragma unroll
        for (int ii = 0; ii < TM; ++ii)
#pragma unroll
            for (int jj = 0; jj < TN; ++jj)
                __stcg(mine + (ii * TN + jj) * THREADS + tid, acc[ii][jj]);
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            const unsigned long long tag = static_cast<unsigned long long>(epoch) << 32;
            atomicMax(p.tile_count + t, tag);
            const unsigned long long old = atomicAdd(p.tile_count + t, 1ull);
            const long long cnt = static_cast<long long>(old - tag) + 1;
            if ((old >> 32) != epoch || cnt > nseg) atomicOr(p.status, STATUS_BAD_SEGMENT);
            sm.flag = (cnt == nseg);
            __threadfence();
        }
        __syncthreads();
        if (sm.flag) {
            // add the segments' partial sums in k order; the loads of up to INFL segments are
            // issued before any of their adds so their latencies overlap
            constexpr int NV = TM * TN;
            constexpr int CHK = NV;                          // values per pass
            constexpr int INFL = NV <= 8 ? 4 : (NV <= 16 ? 2 : 1);  // segments in flight
            T *flat = &acc[0][0];
#pragma unroll
            for (int c0 = 0; c0 < NV; c0 += CHK) {
                for (int gg = g0; gg <= g1; gg += INFL) {
                    T v[INFL][CHK];
#pragma unroll
                    for (int s = 0; s < INFL; ++s) {
                        const int gs = gg + s;
                        if (gs > g1) break;
                        const int64_t lo = S * gs / G;
                        const int gslot = (lo / p.kt == u) ? 0 : 1;
                        const T *src = p.partial + (int64_t)(2 * gs + gslot) * (BM * BN);
#pragma unroll
                        for (int e = 0; e < CHK; ++e)
                            v[s][e] = __ldcg(src + (c0 + e) * THREADS + tid);
                    }
#pragma unroll
                    for (int s = 0; s < INFL; ++s) {
                        const int gs = gg + s;
                        if (gs > g1) break;
#pragma unroll
                        for (int e = 0; e < CHK; ++e)
                            flat[c0 + e] = (gs == g0) ? v[s][e] : flat[c0 + e] + v[s][e];
                    }
                }
            }
            epilogue(p, i, j, acc);
        }
        __syncthreads();
    }

    // Shared packing (the collaborative packing of Sec. 3.5, read for a GPU): before its
    // tiles, every CTA packs a share of the (panel, k-block) tiles of the packed operands.
    // Unit u is k-block u / P of panel u % P (P = packed panels, A's first), CTA g takes u = g,
    // g + grid, ...; the copies run 2 STAGES - 1 units ahead of the stores.  Completion is one
    // epoch-tagged count of packed tiles, not a ready word per tile: a tile reads the raw
    // operand until the count shows every CTA done, then the packed copies, after a single
    // acquire fence (a fence per k-block stalls the warp of the thread that takes it).
    static __device__ void share_pack(const GemmParams<T> &p, Smem &sm, unsigned int epoch)
    {
        // all 2 * STAGES stage buffers take pack units (A and B tiles have the same shape),
        // so that up to 2 * STAGES - 1 units' copies are in flight
        static_assert(BM == BN, "shared packing uses A and B stage buffers alike");
        constexpr int NBUF = 2 * STAGES;
        const int tid = threadIdx.x;
        const int g = blockIdx.x;
        const int pa = (p.mode_a == MODE_FIP) ? p.mt : 0;
        const int pb = (p.mode_b == MODE_FIP) ? p.nt : 0;
        const int64_t per_kb = pa + pb;
        const int64_t units = per_kb * p.kt;
        if (g >= units) return;
        const int mine = static_cast<int>((units - 1 - g) / p.grid) + 1;
        auto buf = [&](int r) -> T * { return (r % NBUF < STAGES) ? sm.a[r % NBUF]
                                                                  : sm.b[r % NBUF - STAGES]; };
        auto locate = [&](int r, int &panel, int &kb) {   // panel < pa: A panel, else B
            const int64_t u = g + (int64_t)r * p.grid;
            kb = static_cast<int>(u / per_kb);
            panel = static_cast<int>(u % per_kb);
        };
        auto issue_unit = [&](int r) {
            int x, kb;
            locate(r, x, kb);
            if (x < pa) {
                LoadA l;
                l.init(p.A, p.lda, x * BM, kb * BK, p.m, tid);
                l.issue(smem_addr(buf(r)), p.k - kb * BK, tid);
            } else {
                LoadB l;
                l.init(p.B, p.ldb, (x - pa) * BN, kb * BK, p.n, tid);
                l.issue(smem_addr(buf(r)), p.k - kb * BK, tid);
            }
        };
#pragma unroll
        for (int q = 0; q < NBUF - 1; ++q) {
            if (q < mine) issue_unit(q);
            cp_async_commit();
        }
        for (int r = 0; r < mine; ++r) {
            cp_async_wait<NBUF - 2>();
            __syncthreads();
            int x, kb;
            locate(r, x, kb);
            if (x < pa)
                store_packed_tile<T, BM, BK, THREADS>(
                    p.pack_a + ((int64_t)x * p.kt + kb) * (BM * BK), buf(r), tid);
            else
                store_packed_tile<T, BN, BK, THREADS>(
                    p.pack_b + ((int64_t)(x - pa) * p.kt + kb) * (BN * BK), buf(r), tid);
            // refills the buffer stored in the previous iteration (read before the barrier)
            const int q = r + NBUF - 1;
            if (q < mine) issue_unit(q);
            cp_async_commit();
        }
        cp_async_wait<0>();
        __syncthreads();
        if (tid == 0) {
            // count this CTA's tiles once its stores (ordered by the barrier) are visible;
            // the count reaching pack_units tells a tile that every panel is complete
            __threadfence();
            const unsigned long long tag = static_cast<unsigned long long>(epoch) << 32;
            atomicMax(p.pack_count, tag);
            atomicAdd(p.pack_count, 2ull * static_cast<unsigned long long>(mine));
        }
    }

    // Thread 0's `epoch` tags the ready words and arrival counters this launch writes (only
    // thread 0 of a CTA reads or writes them).
    static __device__ void run(const GemmParams<T> &p, Smem &sm, unsigned int epoch)
    {
        const int g = blockIdx.x;
        T acc[TM][TN];
        if (!TMASK && p.shared_pack) share_pack(p, sm, epoch);
        // Data-parallel tiles in order: CTA g takes tile g first, then tiles grid, grid + 1,
        // ... from a launch-wide counter (epoch-tagged, so nothing is cleared between
        // launches), so a CTA slowed by extra work, such as a producer's pack stores, takes
        // fewer tiles and the CTAs reach the split wave together.  Thread 0 asks for its next
        // tile while the current one runs.  Tile t still starts in round about t / grid, the
        // round the reuse logic (reused_a/_b) reckons with.
        const unsigned long long tag = static_cast<unsigned long long>(epoch) << 32;
        bool first = true;
        for (int t = g; t < p.dp_tiles; t = sm.next_tile) {
            unsigned long long next = 0;
            if (threadIdx.x == 0) {
                if (first) atomicMax(p.tile_next, tag);   // ordered before the add below
                next = atomicAdd(p.tile_next, 1ull);
            }
            first = false;
            int i, j;
            tile_of(p, t, i, j);
            run_segment(p, sm, i, j, 0, p.kt, acc, epoch);   // its barriers order t's reads
            epilogue(p, i, j, acc);
            if (threadIdx.x == 0) sm.next_tile = p.grid + static_cast<int>(next - tag);
            __syncthreads();
        }
        if (p.sk_iters > 0) {
            const int64_t lo = p.sk_iters * g / p.grid, hi = p.sk_iters * (g + 1) / p.grid;
            const int first_u = static_cast<int>(lo / p.kt);
            int64_t q = lo;
            while (q < hi) {
                const int u = static_cast<int>(q / p.kt);
                const int t = p.dp_tiles + u;
                int i, j;
                tile_of(p, t, i, j);
                const int kb0 = static_cast<int>(q % p.kt);
                const int64_t rest = hi - q;
                const int kb1 =
                    (rest < (int64_t)(p.kt - kb0)) ? kb0 + static_cast<int>(rest) : p.kt;
                run_segment(p, sm, i, j, kb0, kb1, acc, epoch);
                if (kb0 == 0 && kb1 == p.kt) {
                    epilogue(p, i, j, acc);
                    __syncthreads();
                } else {
                    fixup(p, sm, t, i, j, g, (u == first_u) ? 0 : 1, acc, epoch);
                }
                q += kb1 - kb0;
            }
        }
    }
};

// The launch's epoch tags every ready word and arrival counter it writes, so words left by
// earlier launches read as stale and nothing is cleared between calls.  It lives on the
// device: thread 0 of every CTA reads the launch counter at start (epoch = counter + 1), and
// the last CTA to finish stores the new value, so a launch replayed from a CUDA graph gets a
// fresh epoch too.  (The next launch on the stream starts only after this one has finished,
// and every CTA has read the counter before it counts itself finished.)  The counter is held
// in a register: only thread 0 uses it, so its load latency hides behind the first loads.
template <typename T, bool ACONTIG, bool BCONTIG, bool TMASK = false>
__global__ void __launch_bounds__(TileCfg<T>::THREADS, TileCfg<T>::MIN_BLOCKS)
    gemm_kernel(const GemmParams<T> p)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    GemmSmem<T> &sm = *reinterpret_cast<GemmSmem<T> *>(smem_raw);
    unsigned int epoch = 0u;
    if (threadIdx.x == 0) epoch = *(volatile unsigned int *)p.launch_count + 1u;
    Kernel<T, ACONTIG, BCONTIG, TileCfg<T>, TMASK>::run(p, sm, epoch);
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(p.done_count, 1u) == gridDim.x - 1) {
            *(volatile unsigned int *)p.done_count = 0u;
            *(volatile unsigned int *)p.launch_count = epoch;
            __threadfence();
        }
    }
}

// One (panel, k-block) tile of the pack-then-compute variant: raw load into shared memory,
// then the same image the fused kernel writes.
template <typename T, int BX, bool CONTIG>
__device__ __forceinline__ void pack_one(const T *g, int64_t ld, int panel, int kb, int x_ext,
                                         int k_ext, T *dst, T *tile, int tid)
{
    using Cfg = TileCfg<T>;
    RawLoader<T, BX, Cfg::BK, Cfg::THREADS, CONTIG> l;
    l.init(g, ld, panel * BX, kb * Cfg::BK, x_ext, tid);
    l.issue(smem_addr(tile), k_ext - kb * Cfg::BK, tid);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    store_packed_tile<T, BX, Cfg::BK, Cfg::THREADS>(dst, tile, tid);
}

// Pack kernel of the pack-then-compute variant: block b packs one tile, A tiles first.
template <typename T, bool ACONTIG, bool BCONTIG>
__global__ void __launch_bounds__(TileCfg<T>::THREADS) pack_kernel(const PackParams<T> p)
{
    using Cfg = TileCfg<T>;
    constexpr int BM = Cfg::BM, BN = Cfg::BN, BK = Cfg::BK;
    constexpr int BX = BM > BN ? BM : BN;
    __shared__ __align__(128) T tile[TileLayout<T, BX, BK>::ELEMS];
    const int tid = threadIdx.x;
    const int64_t a_tiles = (int64_t)p.mt * p.kt;
    const int64_t b = blockIdx.x;
    if (b < a_tiles) {
        const int i = static_cast<int>(b / p.kt), kb = static_cast<int>(b % p.kt);
        pack_one<T, BM, ACONTIG>(p.A, p.lda, i, kb, p.m, p.k, p.pack_a + b * (BM * BK), tile,
                                 tid);
    } else {
        const int64_t bb = b - a_tiles;
        const int j = static_cast<int>(bb / p.kt), kb = static_cast<int>(bb % p.kt);
        pack_one<T, BN, BCONTIG>(p.B, p.ldb, j, kb, p.n, p.k, p.pack_b + bb * (BN * BK), tile,
                                 tid);
    }
}

// C := beta*C on the m x n region, or on one triangle of it (beta == 0 writes zeros without
// reading C).
template <typename T>
__global__ void scale_kernel(T *C, int64_t ldc, int m, int n, T beta, int tri)
{
    const int64_t total = (int64_t)m * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t col = e / m, row = e % m;
        if ((tri == TRI_LOWER && row < col) || (tri == TRI_UPPER && row > col)) continue;
        T *c = C + row + col * ldc;
        *c = (beta == T(0)) ? T(0) : beta * *c;
    }
}

template <typename T> inline size_t gemm_smem_bytes()
{
    return sizeof(GemmSmem<T>);
}

template <typename T, bool AC, bool BC, bool TM = false> cudaError_t configure_gemm()
{
    static bool configured = false;
    if (configured) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(gemm_kernel<T, AC, BC, TM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(gemm_smem_bytes<T>()));
    if (e == cudaSuccess) configured = true;
    return e;
}

template <typename T, bool AC, bool BC, bool TM>
cudaError_t launch_gemm_t(const GemmParams<T> &p, cudaStream_t s)
{
    cudaError_t e = configure_gemm<T, AC, BC, TM>();
    if (e != cudaSuccess) return e;
    gemm_kernel<T, AC, BC, TM><<<p.grid, TileCfg<T>::THREADS, gemm_smem_bytes<T>(), s>>>(p);
    return cudaGetLastError();
}

// Triangular-operand launches (TRMM) take the instantiation that handles masks.
template <typename T, bool AC, bool BC>
cudaError_t launch_gemm_mask(const GemmParams<T> &p, cudaStream_t s)
{
    return (p.tmask_a || p.tmask_b) ? launch_gemm_t<T, AC, BC, true>(p, s)
                                    : launch_gemm_t<T, AC, BC, false>(p, s);
}

template <typename T> cudaError_t launch_gemm_impl(const GemmParams<T> &p, cudaStream_t s)
{
    // dense FP32 GEMMs run on the warp-specialised tile core; SYRK triangles, TRMM masks and
    // the explicit shared packer stay on this one (same micro-tile and k order: same bits)
    if constexpr (std::is_same<T, float>::value)
        if (p.tri == TRI_NONE && !p.tmask_a && !p.tmask_b && !p.shared_pack)
            return launch_ws_gemm(p, s);
    if (p.a_contig_m)
        return p.b_contig_n ? launch_gemm_mask<T, true, true>(p, s)
                            : launch_gemm_mask<T, true, false>(p, s);
    return p.b_contig_n ? launch_gemm_mask<T, false, true>(p, s)
                        : launch_gemm_mask<T, false, false>(p, s);
}

template <typename T, bool AC, bool BC> int blocks_per_sm_one()
{
    if (configure_gemm<T, AC, BC>() != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gemm_kernel<T, AC, BC>,
                                                      TileCfg<T>::THREADS,
                                                      gemm_smem_bytes<T>()) != cudaSuccess)
        return 0;
    return n;
}

// Resident CTAs per SM: the minimum over the four operand-order instantiations, so the grid
// (and hence the split points and the result bits) does not depend on the operand order.
template <typename T> int gemm_blocks_per_sm_impl()
{
    int n = blocks_per_sm_one<T, true, true>();
    n = std::min(n, blocks_per_sm_one<T, true, false>());
    n = std::min(n, blocks_per_sm_one<T, false, true>());
    n = std::min(n, blocks_per_sm_one<T, false, false>());
    // FP32: the warp-specialised core runs with the same grid, hence the same split points
    if constexpr (std::is_same<T, float>::value) n = std::min(n, ws_blocks_per_sm());
    return n;
}

template <typename T> cudaError_t launch_pack_impl(const PackParams<T> &p, cudaStream_t s)
{
    // FP32 pack-then-compute GEMMs run on the warp-specialised core, which reads its own layout
    if constexpr (std::is_same<T, float>::value) return launch_ws_pack(p, s);
    const int64_t blocks = (int64_t)(p.mt + p.nt) * p.kt;
    if (blocks <= 0) return cudaSuccess;
    const unsigned int nb = static_cast<unsigned int>(blocks);
    const int th = TileCfg<T>::THREADS;
    if (p.a_contig_m) {
        if (p.b_contig_n)
            pack_kernel<T, true, true><<<nb, th, 0, s>>>(p);
        else
            pack_kernel<T, true, false><<<nb, th, 0, s>>>(p);
    } else {
        if (p.b_contig_n)
            pack_kernel<T, false, true><<<nb, th, 0, s>>>(p);
        else
            pack_kernel<T, false, false><<<nb, th, 0, s>>>(p);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scale_impl(T *C, int64_t ldc, int m, int n, T beta, int tri, cudaStream_t s)
{
    const int64_t total = (int64_t)m * n;
    const int threads = 256;
    int64_t blocks = (total + threads - 1) / threads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    scale_kernel<T><<<static_cast<unsigned int>(blocks), threads, 0, s>>>(C, ldc, m, n, beta,
                                                                        tri);
    return cudaGetLastError();
}

}  // namespace gfip

// The triangular-operand (TRMM) instantiations of the GEMM kernel are compiled in a
// translation unit of their own (gfip_f64_tmask.cu, gfip_f32_tmask.cu), so the two halves
// build in parallel.
#define GFIP_TMASK_LAUNCHERS(PREFIX, T)                                                        \
    namespace gfip {                                                                          \
    PREFIX template cudaError_t launch_gemm_t<T, true, true, true>(const GemmParams<T> &,      \
                                                                   cudaStream_t);              \
    PREFIX template cudaError_t launch_gemm_t<T, true, false, true>(const GemmParams<T> &,     \
                                                                    cudaStream_t);             \
    PREFIX template cudaError_t launch_gemm_t<T, false, true, true>(const GemmParams<T> &,     \
                                                                    cudaStream_t);             \
    PREFIX template cudaError_t launch_gemm_t<T, false, false, true>(const GemmParams<T> &,    \
                                                                     cudaStream_t);            \
    }

// Explicit instantiation of the launchers for one element type.
#define GFIP_INSTANTIATE(T)                                                                   \
    namespace gfip {                                                                          \
    template <> cudaError_t launch_gemm<T>(const GemmParams<T> &p, cudaStream_t s)            \
    {                                                                                         \
        return launch_gemm_impl<T>(p, s);                                                     \
    }                                                                                         \
    template <> cudaError_t launch_pack<T>(const PackParams<T> &p, cudaStream_t s)            \
    {                                                                                         \
        return launch_pack_impl<T>(p, s);                                                     \
    }                                                                                         \
    template <>                                                                               \
    cudaError_t launch_scale<T>(T * C, int64_t ldc, int m, int n, T beta, int tri,            \
                                cudaStream_t s)                                               \
    {                                                                                         \
        return launch_scale_impl<T>(C, ldc, m, n, beta, tri, s);                              \
    }                                                                                         \
    template <> int gemm_blocks_per_sm<T>()                                                   \
    {                                                                                         \
        return gemm_blocks_per_sm_impl<T>();                                                  \
    }                                                                                         \
    }
