// gfip_api.cu -- C ABI of the fused-in-packing GEMM: argument checks (reference-BLAS
// codes), quick returns, the launch plan (tile grid, schedule, pack modes), the workspace
// layout, and the launches.  See include/gemmfip.h for the contract.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <mutex>
#include <new>

#include <cuda_runtime.h>

#include "../../include/gemmfip.h"
#include "gfip_grouped.h"
#include "gfip_internal.h"
#include "gfip_testing.h"

namespace {

constexpr uint32_t kMagic = 0x67666970u;  // "gfip"
constexpr size_t kAlign = 256;
constexpr size_t kHeader = 256;             // status word, launch counters, spare
constexpr size_t kLaunchCountOffset = 64;   // header word: GEMM launches so far (epochs)
constexpr size_t kDoneCountOffset = 128;    // header word: finished CTAs of the running launch
constexpr size_t kPackCountOffset = 192;    // header word: tiles packed by shared packing
constexpr size_t kTileNextOffset = 32;      // header word: data-parallel tiles taken
constexpr size_t kCtrlGranule = 64 * 1024;  // control region grows in these steps
constexpr int kMinSplitRun = 8;              // shortest k run per CTA in a split wave
// Split tiles of an FP32 launch with fewer tiles than CTAs: each CTA takes at least this many
// k-blocks, so a 128 x 128 tile is summed from a few partial tiles, not from one per k-block.
constexpr int kMinSplitRunF32 = 4;
constexpr unsigned long long kOzakiWaitNs = 2000000000ull;  // 2 s per pipeline wait

struct Handle {
    uint32_t magic = kMagic;
    int device = 0;
    int sms = 0;
    cudaStream_t stream = nullptr;
    unsigned char *ws = nullptr;
    size_t ws_bytes = 0;
    // Bytes at the start of the workspace that hold only control words (zeros, or words a
    // kernel of this handle tagged with an older epoch).  Data never lives below this mark.
    size_t ctrl_bytes = 0;
    int pack_policy = GFIP_PACK_AUTO;
    int packer = GFIP_PACKER_AUTO;
    unsigned long long oz_wait_ns = kOzakiWaitNs;  // budget of the emulation kernel's waits
    int oz_inject = 0;                             // test hook (gfip_debug_ozaki_timeout)
    int last_launches = 0;
    int last_grid = 0;
    int bps_f64 = 0;
    int bps_f32 = 0;
};

Handle *get(gfip_handle_t h)
{
    Handle *p = reinterpret_cast<Handle *>(h);
    if (p == nullptr || p->magic != kMagic) return nullptr;
    return p;
}

size_t round_up(size_t x, size_t a)
{
    return (x + a - 1) / a * a;
}

bool is_trans_char(char t)
{
    return t == 'N' || t == 'n' || t == 'T' || t == 't' || t == 'C' || t == 'c';
}

bool is_notrans(char t)
{
    return t == 'N' || t == 'n';
}

// Reference-BLAS argument check (xerbla positions, negated).
int check_args(char transa, char transb, int64_t m, int64_t n, int64_t k, int64_t lda,
               int64_t ldb, int64_t ldc)
{
    if (!is_trans_char(transa)) return -1;
    if (!is_trans_char(transb)) return -2;
    if (m < 0) return -3;
    if (n < 0) return -4;
    if (k < 0) return -5;
    const int64_t rows_a = is_notrans(transa) ? m : k;
    const int64_t rows_b = is_notrans(transb) ? k : n;
    if (lda < std::max<int64_t>(1, rows_a)) return -8;
    if (ldb < std::max<int64_t>(1, rows_b)) return -10;
    if (ldc < std::max<int64_t>(1, m)) return -13;
    return 0;
}

enum class Variant { Fused, Direct, PackThenCompute };

template <typename T> struct Plan {
    int mt = 0, nt = 0, kt = 0, tiles = 0;
    int tri = gfip::TRI_NONE;   // triangle of C computed (SYRK), else the whole rectangle
    int grid = 0, dp_tiles = 0;
    int64_t sk_iters = 0;
    int mode_a = gfip::MODE_RAW, mode_b = gfip::MODE_RAW;
    bool shared = false;        // all CTAs pack first (else the first tile line packs)
    // workspace layout (byte offsets from the workspace base)
    size_t ctrl_needed = 0;
    size_t off_count = 0, off_state_a = 0, off_state_b = 0;
    size_t data_partial = 0, data_pack_a = 0, data_pack_b = 0, data_bytes = 0;
};

template <typename T> int blocks_per_sm(Handle *h)
{
    int &slot = (sizeof(T) == 8) ? h->bps_f64 : h->bps_f32;
    if (slot == 0) slot = gfip::gemm_blocks_per_sm<T>();
    return slot;
}

template <typename T>
Plan<T> make_plan(Handle *h, Variant v, int m, int n, int k, int tri = gfip::TRI_NONE,
                  bool masked = false)
{
    using Cfg = gfip::TileCfg<T>;
    Plan<T> pl;
    pl.mt = (m + Cfg::BM - 1) / Cfg::BM;
    pl.nt = (n + Cfg::BN - 1) / Cfg::BN;
    pl.kt = (k + Cfg::BK - 1) / Cfg::BK;
    pl.tri = tri;
    // a triangle (m == n, square tiles) holds the tiles on and on one side of the diagonal
    pl.tiles = tri ? pl.mt * (pl.mt + 1) / 2 : pl.mt * pl.nt;

    // Schedule: data-parallel waves of whole tiles, then the remaining tiles (the partial
    // wave, with one full wave more when the partial one is short) split evenly along k over
    // all CTAs.
    const int bps = std::max(1, blocks_per_sm<T>(h));
    const int full = h->sms * bps;
    const int64_t total_iters = (int64_t)pl.tiles * pl.kt;
    if (pl.tiles % full == 0) {
        pl.grid = full;
        pl.dp_tiles = pl.tiles;
        pl.sk_iters = 0;
    } else if (pl.tiles < full) {
        const int64_t run = sizeof(T) == 4 ? kMinSplitRunF32 : 1;
        pl.grid = static_cast<int>(std::min<int64_t>(full, std::max<int64_t>(
                                                               pl.tiles, (total_iters + run - 1) / run)));
        pl.dp_tiles = 0;
        pl.sk_iters = total_iters;
    } else {
        // The partial last wave is split along k.  If that would give each CTA a short run
        // (fewer than kMinSplitRun k-blocks, where the fix-up would dominate), one full wave
        // more is split with it.
        const int rem = pl.tiles % full;
        const bool short_run = (int64_t)rem * pl.kt < (int64_t)kMinSplitRun * full;
        const int sk_tiles = short_run ? rem + full : rem;
        pl.grid = full;
        pl.dp_tiles = pl.tiles - sk_tiles;
        pl.sk_iters = (int64_t)sk_tiles * pl.kt;
    }

    // Who packs: the first tile line (Alg. 1) at every size; the collaborative pre-pass only on
    // request, and only for whole rectangles of dense operands (a triangle's panels are shared
    // by both roles, and masked blocks are never packed whole).
    if (v == Variant::Fused && tri == gfip::TRI_NONE && !masked)
        pl.shared = h->packer == GFIP_PACKER_SHARED;

    // Which operands are packed, and how (Sec. 3.3 option table for the fused variant).
    switch (v) {
    case Variant::Direct:
        pl.mode_a = pl.mode_b = gfip::MODE_RAW;
        break;
    case Variant::PackThenCompute:
        pl.mode_a = pl.mode_b = gfip::MODE_PACKED;
        break;
    case Variant::Fused:
        switch (h->pack_policy) {
        case GFIP_PACK_NONE:
            pl.mode_a = pl.mode_b = gfip::MODE_RAW;
            break;
        case GFIP_PACK_A:
            pl.mode_a = gfip::MODE_FIP;
            pl.mode_b = gfip::MODE_RAW;
            break;
        case GFIP_PACK_B:
            pl.mode_a = gfip::MODE_RAW;
            pl.mode_b = gfip::MODE_FIP;
            break;
        case GFIP_PACK_BOTH:
            pl.mode_a = pl.mode_b = gfip::MODE_FIP;
            break;
        default:
            // AUTO: Sec. 3.3's table: an A panel is reused only across tile columns, a B
            // panel only across tile rows, so pack A iff there is more than one tile column
            // and B iff there is more than one tile row.  Whether a consumer finds a k-block
            // already published is decided at run time, per k-block (Sec. 3.2's cases).
            pl.mode_a = (pl.nt > 1) ? gfip::MODE_FIP : gfip::MODE_RAW;
            pl.mode_b = (pl.mt > 1) ? gfip::MODE_FIP : gfip::MODE_RAW;
            break;
        }
        break;
    }
    // (the count of packed tiles keeps twice their number in 32 bits)
    const int64_t units = (int64_t)((pl.mode_a == gfip::MODE_FIP ? pl.mt : 0) +
                                    (pl.mode_b == gfip::MODE_FIP ? pl.nt : 0)) * pl.kt;
    if (units == 0 || units >= (int64_t(1) << 30)) pl.shared = false;
    if (tri) {
        // SYRK: both operand roles read panels of the same matrix A, so one packed copy
        // serves both; any packing policy packs A's panels once (or not at all)
        const bool pack = (pl.mode_a != gfip::MODE_RAW) || (pl.mode_b != gfip::MODE_RAW);
        pl.mode_a = pl.mode_b = pack ? gfip::MODE_FIP : gfip::MODE_RAW;
    }

    // Control region: header, arrival counters of split tiles, ready words of packed tiles.
    size_t off = kHeader;
    pl.off_count = off;
    off += round_up((size_t)pl.tiles * 8, kAlign);
    pl.off_state_a = off;
    if (pl.mode_a == gfip::MODE_FIP) off += round_up((size_t)pl.mt * (pl.kt + 1) * 8, kAlign);
    pl.off_state_b = tri ? pl.off_state_a : off;
    if (pl.mode_b == gfip::MODE_FIP && !tri)
        off += round_up((size_t)pl.nt * (pl.kt + 1) * 8, kAlign);
    pl.ctrl_needed = off;

    // Data region (relative to its start): partial sums, packed A, packed B.
    size_t d = 0;
    pl.data_partial = d;
    if (pl.sk_iters > 0) d += round_up((size_t)pl.grid * 2 * Cfg::BM * Cfg::BN * sizeof(T), kAlign);
    pl.data_pack_a = d;
    if (pl.mode_a != gfip::MODE_RAW)
        d += round_up((size_t)pl.mt * pl.kt * Cfg::BM * Cfg::BK * sizeof(T), kAlign);
    pl.data_pack_b = tri ? pl.data_pack_a : d;
    if (pl.mode_b != gfip::MODE_RAW && !tri)
        d += round_up((size_t)pl.nt * pl.kt * Cfg::BN * Cfg::BK * sizeof(T), kAlign);
    pl.data_bytes = d;
    return pl;
}

template <typename T> size_t total_bytes(Handle *h, const Plan<T> &pl)
{
    const size_t ctrl = std::max(h->ctrl_bytes, round_up(pl.ctrl_needed, kCtrlGranule));
    return ctrl + pl.data_bytes;
}

// Grows the handle's control region to `want` bytes.  The new part may hold data of earlier
// calls, so it is cleared with a memset ordered on the handle's stream after them.  That
// memset must not be recorded into a CUDA graph: a replay would clear the launch counter and
// the ready words again while words of later eager calls kept their tags, so a stale word
// could read as ready.  A call that needs the clear therefore returns GFIP_ERR_CAPTURE, with
// nothing enqueued, when its stream is capturing.
int grow_ctrl(Handle *h, size_t want)
{
    if (want <= h->ctrl_bytes) return GFIP_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(h->stream, &cs) != cudaSuccess) return GFIP_ERR_CUDA;
    if (cs != cudaStreamCaptureStatusNone) return GFIP_ERR_CAPTURE;
    if (cudaMemsetAsync(h->ws + h->ctrl_bytes, 0, want - h->ctrl_bytes, h->stream) != cudaSuccess)
        return GFIP_ERR_CUDA;
    h->ctrl_bytes = want;
    return GFIP_OK;
}

bool too_big(int64_t v)
{
    return v > std::numeric_limits<int32_t>::max();
}

template <typename T>
int launch_plan(Handle *h, Variant v, int tri, char transa, char transb, int64_t m, int64_t n,
                int64_t k, T alpha, const T *A, int64_t lda, const T *B, int64_t ldb, T beta,
                T *C, int64_t ldc, int tmask_a = 0, int tmask_b = 0);

template <typename T>
int gemm_entry(gfip_handle_t handle, Variant v, char transa, char transb, int64_t m, int64_t n,
               int64_t k, T alpha, const T *A, int64_t lda, const T *B, int64_t ldb, T beta, T *C,
               int64_t ldc)
{
    const int info = check_args(transa, transb, m, n, k, lda, ldb, ldc);
    if (info != 0) return info;
    Handle *h = get(handle);
    if (h == nullptr) return GFIP_ERR_HANDLE;
    h->last_launches = 0;
    h->last_grid = 0;
    if (m == 0 || n == 0) return GFIP_OK;
    const bool use_ab = !(alpha == T(0) || k == 0);
    if (!use_ab && beta == T(1)) return GFIP_OK;
    if (too_big(m) || too_big(n) || too_big(k) || too_big(lda) || too_big(ldb) || too_big(ldc))
        return GFIP_ERR_SIZE;
    if (C == nullptr) return GFIP_ERR_NULLPTR;
    if (!use_ab) {
        if (gfip::launch_scale<T>(C, ldc, (int)m, (int)n, beta, gfip::TRI_NONE, h->stream) != cudaSuccess)
            return GFIP_ERR_CUDA;
        h->last_launches = 1;
        return GFIP_OK;
    }
    if (A == nullptr || B == nullptr) return GFIP_ERR_NULLPTR;
    return launch_plan<T>(h, v, gfip::TRI_NONE, transa, transb, m, n, k, alpha, A, lda, B, ldb,
                          beta, C, ldc);
}

// Plans and launches one GEMM (or the triangle `tri` of one) whose arguments are checked
// and whose quick returns are taken.
template <typename T>
int launch_plan(Handle *h, Variant v, int tri, char transa, char transb, int64_t m, int64_t n,
                int64_t k, T alpha, const T *A, int64_t lda, const T *B, int64_t ldb, T beta,
                T *C, int64_t ldc, int tmask_a, int tmask_b)
{
    Plan<T> pl = make_plan<T>(h, v, (int)m, (int)n, (int)k, tri, tmask_a || tmask_b);
    if (h->ws == nullptr) return GFIP_ERR_WORKSPACE;
    if (total_bytes(h, pl) > h->ws_bytes) return GFIP_ERR_WORKSPACE;

    // Grow the control region if this plan needs more of it.
    if (const int rc = grow_ctrl(h, round_up(pl.ctrl_needed, kCtrlGranule)); rc != GFIP_OK)
        return rc;

    unsigned char *data = h->ws + h->ctrl_bytes;
    gfip::GemmParams<T> p{};
    p.A = A;
    p.B = B;
    p.C = C;
    p.lda = lda;
    p.ldb = ldb;
    p.ldc = ldc;
    p.m = (int)m;
    p.n = (int)n;
    p.k = (int)k;
    p.alpha = alpha;
    p.beta = beta;
    p.a_contig_m = is_notrans(transa) ? 1 : 0;
    p.b_contig_n = is_notrans(transb) ? 0 : 1;
    p.mt = pl.mt;
    p.nt = pl.nt;
    p.kt = pl.kt;
    p.tiles = pl.tiles;
    // consumer bands of about sqrt(grid) tile rows: a wave spans ~sqrt(grid) panels each way
    p.band = std::max(1, std::min(pl.mt - 1, static_cast<int>(std::lround(std::sqrt(
                                                 static_cast<double>(pl.grid))))));
    p.grid = pl.grid;
    p.dp_tiles = pl.dp_tiles;
    p.sk_iters = pl.sk_iters;
    p.mode_a = pl.mode_a;
    p.mode_b = pl.mode_b;
    p.tri = tri;
    // the operand whose first tile line packs: A (first tile column) unless the triangle is
    // the upper one, whose first tile line is the first tile row (B's producers)
    p.a_produces = (tri != gfip::TRI_UPPER && !pl.shared) ? 1 : 0;
    p.b_produces = ((tri == gfip::TRI_NONE || tri == gfip::TRI_UPPER) && !pl.shared) ? 1 : 0;
    p.shared_pack = pl.shared ? 1 : 0;
    p.pack_units = pl.shared ? (int64_t)((pl.mode_a == gfip::MODE_FIP ? pl.mt : 0) +
                                         (pl.mode_b == gfip::MODE_FIP ? pl.nt : 0)) * pl.kt
                             : 0;
    p.tmask_a = tmask_a;
    p.tmask_b = tmask_b;
    p.state_a = reinterpret_cast<unsigned long long *>(h->ws + pl.off_state_a);
    p.state_b = reinterpret_cast<unsigned long long *>(h->ws + pl.off_state_b);
    p.tile_count = reinterpret_cast<unsigned long long *>(h->ws + pl.off_count);
    p.pack_a = reinterpret_cast<T *>(data + pl.data_pack_a);
    p.pack_b = reinterpret_cast<T *>(data + pl.data_pack_b);
    p.partial = reinterpret_cast<T *>(data + pl.data_partial);
    p.status = reinterpret_cast<unsigned int *>(h->ws);
    p.launch_count = reinterpret_cast<unsigned int *>(h->ws + kLaunchCountOffset);
    p.done_count = reinterpret_cast<unsigned int *>(h->ws + kDoneCountOffset);
    p.pack_count = reinterpret_cast<unsigned long long *>(h->ws + kPackCountOffset);
    p.tile_next = reinterpret_cast<unsigned long long *>(h->ws + kTileNextOffset);

    int launches = 0;
    if (v == Variant::PackThenCompute) {
        gfip::PackParams<T> pp{};
        pp.A = A;
        pp.B = B;
        pp.lda = lda;
        pp.ldb = ldb;
        pp.m = p.m;
        pp.n = p.n;
        pp.k = p.k;
        pp.a_contig_m = p.a_contig_m;
        pp.b_contig_n = p.b_contig_n;
        pp.mt = pl.mt;
        pp.nt = pl.nt;
        pp.kt = pl.kt;
        pp.pack_a = p.pack_a;
        pp.pack_b = p.pack_b;
        if (gfip::launch_pack<T>(pp, h->stream) != cudaSuccess) return GFIP_ERR_CUDA;
        ++launches;
    }
    if (gfip::launch_gemm<T>(p, h->stream) != cudaSuccess) return GFIP_ERR_CUDA;
    ++launches;
    h->last_launches = launches;
    h->last_grid = pl.grid;
    return GFIP_OK;
}

// Workspace of the tensor-core FP64 emulation: digit tiles and exponents after a control
// region of at least the header (which holds the status word).
struct OzPlan {
    int mt = 0, nt = 0, kt = 0, ks_a = 1, ks_b = 1;
    size_t off_ea = 0, off_eb = 0, off_sa = 0, off_sb = 0, data_bytes = 0;
};

OzPlan oz_plan(int64_t m, int64_t n, int64_t k, int slices)
{
    OzPlan o;
    o.mt = static_cast<int>((m + 127) / 128);
    o.nt = static_cast<int>((n + 127) / 128);
    o.kt = static_cast<int>((k + 63) / 64);
    // enough exponent-reduction blocks to cover the GPU (about 600), at most 64 k-ranges
    o.ks_a = std::max(1, std::min({64, o.kt, (600 + o.mt - 1) / std::max(1, o.mt)}));
    o.ks_b = std::max(1, std::min({64, o.kt, (600 + o.nt - 1) / std::max(1, o.nt)}));
    size_t d = 0;
    o.off_ea = d;
    d += round_up((size_t)o.ks_a * o.mt * 128 * sizeof(int), kAlign);
    o.off_eb = d;
    d += round_up((size_t)o.ks_b * o.nt * 128 * sizeof(int), kAlign);
    o.off_sa = d;
    d += (size_t)slices * o.mt * o.kt * 16384;
    o.off_sb = d;
    d += (size_t)slices * o.nt * o.kt * 16384;
    o.data_bytes = d;
    return o;
}

// Workspace layout of a grouped launch (after the control region): descriptors, per-rank
// units / split tiles / partial-sum elements, prefix sums, arrival counters, partial sums.
struct GroupedLayout {
    size_t desc = 0, units = 0, stiles = 0, pelems = 0, prefix = 0, counters = 0, partial = 0;
    size_t bytes = 0;
    int max_split_tiles = 0;
};

GroupedLayout grouped_layout(int count, int64_t split_elems, int es)
{
    GroupedLayout l;
    size_t d = 0;
    l.desc = d;
    d += round_up(gfip::grouped_desc_bytes(count, es), kAlign);
    l.units = d;
    d += round_up((size_t)count * sizeof(int), kAlign);
    l.stiles = d;
    d += round_up((size_t)count * sizeof(int), kAlign);
    l.pelems = d;
    d += round_up((size_t)count * sizeof(int64_t), kAlign);
    l.prefix = d;
    d += round_up(((size_t)count + 1) * sizeof(int), kAlign);
    // a split tile holds at least 2 x 16 x 16 partial sums
    l.max_split_tiles = static_cast<int>(std::min<int64_t>(split_elems / 512, 1 << 30));
    l.counters = d;
    d += round_up((size_t)l.max_split_tiles * sizeof(int) + sizeof(int), kAlign);
    l.partial = d;
    d += round_up((size_t)split_elems * es, kAlign);
    l.bytes = d;
    return l;
}

template <typename T>
size_t workspace_size_impl(Handle *h, char transa, char transb, int64_t m, int64_t n, int64_t k,
                           Variant v)
{
    if (check_args(transa, transb, m, n, k, is_notrans(transa) ? std::max<int64_t>(1, m)
                                                              : std::max<int64_t>(1, k),
                   is_notrans(transb) ? std::max<int64_t>(1, k) : std::max<int64_t>(1, n),
                   std::max<int64_t>(1, m)) != 0)
        return 0;
    if (too_big(m) || too_big(n) || too_big(k)) return 0;
    if (m == 0 || n == 0 || k == 0) return round_up(kHeader, kCtrlGranule);
    const Plan<T> pl = make_plan<T>(h, v, (int)m, (int)n, (int)k);
    return total_bytes(h, pl);
}

// Reference-BLAS dsyrk argument check: 0, or minus the 1-based position of the first bad
// argument in (uplo, trans, n, k, alpha, A, lda, beta, C, ldc).
int check_syrk(char uplo, char trans, int64_t n, int64_t k, int64_t lda, int64_t ldc)
{
    const bool up_ok = uplo == 'L' || uplo == 'l' || uplo == 'U' || uplo == 'u';
    const bool tr_ok = trans == 'N' || trans == 'n' || trans == 'T' || trans == 't' ||
                       trans == 'C' || trans == 'c';
    if (!up_ok) return -1;
    if (!tr_ok) return -2;
    if (n < 0) return -3;
    if (k < 0) return -4;
    const int64_t rows_a = is_notrans(trans) ? n : k;
    if (lda < std::max<int64_t>(1, rows_a)) return -7;
    if (ldc < std::max<int64_t>(1, n)) return -10;
    return 0;
}

// SYRK on the fused kernel: op(A) op(A)^T with the same matrix in both operand roles, only
// the tiles of the requested triangle, and one packed copy per panel of A serving both roles.
template <typename T>
int syrk_entry(gfip_handle_t handle, char uplo, char trans, int64_t n, int64_t k, T alpha,
               const T *A, int64_t lda, T beta, T *C, int64_t ldc)
{
    const int info = check_syrk(uplo, trans, n, k, lda, ldc);
    if (info != 0) return info;
    Handle *h = get(handle);
    if (h == nullptr) return GFIP_ERR_HANDLE;
    h->last_launches = 0;
    h->last_grid = 0;
    if (n == 0) return GFIP_OK;
    const bool use_ab = !(alpha == T(0) || k == 0);
    if (!use_ab && beta == T(1)) return GFIP_OK;
    if (too_big(n) || too_big(k) || too_big(lda) || too_big(ldc)) return GFIP_ERR_SIZE;
    if (C == nullptr) return GFIP_ERR_NULLPTR;
    const int tri = (uplo == 'L' || uplo == 'l') ? gfip::TRI_LOWER : gfip::TRI_UPPER;
    if (!use_ab) {
        if (gfip::launch_scale<T>(C, ldc, (int)n, (int)n, beta, tri, h->stream) != cudaSuccess)
            return GFIP_ERR_CUDA;
        h->last_launches = 1;
        return GFIP_OK;
    }
    if (A == nullptr) return GFIP_ERR_NULLPTR;
    // trans 'N': C = A A^T  -> op(A) = A ('N'), op(B) = A^T ('T' on the same storage);
    // trans 'T': C = A^T A  -> op(A) = A^T ('T'), op(B) = A ('N')
    const char ta = is_notrans(trans) ? 'N' : 'T';
    const char tb = is_notrans(trans) ? 'T' : 'N';
    return launch_plan<T>(h, Variant::Fused, tri, ta, tb, n, n, k, alpha, A, lda, A, lda, beta,
                          C, ldc);
}

template <typename T>
size_t syrk_workspace_impl(Handle *h, char uplo, char trans, int64_t n, int64_t k)
{
    const int64_t rows_a = is_notrans(trans) ? n : k;
    if (check_syrk(uplo, trans, n, k, std::max<int64_t>(1, rows_a), std::max<int64_t>(1, n)) !=
        0)
        return 0;
    if (too_big(n) || too_big(k)) return 0;
    if (n == 0 || k == 0) return round_up(kHeader, kCtrlGranule);
    const int tri = (uplo == 'L' || uplo == 'l') ? gfip::TRI_LOWER : gfip::TRI_UPPER;
    const Plan<T> pl = make_plan<T>(h, Variant::Fused, (int)n, (int)n, (int)k, tri);
    return total_bytes(h, pl);
}

// Reference-BLAS dtrmm argument check: 0, or minus the 1-based position of the first bad
// argument in (side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb).
int check_trmm(char side, char uplo, char transa, char diag, int64_t m, int64_t n, int64_t lda,
               int64_t ldb)
{
    const bool left = side == 'L' || side == 'l';
    if (!left && side != 'R' && side != 'r') return -1;
    if (uplo != 'L' && uplo != 'l' && uplo != 'U' && uplo != 'u') return -2;
    if (!is_notrans(transa) && transa != 'T' && transa != 't' && transa != 'C' &&
        transa != 'c')
        return -3;
    if (diag != 'U' && diag != 'u' && diag != 'N' && diag != 'n') return -4;
    if (m < 0) return -5;
    if (n < 0) return -6;
    if (lda < std::max<int64_t>(1, left ? m : n)) return -9;
    if (ldb < std::max<int64_t>(1, m)) return -11;
    return 0;
}

// The triangle mask of op(A) in the operand role TRMM gives it (see gfip::TriMask): the
// A role of side 'L' (x = row i, k = p: lower op(A) keeps i >= p), the B role of side 'R'
// (x = column j, k = p: lower op(A) keeps p >= j); a unit diagonal makes it strict.
int trmm_mask(char side, char uplo, char transa, char diag)
{
    const bool left = side == 'L' || side == 'l';
    const bool lower_op = (uplo == 'L' || uplo == 'l') != !is_notrans(transa);
    int mask = gfip::TMASK_ON;
    if (diag == 'U' || diag == 'u') mask |= gfip::TMASK_STRICT;
    if (left ? lower_op : !lower_op) mask |= gfip::TMASK_KEEP_GE;
    return mask;
}

template <typename T>
size_t trmm_workspace_impl(Handle *h, char side, int64_t m, int64_t n)
{
    const bool left = side == 'L' || side == 'l';
    const Plan<T> pl =
        make_plan<T>(h, Variant::Fused, (int)m, (int)n, (int)(left ? m : n), gfip::TRI_NONE, true);
    return round_up(total_bytes(h, pl), kAlign) + round_up((size_t)m * n * sizeof(T), kAlign);
}

// TRMM on the fused kernel: W := alpha op(A) B (or alpha B op(A)) with op(A) read through a
// triangular mask (blocks outside the triangle skipped, blocks on the diagonal masked as
// they are staged, so the producers pack masked panels), a unit diagonal added as beta =
// alpha on a copy of B in W; then B := W.  W lives in the workspace after the GEMM's part.
template <typename T>
int trmm_entry(gfip_handle_t handle, char side, char uplo, char transa, char diag, int64_t m,
               int64_t n, T alpha, const T *A, int64_t lda, T *B, int64_t ldb)
{
    const int info = check_trmm(side, uplo, transa, diag, m, n, lda, ldb);
    if (info != 0) return info;
    Handle *h = get(handle);
    if (h == nullptr) return GFIP_ERR_HANDLE;
    h->last_launches = 0;
    h->last_grid = 0;
    if (m == 0 || n == 0) return GFIP_OK;
    if (too_big(m) || too_big(n) || too_big(lda) || too_big(ldb)) return GFIP_ERR_SIZE;
    if (B == nullptr) return GFIP_ERR_NULLPTR;
    if (alpha == T(0)) {   // B := 0, neither A nor B read
        if (gfip::launch_scale<T>(B, ldb, (int)m, (int)n, T(0), gfip::TRI_NONE, h->stream) !=
            cudaSuccess)
            return GFIP_ERR_CUDA;
        h->last_launches = 1;
        return GFIP_OK;
    }
    if (A == nullptr) return GFIP_ERR_NULLPTR;
    if (h->ws == nullptr) return GFIP_ERR_WORKSPACE;
    const bool left = side == 'L' || side == 'l';
    const bool unit = diag == 'U' || diag == 'u';
    const int64_t kdim = left ? m : n;
    const Plan<T> pl =
        make_plan<T>(h, Variant::Fused, (int)m, (int)n, (int)kdim, gfip::TRI_NONE, true);
    const size_t w_off = round_up(total_bytes(h, pl), kAlign);
    const size_t w_bytes = (size_t)m * n * sizeof(T);
    if (w_off + w_bytes > h->ws_bytes) return GFIP_ERR_WORKSPACE;
    T *W = reinterpret_cast<T *>(h->ws + w_off);
    const size_t row_bytes = (size_t)m * sizeof(T);
    if (unit && cudaMemcpy2DAsync(W, row_bytes, B, (size_t)ldb * sizeof(T), row_bytes, (size_t)n,
                                  cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
        return GFIP_ERR_CUDA;
    const T beta = unit ? alpha : T(0);
    const int mask = trmm_mask(side, uplo, transa, diag);
    const char ta = is_notrans(transa) ? 'N' : 'T';
    const int rc = left ? launch_plan<T>(h, Variant::Fused, gfip::TRI_NONE, ta, 'N', m, n, m,
                                         alpha, A, lda, B, ldb, beta, W, m, mask, 0)
                        : launch_plan<T>(h, Variant::Fused, gfip::TRI_NONE, 'N', ta, m, n, n,
                                         alpha, B, ldb, A, lda, beta, W, m, 0, mask);
    if (rc != GFIP_OK) return rc;
    if (cudaMemcpy2DAsync(B, (size_t)ldb * sizeof(T), W, row_bytes, row_bytes, (size_t)n,
                          cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
        return GFIP_ERR_CUDA;
    return GFIP_OK;
}

template <typename T>
size_t trsm_workspace_impl(Handle *h, char side, int64_t m, int64_t n)
{
    // every update is at most all of B (m x n) against one panel of unknowns, and its plan's
    // workspace grows with each dimension
    const bool left = side == 'L' || side == 'l';
    const int na = (int)(left ? m : n);
    const Plan<T> panel =
        make_plan<T>(h, Variant::Fused, (int)m, (int)n, std::min(gfip::TRSM_PANEL, na));
    return total_bytes(h, panel);
}

// TRSM, blocked: B := alpha B, then over panels of op(A)'s diagonal in solve order (forward
// for a lower triangular system, backward for an upper one; for side 'R' the system of each
// row of X is op(A)^T): solve the panel's unknowns for every right-hand side in one launch
// (trsm::panel_kernel), then subtract their contribution from the unknowns still to be
// solved with one fused GEMM (alpha = -1, beta = 1, k = the panel's width) that packs the
// solved rows of X (and the panel of op(A)) once for all its tiles.  Only the triangle of A
// is read.
template <typename T>
int trsm_entry(gfip_handle_t handle, char side, char uplo, char transa, char diag, int64_t m,
               int64_t n, T alpha, const T *A, int64_t lda, T *B, int64_t ldb)
{
    const int info = check_trmm(side, uplo, transa, diag, m, n, lda, ldb);
    if (info != 0) return info;
    Handle *h = get(handle);
    if (h == nullptr) return GFIP_ERR_HANDLE;
    h->last_launches = 0;
    h->last_grid = 0;
    if (m == 0 || n == 0) return GFIP_OK;
    if (too_big(m) || too_big(n) || too_big(lda) || too_big(ldb)) return GFIP_ERR_SIZE;
    if (B == nullptr) return GFIP_ERR_NULLPTR;
    if (alpha != T(0)) {
        // every check before the first launch
        if (A == nullptr) return GFIP_ERR_NULLPTR;
        if (h->ws == nullptr) return GFIP_ERR_WORKSPACE;
        if (trsm_workspace_impl<T>(h, side, m, n) > h->ws_bytes) return GFIP_ERR_WORKSPACE;
    }
    if (alpha != T(1)) {   // B := alpha B (alpha == 0: zeros, B not read)
        if (gfip::launch_scale<T>(B, ldb, (int)m, (int)n, alpha, gfip::TRI_NONE, h->stream) !=
            cudaSuccess)
            return GFIP_ERR_CUDA;
        if (alpha == T(0)) return GFIP_OK;
    }
    if (A == nullptr) return GFIP_ERR_NULLPTR;
    const bool left = side == 'L' || side == 'l';
    const bool trans = !is_notrans(transa);
    const bool lower_op = (uplo == 'L' || uplo == 'l') != trans;
    const bool lower_t = left ? lower_op : !lower_op;
    const bool unit = diag == 'U' || diag == 'u';
    const int na = (int)(left ? m : n);
    const char ta = trans ? 'T' : 'N';
    // B[rest] -= op(A)[rest, k0:k0+kb] X[k0:k0+kb] for the unknowns r0..r1-1 (side L), or
    // B[:, rest] -= X[:, k0:k0+kb] op(A)[k0:k0+kb, rest] (side R)
    auto update = [&](int k0, int kb, int r0, int r1) -> int {
        if (r1 <= r0) return GFIP_OK;
        if (left) {
            const T *ap = trans ? A + k0 + (int64_t)r0 * lda : A + r0 + (int64_t)k0 * lda;
            return launch_plan<T>(h, Variant::Fused, gfip::TRI_NONE, ta, 'N', r1 - r0, n, kb,
                                  T(-1), ap, lda, B + k0, ldb, T(1), B + r0, ldb);
        }
        const T *ap = trans ? A + r0 + (int64_t)k0 * lda : A + k0 + (int64_t)r0 * lda;
        return launch_plan<T>(h, Variant::Fused, gfip::TRI_NONE, 'N', ta, m, r1 - r0, kb,
                              T(-1), B + (int64_t)k0 * ldb, ldb, ap, lda, T(1),
                              B + (int64_t)r0 * ldb, ldb);
    };
    const int npanels = (na + gfip::TRSM_PANEL - 1) / gfip::TRSM_PANEL;
    for (int ps = 0; ps < npanels; ++ps) {
        const int pi = lower_t ? ps : npanels - 1 - ps;
        const int p0 = pi * gfip::TRSM_PANEL;
        const int pw = std::min(gfip::TRSM_PANEL, na - p0);
        // the panel's unknowns: rows p0.. of B (side L) or its columns p0.. (side R)
        const cudaError_t e =
            left ? gfip::launch_trsm_panel<T>(B + p0, ldb, 1, (int)n, A, lda, trans, p0, pw,
                                              lower_t, 0, unit, h->stream)
                 : gfip::launch_trsm_panel<T>(B + (int64_t)p0 * ldb, 1, ldb, (int)m, A, lda,
                                              trans, p0, pw, lower_t, 1, unit, h->stream);
        if (e != cudaSuccess) return GFIP_ERR_CUDA;
        const int rc = lower_t ? update(p0, pw, p0 + pw, na) : update(p0, pw, 0, p0);
        if (rc != GFIP_OK) return rc;
    }
    return GFIP_OK;
}

}  // namespace

extern "C" {

int gfip_create(gfip_handle_t *handle)
{
    if (handle == nullptr) return GFIP_ERR_ARG;
    *handle = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GFIP_ERR_CUDA;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return GFIP_ERR_CUDA;
    if (!(prop.major == 10 && prop.minor == 3)) return GFIP_ERR_DEVICE;
    Handle *h = new (std::nothrow) Handle();
    if (h == nullptr) return GFIP_ERR_ARG;
    h->device = dev;
    h->sms = prop.multiProcessorCount;
    *handle = reinterpret_cast<gfip_handle_t>(h);
    return GFIP_OK;
}

int gfip_destroy(gfip_handle_t handle)
{
    Handle *h = get(handle);
    if (h == nullptr) return GFIP_ERR_HANDLE;
    h->magic = 0;
    delete h;
    return GFIP_OK;
}

int gfip_set_stream(gfip_handle_t handle, void *stream)
{
    Handle *h = get(handle);
    if (h == nullptr) return GFIP_ERR_HANDLE;
    h->stream = reinterpret_cast<cudaStream_t>(stream);
    return GFIP_OK;
}

size_t gfip_workspace_size(gfip_handle_t handle, char transa, char transb, int64_t m, int64_t n,
                           int64_t k, int elem_bytes)
{
    Handle *h = get(handle);
    if (h == nullptr) return 0;
    // The largest of the three variants, so one workspace serves all of them.
    if (elem_bytes == 8) {
        size_t s = 0;
        for (Variant v : {Variant::Fused, Variant::Direct, Variant::PackThenCompute}) {
            const int saved = h->pack_policy;
            if (v == Variant::Fused) h->pack_policy = GFIP_PACK_BOTH;
            s = std::max(s, workspace_size_impl<double>(h, transa, transb, m, n, k, v));
            h->pack_policy = saved;
        }
        return s;
    }
    if (elem_bytes == 4) {
        size_t s = 0;
        for (Variant v : {Variant::Fused, Variant::Direct, Variant::PackThenCompute}) {
            const int saved = h->pack_policy;
            if (v == Variant::Fused) h->pack_policy = GFIP_PACK_BOTH;
            s = std::max(s, workspace_size_impl<float>(h, transa, transb, m, n, k, v));
            h->pack_policy = saved;
        }
        return s;
    }
    return 0;
}

int gfip_set_workspace(gfip_handle_t handle, void *dev_ptr, size_t bytes)
{
    Handle *h = get(handle);
    if (h == nullptr) return GFIP_ERR_HANDLE;
    if (dev_ptr != nullptr && (reinterpret_cast<uintptr_t>(dev_ptr) % 16) != 0) return GFIP_ERR_ARG;
    h->ws = reinterpret_cast<unsigned char *>(dev_ptr);
    h->ws_bytes = dev_ptr ? bytes : 0;
    h->ctrl_bytes = 0;
    return GFIP_OK;
}

int gfip_debug_ozaki_timeout(gfip_handle_t handle, int enable, uint64_t wait_ns)
{
    Handle *h = get(handle);
    if (h == nullptr) return GFIP_ERR_HANDLE;
    h->oz_inject = enable ? 1 : 0;
    h->oz_wait_ns = wait_ns ? wait_ns : kOzakiWaitNs;
    return GFIP_OK;
}

int gfip_set_pack_policy(gfip_handle_t handle, int policy)
{
    Handle *h = get(handle);
    if (h == nullptr) return GFIP_ERR_HANDLE;
    if (policy < GFIP_PACK_AUTO || policy > GFIP_PACK_BOTH) return GFIP_ERR_ARG;
    h->pack_policy = policy;
    return GFIP_OK;
}

int gfip_set_packer(gfip_handle_t handle, int packer)
{
    Handle *h = get(handle);
    if (h == nullptr) return GFIP_ERR_HANDLE;
    if (packer < GFIP_PACKER_AUTO || packer > GFIP_PACKER_SHARED) return GFIP_ERR_ARG;
    h->packer = packer;
    return GFIP_OK;
}

size_t gfip_syrk_workspace_size(gfip_handle_t handle, char uplo, char trans, int64_t n,
                                int64_t k, int elem_bytes)
{
    Handle *h = get(handle);
    if (h == nullptr) return 0;
    if (elem_bytes == 8) return syrk_workspace_impl<double>(h, uplo, trans, n, k);
    if (elem_bytes == 4) return syrk_workspace_impl<float>(h, uplo, trans, n, k);
    return 0;
}

int gfip_dsyrk(gfip_handle_t handle, char uplo, char trans, int64_t n, int64_t k, double alpha,
               const double *A, int64_t lda, double beta, double *C, int64_t ldc)
{
    return syrk_entry<double>(handle, uplo, trans, n, k, alpha, A, lda, beta, C, ldc);
}

int gfip_ssyrk(gfip_handle_t handle, char uplo, char trans, int64_t n, int64_t k, float alpha,
               const float *A, int64_t lda, float beta, float *C, int64_t ldc)
{
    return syrk_entry<float>(handle, uplo, trans, n, k, alpha, A, lda, beta, C, ldc);
}

size_t gfip_trmm_workspace_size(gfip_handle_t handle, char side, char uplo, char transa,
                                char diag, int64_t m, int64_t n, int elem_bytes)
{
    Handle *h = get(handle);
    if (h == nullptr) return 0;
    const bool left = side == 'L' || side == 'l';
    if (check_trmm(side, uplo, transa, diag, m, n, std::max<int64_t>(1, left ? m : n),
                   std::max<int64_t>(1, m)) != 0)
        return 0;
    if (too_big(m) || too_big(n)) return 0;
    if (m == 0 || n == 0) return round_up(kHeader, kCtrlGranule);
    if (elem_bytes == 8) return trmm_workspace_impl<double>(h, side, m, n);
    if (elem_bytes == 4) return trmm_workspace_impl<float>(h, side, m, n);
    return 0;
}

int gfip_dtrmm(gfip_handle_t handle, char side, char uplo, char transa, char diag, int64_t m,
               int64_t n, double alpha, const double *A, int64_t lda, double *B, int64_t ldb)
{
    return trmm_entry<double>(handle, side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb);
}

int gfip_strmm(gfip_handle_t handle, char side, char uplo, char transa, char diag, int64_t m,
               int64_t n, float alpha, const float *A, int64_t lda, float *B, int64_t ldb)
{
    return trmm_entry<float>(handle, side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb);
}

size_t gfip_trsm_workspace_size(gfip_handle_t handle, char side, char uplo, char transa,
                                char diag, int64_t m, int64_t n, int elem_bytes)
{
    Handle *h = get(handle);
    if (h == nullptr) return 0;
    const bool left = side == 'L' || side == 'l';
    if (check_trmm(side, uplo, transa, diag, m, n, std::max<int64_t>(1, left ? m : n),
                   std::max<int64_t>(1, m)) != 0)
        return 0;
    if (too_big(m) || too_big(n)) return 0;
    if (m == 0 || n == 0) return round_up(kHeader, kCtrlGranule);
    if (elem_bytes == 8) return trsm_workspace_impl<double>(h, side, m, n);
    if (elem_bytes == 4) return trsm_workspace_impl<float>(h, side, m, n);
    return 0;
}

int gfip_dtrsm(gfip_handle_t handle, char side, char uplo, char transa, char diag, int64_t m,
               int64_t n, double alpha, const double *A, int64_t lda, double *B, int64_t ldb)
{
    return trsm_entry<double>(handle, side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb);
}

int gfip_strsm(gfip_handle_t handle, char side, char uplo, char transa, char diag, int64_t m,
               int64_t n, float alpha, const float *A, int64_t lda, float *B, int64_t ldb)
{
    return trsm_entry<float>(handle, side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb);
}

int gfip_dgemm(gfip_handle_t handle, char transa, char transb, int64_t m, int64_t n, int64_t k,
               double alpha, const double *A, int64_t lda, const double *B, int64_t ldb,
               double beta, double *C, int64_t ldc)
{
    return gemm_entry<double>(handle, Variant::Fused, transa, transb, m, n, k, alpha, A, lda, B,
                              ldb, beta, C, ldc);
}

int gfip_sgemm(gfip_handle_t handle, char transa, char transb, int64_t m, int64_t n, int64_t k,
               float alpha, const float *A, int64_t lda, const float *B, int64_t ldb, float beta,
               float *C, int64_t ldc)
{
    return gemm_entry<float>(handle, Variant::Fused, transa, transb, m, n, k, alpha, A, lda, B,
                             ldb, beta, C, ldc);
}

int gfip_dgemm_direct(gfip_handle_t handle, char transa, char transb, int64_t m, int64_t n,
                      int64_t k, double alpha, const double *A, int64_t lda, const double *B,
                      int64_t ldb, double beta, double *C, int64_t ldc)
{
    return gemm_entry<double>(handle, Variant::Direct, transa, transb, m, n, k, alpha, A, lda,
                              B, ldb, beta, C, ldc);
}

int gfip_sgemm_direct(gfip_handle_t handle, char transa, char transb, int64_t m, int64_t n,
                      int64_t k, float alpha, const float *A, int64_t lda, const float *B,
                      int64_t ldb, float beta, float *C, int64_t ldc)
{
    return gemm_entry<float>(handle, Variant::Direct, transa, transb, m, n, k, alpha, A, lda, B,
                             ldb, beta, C, ldc);
}

int gfip_dgemm_pack_then_compute(gfip_handle_t handle, char transa, char transb, int64_t m,
                                 int64_t n, int64_t k, double alpha, const double *A,
                                 int64_t lda, const double *B, int64_t ldb, double beta,
                                 double *C, int64_t ldc)
{
    return gemm_entry<double>(handle, Variant::PackThenCompute, transa, transb, m, n, k, alpha, A,
                              lda, B, ldb, beta, C, ldc);
}

int gfip_sgemm_pack_then_compute(gfip_handle_t handle, char transa, char transb, int64_t m,
                                 int64_t n, int64_t k, float alpha, const float *A, int64_t lda,
                                 const float *B, int64_t ldb, float beta, float *C,
                                 int64_t ldc)
{
    return gemm_entry<float>(handle, Variant::PackThenCompute, transa, transb, m, n, k, alpha, A,
                             lda, B, ldb, beta, C, ldc);
}

int gfip_get_status(gfip_handle_t handle, uint32_t *status)
{
    Handle *h = get(handle);
    if (h == nullptr) return GFIP_ERR_HANDLE;
    if (status == nullptr) return GFIP_ERR_ARG;
    if (h->ws == nullptr) return GFIP_ERR_WORKSPACE;
    *status = 0;
    if (h->ctrl_bytes == 0) return GFIP_OK;  // no kernel has written a status yet
    uint32_t v = 0;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return GFIP_ERR_CUDA;
    if (cudaMemcpy(&v, h->ws, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess)
        return GFIP_ERR_CUDA;
    if (cudaMemsetAsync(h->ws, 0, sizeof(v), h->stream) != cudaSuccess) return GFIP_ERR_CUDA;
    *status = v;
    return GFIP_OK;
}

int gfip_last_launch_info(gfip_handle_t handle, int *launches, int *grid)
{
    Handle *h = get(handle);
    if (h == nullptr) return GFIP_ERR_HANDLE;
    if (launches) *launches = h->last_launches;
    if (grid) *grid = h->last_grid;
    return GFIP_OK;
}

const char *gfip_error_string(int code)
{
    if (code < 0) {
        switch (code) {
        case -1: return "invalid argument 1 (transa of gemm, uplo of syrk)";
        case -2: return "invalid argument 2 (transb of gemm, trans of syrk)";
        case -3: return "invalid argument 3 (m < 0 of gemm, n < 0 of syrk)";
        case -4: return "invalid argument 4 (n < 0 of gemm, k < 0 of syrk)";
        case -5: return "invalid argument 5 (k < 0)";
        case -8: return "invalid argument 8 (lda < max(1, rows of A))";
        case -7: return "invalid argument 7 (lda of syrk < max(1, rows of A))";
        case -10: return "invalid argument 10 (ldb of gemm < max(1, rows of B), ldc of syrk < max(1, n))";
        case -13: return "invalid argument 13 (ldc < max(1, m))";
        default: return "invalid argument";
        }
    }
    switch (code) {
    case GFIP_OK: return "success";
    case GFIP_ERR_HANDLE: return "invalid handle";
    case GFIP_ERR_CUDA: return "CUDA runtime error";
    case GFIP_ERR_WORKSPACE: return "workspace missing or too small";
    case GFIP_ERR_NULLPTR: return "null matrix pointer";
    case GFIP_ERR_DEVICE: return "device is not sm_103";
    case GFIP_ERR_SIZE: return "dimension exceeds 2^31-1";
    case GFIP_ERR_ARG: return "invalid argument value";
    case GFIP_ERR_SCRATCH_LIMIT:
        return "problem needs more scratch than the allocation-free routine's static array";
    case GFIP_ERR_CAPTURE:
        return "the call must clear control words first, which cannot happen while its stream "
               "is capturing a CUDA graph";
    default: return "unknown error";
    }
}

size_t gfip_grouped_workspace_size(gfip_handle_t handle, int count)
{
    Handle *h = get(handle);
    if (h == nullptr || count < 0) return 0;
    return std::max(h->ctrl_bytes, kCtrlGranule) + grouped_layout(count, 0, 8).bytes;
}

size_t gfip_ozaki_workspace_size(gfip_handle_t handle, int64_t m, int64_t n, int64_t k,
                                 int slices)
{
    Handle *h = get(handle);
    if (h == nullptr || m < 0 || n < 0 || k < 0 || slices < 1 || slices > 10) return 0;
    const OzPlan o = oz_plan(m, n, k, slices);
    return std::max(h->ctrl_bytes, kCtrlGranule) + o.data_bytes;
}

int gfip_dgemm_ozaki(gfip_handle_t handle, char transa, char transb, int64_t m, int64_t n,
                     int64_t k, double alpha, const double *A, int64_t lda, const double *B,
                     int64_t ldb, double beta, double *C, int64_t ldc, int slices)
{
    const int info = check_args(transa, transb, m, n, k, lda, ldb, ldc);
    if (info != 0) return info;
    Handle *h = get(handle);
    if (h == nullptr) return GFIP_ERR_HANDLE;
    if (slices < 1 || slices > 10) return GFIP_ERR_ARG;
    h->last_launches = 0;
    h->last_grid = 0;
    if (m == 0 || n == 0) return GFIP_OK;
    const bool use_ab = !(alpha == 0.0 || k == 0);
    if (!use_ab && beta == 1.0) return GFIP_OK;
    if (too_big(m) || too_big(n) || too_big(k)) return GFIP_ERR_SIZE;
    if (C == nullptr) return GFIP_ERR_NULLPTR;
    if (!use_ab) {
        if (gfip::launch_scale<double>(C, ldc, (int)m, (int)n, beta, gfip::TRI_NONE, h->stream) != cudaSuccess)
            return GFIP_ERR_CUDA;
        h->last_launches = 1;
        return GFIP_OK;
    }
    if (A == nullptr || B == nullptr) return GFIP_ERR_NULLPTR;
    if (h->ws == nullptr) return GFIP_ERR_WORKSPACE;
    const OzPlan o = oz_plan(m, n, k, slices);
    const size_t ctrl_want = std::max(h->ctrl_bytes, kCtrlGranule);
    if (ctrl_want + o.data_bytes > h->ws_bytes) return GFIP_ERR_WORKSPACE;
    if (const int rc = grow_ctrl(h, ctrl_want); rc != GFIP_OK) return rc;
    unsigned char *data = h->ws + h->ctrl_bytes;
    gfip::OzakiParams p{};
    p.A = A;
    p.B = B;
    p.C = C;
    p.lda = lda;
    p.ldb = ldb;
    p.ldc = ldc;
    p.m = (int)m;
    p.n = (int)n;
    p.k = (int)k;
    p.alpha = alpha;
    p.beta = beta;
    p.a_contig_rows = is_notrans(transa) ? 1 : 0;
    p.b_contig_rows = is_notrans(transb) ? 0 : 1;
    p.slices = slices;
    p.mt = o.mt;
    p.nt = o.nt;
    p.kt = o.kt;
    p.ks_a = o.ks_a;
    p.ks_b = o.ks_b;
    p.ea = reinterpret_cast<int *>(data + o.off_ea);
    p.eb = reinterpret_cast<int *>(data + o.off_eb);
    p.sa = reinterpret_cast<uint16_t *>(data + o.off_sa);
    p.sb = reinterpret_cast<uint16_t *>(data + o.off_sb);
    p.status = reinterpret_cast<unsigned int *>(h->ws);
    p.wait_ns = h->oz_wait_ns;
    p.inject_timeout = h->oz_inject;
    if (gfip::launch_ozaki(p, h->stream) != cudaSuccess) return GFIP_ERR_CUDA;
    h->last_launches = 5;
    h->last_grid = o.mt * o.nt;
    return GFIP_OK;
}

}  // extern "C"


namespace {

template <typename T>
int grouped_entry(gfip_handle_t handle, int count, const char *transa, const char *transb,
                  const int *m, const int *n, const int *k, const T *alpha, const T *const *A,
                  const int64_t *lda, const T *const *B, const int64_t *ldb, const T *beta,
                  T *const *C, const int64_t *ldc, int tile, const int *plan, const int *order,
                  int64_t split_elems)
{
    Handle *h = get(handle);
    if (h == nullptr) return GFIP_ERR_HANDLE;
    if (count < 0 || tile < GFIP_GROUP_TILE_DEFAULT || tile > GFIP_GROUP_TILE_8X16 ||
        split_elems < 0)
        return GFIP_ERR_ARG;
    h->last_launches = 0;
    h->last_grid = 0;
    if (count == 0) return GFIP_OK;
    if (!transa || !transb || !m || !n || !k || !alpha || !A || !lda || !B || !ldb || !beta ||
        !C || !ldc)
        return GFIP_ERR_NULLPTR;
    if (h->ws == nullptr) return GFIP_ERR_WORKSPACE;
    const GroupedLayout l = grouped_layout(count, split_elems, static_cast<int>(sizeof(T)));
    const size_t ctrl_want = std::max(h->ctrl_bytes, kCtrlGranule);
    if (ctrl_want + l.bytes > h->ws_bytes) return GFIP_ERR_WORKSPACE;
    if (const int rc = grow_ctrl(h, ctrl_want); rc != GFIP_OK) return rc;
    unsigned char *data = h->ws + h->ctrl_bytes;
    gfip::GroupParams<T> gp{};
    gp.count = count;
    gp.transa = transa;
    gp.transb = transb;
    gp.m = m;
    gp.n = n;
    gp.k = k;
    gp.alpha = alpha;
    gp.beta = beta;
    gp.A = A;
    gp.B = B;
    gp.C = C;
    gp.lda = lda;
    gp.ldb = ldb;
    gp.ldc = ldc;
    gp.plan = plan;
    gp.order = order;
    gp.uniform_shape = tile;
    gp.desc = reinterpret_cast<gfip::GroupDesc<T> *>(data + l.desc);
    gp.units = reinterpret_cast<int *>(data + l.units);
    gp.stiles = reinterpret_cast<int *>(data + l.stiles);
    gp.pelems = reinterpret_cast<int64_t *>(data + l.pelems);
    gp.prefix = reinterpret_cast<int *>(data + l.prefix);
    gp.counters = reinterpret_cast<int *>(data + l.counters);
    gp.max_split_tiles = l.max_split_tiles;
    gp.partial = reinterpret_cast<T *>(data + l.partial);
    gp.partial_capacity = split_elems;
    gp.status = reinterpret_cast<unsigned int *>(h->ws);
    if (gfip::launch_grouped<T>(gp, h->stream) != cudaSuccess) return GFIP_ERR_CUDA;
    h->last_launches = 3;
    return GFIP_OK;
}

}  // namespace

extern "C" {

int gfip_dgemm_grouped(gfip_handle_t handle, int count, const char *transa, const char *transb,
                       const int *m, const int *n, const int *k, const double *alpha,
                       const double *const *A, const int64_t *lda, const double *const *B,
                       const int64_t *ldb, const double *beta, double *const *C,
                       const int64_t *ldc, int tile)
{
    return grouped_entry<double>(handle, count, transa, transb, m, n, k, alpha, A, lda, B, ldb,
                                 beta, C, ldc, tile, nullptr, nullptr, 0);
}

int gfip_sgemm_grouped(gfip_handle_t handle, int count, const char *transa, const char *transb,
                       const int *m, const int *n, const int *k, const float *alpha,
                       const float *const *A, const int64_t *lda, const float *const *B,
                       const int64_t *ldb, const float *beta, float *const *C,
                       const int64_t *ldc, int tile)
{
    return grouped_entry<float>(handle, count, transa, transb, m, n, k, alpha, A, lda, B, ldb,
                                beta, C, ldc, tile, nullptr, nullptr, 0);
}

size_t gfip_grouped_plan_workspace_size(gfip_handle_t handle, int count, int64_t split_elems,
                                        int elem_bytes)
{
    Handle *h = get(handle);
    if (h == nullptr || count < 0 || split_elems < 0 || (elem_bytes != 4 && elem_bytes != 8))
        return 0;
    return std::max(h->ctrl_bytes, kCtrlGranule) +
           grouped_layout(count, split_elems, elem_bytes).bytes;
}

int gfip_dgemm_grouped_plan(gfip_handle_t handle, int count, const char *transa,
                            const char *transb, const int *m, const int *n, const int *k,
                            const double *alpha, const double *const *A, const int64_t *lda,
                            const double *const *B, const int64_t *ldb, const double *beta,
                            double *const *C, const int64_t *ldc, const int *plan,
                            const int *order, int64_t split_elems)
{
    if (plan == nullptr) return GFIP_ERR_NULLPTR;
    return grouped_entry<double>(handle, count, transa, transb, m, n, k, alpha, A, lda, B, ldb,
                                 beta, C, ldc, 0, plan, order, split_elems);
}

int gfip_sgemm_grouped_plan(gfip_handle_t handle, int count, const char *transa,
                            const char *transb, const int *m, const int *n, const int *k,
                            const float *alpha, const float *const *A, const int64_t *lda,
                            const float *const *B, const int64_t *ldb, const float *beta,
                            float *const *C, const int64_t *ldc, const int *plan,
                            const int *order, int64_t split_elems)
{
    if (plan == nullptr) return GFIP_ERR_NULLPTR;
    return grouped_entry<float>(handle, count, transa, transb, m, n, k, alpha, A, lda, B, ldb,
                                beta, C, ldc, 0, plan, order, split_elems);
}

}  // extern "C"

// ---- Allocation-free entry point ---------------------------------------------------------
// Scratch of gfip_dgemm_noalloc: one static device array per GPU that loads this library.
// In host code `g_noalloc_scratch` is only a stand-in symbol, never a device address; the
// address comes from cudaGetSymbolAddress at set-up.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GFIP_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kNoAllocMaxDevices = 64;

struct NoAllocDevice {
    std::mutex mu;          // serialises host-side use of this device's state
    bool ready = false;
    Handle h;               // static-storage handle whose workspace is the static array
};

NoAllocDevice g_noalloc[kNoAllocMaxDevices];

// Set-up for the current device: check the device once, then on every call look up the
// array's device address with that device current (cheap).  If the address changed -- the
// device's context was destroyed and created again, which loads the module anew -- the
// control words recorded as cleared belong to the old array, so the handle starts over with
// an empty control region; the next call clears it on its stream.
int noalloc_setup(NoAllocDevice &d, int dev)
{
    if (!d.ready) {
        int major = 0, minor = 0, sms = 0;
        if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return GFIP_ERR_CUDA;
        if (!(major == 10 && minor == 3)) return GFIP_ERR_DEVICE;
        d.h.device = dev;
        d.h.sms = sms;
        d.h.ws_bytes = GFIP_NOALLOC_SCRATCH_BYTES;
        d.h.pack_policy = GFIP_PACK_AUTO;
    }
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr)
        return GFIP_ERR_CUDA;
    if (!d.ready || d.h.ws != ptr) {
        d.h.ws = reinterpret_cast<unsigned char *>(ptr);
        d.h.ctrl_bytes = 0;
        d.h.bps_f64 = 0;
        d.h.bps_f32 = 0;
    }
    d.ready = true;
    return GFIP_OK;
}

}  // namespace

extern "C" int gfip_dgemm_noalloc(char transa, char transb, int64_t m, int64_t n, int64_t k,
                                  double alpha, const double *A, int64_t lda, const double *B,
                                  int64_t ldb, double beta, double *C, int64_t ldc, void *stream)
{
    const int info = check_args(transa, transb, m, n, k, lda, ldb, ldc);
    if (info != 0) return info;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GFIP_ERR_CUDA;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return GFIP_ERR_DEVICE;
    NoAllocDevice &d = g_noalloc[dev];
    std::lock_guard<std::mutex> lock(d.mu);
    const int rc = noalloc_setup(d, dev);
    if (rc != GFIP_OK) return rc;
    d.h.stream = reinterpret_cast<cudaStream_t>(stream);
    // Reject, before launching anything, a problem whose scratch does not fit the array.
    const bool use_ab = !(alpha == 0.0 || k == 0);
    if (m > 0 && n > 0 && use_ab && !too_big(m) && !too_big(n) && !too_big(k)) {
        const Plan<double> pl = make_plan<double>(&d.h, Variant::Fused, (int)m, (int)n, (int)k);
        if (total_bytes(&d.h, pl) > d.h.ws_bytes) return GFIP_ERR_SCRATCH_LIMIT;
    }
    return gemm_entry<double>(reinterpret_cast<gfip_handle_t>(&d.h), Variant::Fused, transa,
                              transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
}
