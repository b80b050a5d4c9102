// gfip_grouped.cu -- many independent GEMMs of uneven sizes in one persistent launch.
//
// The small-to-large unification of GEMMFIP (Sec. 1 and Sec. 3: one code path whatever the
// problem size) read for a batch on a GPU: every problem C_g := alpha_g op(A_g) op(B_g) +
// beta_g C_g, with its own sizes, operand orders and leading dimensions, runs inside ONE
// persistent launch.  The unit of work is a warp: each warp computes one small tile of one
// problem at a time, with a 3-stage k-chunk pipeline of its own (element copies of the raw
// strided operands into a private slice of shared memory, zero-filled at fringes, Sec. 2.2)
// and no barrier with any other warp, so an SM keeps many small tiles in flight.  Because the
// unit is a warp, one launch mixes tile shapes: each problem carries the shape and k-split
// factor that the autotuner (grouped.py) chose for its size bucket.  A split tile's k-ranges
// run on different warps; each stores its partial sums, and the last to arrive adds them in
// k-range order (so the bits do not depend on timing) and applies alpha and beta.
//
// Everything the launch needs is derived on the device from the caller's device arrays, so a
// call enqueues three kernels and reads nothing back; it can be captured in a CUDA graph:
//   prepare  one thread per problem: validates the arguments (an invalid problem gets no work
//            and raises GFIP_STATUS_BAD_PROBLEM), fills its descriptor, counts its work units
//   scan     one CTA: prefix sums of units, split tiles and partial-sum elements in the
//            processing order (problems whose partial sums would overflow the workspace run
//            unsplit), and clears the arrival counters
//   grouped  persistent warps are dealt the units in bands of all warps, alternately forwards
//            and backwards, costliest first when the caller orders the problems so; the C tile
//            of a unit goes through the warp's shared memory, so C is read and written
//            column by column with lanes along its rows
#include <climits>
#include <cstdint>
#include <type_traits>

#include "gfip_grouped.h"
#include "gfip_kernels.cuh"

namespace gfip {

constexpr unsigned int STATUS_BAD_PROBLEM = 0x4u;  // mirrors GFIP_STATUS_BAD_PROBLEM

namespace grp {

// Per element type: k rows per chunk (KC), chunk stages per warp (STAGES - 1 chunks in flight
// while one computes), warps per CTA (two CTAs per SM), the fastest of a measured sweep on the
// 4096-problem batch.  (Overridable at build time for such sweeps.)
#ifndef GFIP_GRP_F32_KC
#define GFIP_GRP_F32_KC 8
#endif
#ifndef GFIP_GRP_F32_STAGES
#define GFIP_GRP_F32_STAGES 3
#endif
#ifndef GFIP_GRP_F32_WARPS
#define GFIP_GRP_F32_WARPS 10
#endif
template <typename T> struct Pipe;
template <> struct Pipe<float> {
    static constexpr int KC = GFIP_GRP_F32_KC, STAGES = GFIP_GRP_F32_STAGES,
                         WARPS = GFIP_GRP_F32_WARPS;
};
#ifndef GFIP_GRP_F64_WARPS
#define GFIP_GRP_F64_WARPS 8
#endif
template <> struct Pipe<double> {
    static constexpr int KC = 8, STAGES = 3, WARPS = GFIP_GRP_F64_WARPS;
};
constexpr int MAX_SPLITS = 8;

// Warp tile shapes (GFIP_GROUP_TILE_*), the same for both element types: BM x BN per warp,
// TM x TN per lane, lanes BM/TM along m by BN/TN along n.  Small warp tiles keep registers and
// shared memory per warp low, so that an SM holds many warps, each with chunks in flight; the
// smallest ones cut the padding of tiny problems, which matters where the arithmetic pipe
// bounds the batch (FP64).
template <typename T, int SHAPE> struct Shape;
template <typename T> struct Shape<T, 0> { static constexpr int BM = 32, BN = 32, TM = 8, TN = 4; };
template <typename T> struct Shape<T, 1> { static constexpr int BM = 32, BN = 16, TM = 8, TN = 2; };
template <typename T> struct Shape<T, 2> { static constexpr int BM = 16, BN = 16, TM = 4, TN = 2; };
template <typename T> struct Shape<T, 3> { static constexpr int BM = 16, BN = 8, TM = 2, TN = 2; };
template <typename T> struct Shape<T, 4> { static constexpr int BM = 8, BN = 16, TM = 2, TN = 2; };
constexpr int NUM_SHAPES = 5;

__host__ __device__ constexpr int shape_bm(int es, int shape)
{
    return (void)es, shape <= 1 ? 32 : shape <= 3 ? 16 : 8;
}
__host__ __device__ constexpr int shape_bn(int es, int shape)
{
    return (void)es, shape == 0 ? 32 : shape == 3 ? 8 : 16;
}

// Shared-memory pitch of a chunk row: 16 bytes of padding spread the transposing copies over
// the banks and keep every fragment read 16-byte aligned.
template <typename T> __host__ __device__ constexpr int pitch(int bx)
{
    return bx + 16 / static_cast<int>(sizeof(T));
}

// Per-warp shared memory: STAGES chunk stages of the largest shape (32 x 32).
template <typename T> struct WarpStage {
    static constexpr int STAGE = Pipe<T>::KC * (pitch<T>(32) + pitch<T>(32));
    static constexpr int ELEMS = Pipe<T>::STAGES * STAGE;
};

// CTA of independent warps, two CTAs per SM.  Each CTA also keeps a coarse copy of the unit
// prefix sums (every COARSE-th entry) for the unit look-up.
constexpr int COARSE = 32;       // a warp reads the entries between two coarse ones at once
constexpr int COARSE_MAX = 512;    // entries kept in shared memory (batches up to 16384)
template <typename T> struct Launch {
    static constexpr int WARPS = Pipe<T>::WARPS;
    static constexpr int MIN_BLOCKS = 2;
    static constexpr size_t SMEM =
        (size_t)WARPS * WarpStage<T>::ELEMS * sizeof(T) + COARSE_MAX * sizeof(int);
};

__device__ __forceinline__ bool trans_ok(char t)
{
    return t == 'N' || t == 'n' || t == 'T' || t == 't' || t == 'C' || t == 'c';
}

// Element copies of the k chunks of one BX-wide operand tile at x0 (chunk rows kk at kk * P in
// the stage); element (x, kk) of op(X) sits at g[x + kk*ld] when contig, else at g[kk + x*ld].
// When contig, a warp row copies BX consecutive elements of 32 / BX k rows; otherwise KC
// lanes copy the KC consecutive k values of one x.  Either way a lane's N elements of a chunk
// lie rstep apart in global memory and a constant apart in the stage, and the next chunk's
// are one chunk further on.  Elements whose x lies past the problem's edge are zero-filled
// without a read (bit r of the mask); rows of k past the range's end only occur in its last
// chunk (kext < KC there).  Five registers of state: the pointer, its stride, the mask.
template <typename T, int BX> struct ChunkLoader {
    static constexpr int KC = Pipe<T>::KC;
    static constexpr int P = pitch<T>(BX);
    static constexpr int N = BX * KC / 32;
    static constexpr uint32_t CONTIG = 1u << 31;
    static_assert(N <= 31, "one mask bit per element");
    const T *p;
    int64_t rstep;
    uint32_t mask;   // bit r: element r is inside the problem; CONTIG: the layout

    __device__ __forceinline__ ChunkLoader(const T *g, int64_t ld, bool contig, int x0,
                                           int x_ext, int k0, int lane)
    {
        int xl, xstep;
        if (contig) {
            xl = lane % BX;
            xstep = 0;
            p = g + (x0 + xl) + (int64_t)(k0 + lane / BX) * ld;
            rstep = (int64_t)(32 / BX) * ld;
        } else {
            xl = lane / KC;
            xstep = 32 / KC;
            p = g + (k0 + lane % KC) + (int64_t)(x0 + xl) * ld;
            rstep = (int64_t)xstep * ld;
        }
        mask = contig ? CONTIG : 0u;
#pragma unroll
        for (int r = 0; r < N; ++r)
            if (x0 + xl + r * xstep < x_ext) mask |= 1u << r;
    }

    // Copies the next chunk (kext of its KC rows exist) into the stage at sdst; safe is any
    // readable address, passed for the elements not read.
    __device__ __forceinline__ void issue(uint32_t sdst, const T *safe, int kext, int lane)
    {
        if (mask & CONTIG) {
            constexpr int KS = 32 / BX;
            const int kk0 = lane / BX;
            const uint32_t d0 = sdst + (uint32_t)(kk0 * P + lane % BX) * sizeof(T);
#pragma unroll
            for (int r = 0; r < N; ++r) {
                const bool ok = ((mask >> r) & 1u) && (kk0 + r * KS < kext);
                cp_async_elem<sizeof(T)>(d0 + (uint32_t)(r * KS * P) * sizeof(T),
                                         ok ? p + r * rstep : safe, ok);
            }
            p += rstep * N;   // KC rows of k
        } else {
            constexpr int XS = 32 / KC;
            const int kk0 = lane % KC;
            const bool kok = kk0 < kext;
            const uint32_t d0 = sdst + (uint32_t)(kk0 * P + lane / KC) * sizeof(T);
#pragma unroll
            for (int r = 0; r < N; ++r) {
                const bool ok = ((mask >> r) & 1u) && kok;
                cp_async_elem<sizeof(T)>(d0 + (uint32_t)(r * XS) * sizeof(T),
                                         ok ? p + r * rstep : safe, ok);
            }
            p += KC;
        }
    }
};

__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p));
}

template <typename T, int N> __device__ __forceinline__ void lds_vec(T *d, const T *s)
{
    static_assert((N * sizeof(T)) % 8 == 0, "fragments are whole 8-byte words");
    if constexpr ((N * sizeof(T)) % 16 == 0) {
#pragma unroll
        for (int c = 0; c < N * static_cast<int>(sizeof(T)) / 16; ++c) {
            const uint4 v = reinterpret_cast<const uint4 *>(s)[c];
            reinterpret_cast<uint4 *>(d)[c] = v;
        }
    } else {
        const uint2 v = *reinterpret_cast<const uint2 *>(s);
        *reinterpret_cast<uint2 *>(d) = v;
    }
}

// acc[ii][jj] += a[ii] * b[jj]; FP32 pairs rows with the paired FMA (bit-identical to fmaf).
template <typename T, int TM, int TN>
__device__ __forceinline__ void fma_tile(const T (&a)[TM], const T (&b)[TN], T (&acc)[TM][TN])
{
    if constexpr (std::is_same<T, float>::value) {
#pragma unroll
        for (int jj = 0; jj < TN; ++jj) {
            const float2 bb = make_float2(b[jj], b[jj]);
#pragma unroll
            for (int ii = 0; ii < TM; ii += 2) {
                const float2 c = __ffma2_rn(make_float2(a[ii], a[ii + 1]), bb,
                                            make_float2(acc[ii][jj], acc[ii + 1][jj]));
                acc[ii][jj] = c.x;
                acc[ii + 1][jj] = c.y;
            }
        }
    } else {
#pragma unroll
        for (int ii = 0; ii < TM; ++ii)
#pragma unroll
            for (int jj = 0; jj < TN; ++jj) acc[ii][jj] = fma(a[ii], b[jj], acc[ii][jj]);
    }
}

// One warp computes split s of tile (i, j) of problem d.
template <typename T, int SHAPE>
__device__ void warp_tile(const GroupParams<T> &gp, const GroupDesc<T> &d, int tile, int s,
                          T *stage, int lane)
{
    using S = Shape<T, SHAPE>;
    constexpr int BM = S::BM, BN = S::BN, TM = S::TM, TN = S::TN;
    constexpr int KC = Pipe<T>::KC, STAGES = Pipe<T>::STAGES;
    constexpr int LR = BM / TM;
    static_assert(LR * (BN / TN) == 32, "a tile shape must spread over 32 lanes");
    constexpr int PA = pitch<T>(BM), PB = pitch<T>(BN);
    constexpr int SA = KC * PA;   // elements of A per stage (B follows)
    const int i = tile % d.mt, j = tile / d.mt;
    const int lr = lane % LR, lc = lane / LR;
    T acc[TM][TN];
#pragma unroll
    for (int ii = 0; ii < TM; ++ii)
#pragma unroll
        for (int jj = 0; jj < TN; ++jj) acc[ii][jj] = T(0);

    if (d.beta != T(0) && lane < BN && j * BN + lane < d.n) {
        // the epilogue reads this tile of C: bring its columns into L2 while the k loop runs
        const T *c0 = d.C + (int64_t)(j * BN + lane) * d.ldc + i * BM;
        const int rows = min(BM, d.m - i * BM);
        constexpr int LINE = 128 / static_cast<int>(sizeof(T));
#pragma unroll
        for (int r = 0; r < BM; r += LINE)
            if (r < rows) prefetch_l2(c0 + r);
        prefetch_l2(c0 + rows - 1);
    }

    if (d.ks > 0) {
        const int kb = s * d.ks, ke = min(d.k, kb + d.ks);
        const int nch = (ke - kb + KC - 1) / KC;
        const bool acon = d.order & 1, bcon = (d.order >> 1) & 1;
        const uint32_t s0 = smem_addr(stage);
        constexpr int ST = WarpStage<T>::STAGE;
        ChunkLoader<T, BM> la(d.A, d.lda, acon, i * BM, d.m, kb, lane);
        ChunkLoader<T, BN> lb(d.B, d.ldb, bcon, j * BN, d.n, kb, lane);
        auto issue = [&](int c) {   // chunks are issued in order
            const uint32_t sa = s0 + (uint32_t)((c % STAGES) * ST) * sizeof(T);
            const int kext = min(KC, ke - (kb + c * KC));
            la.issue(sa, d.A, kext, lane);
            lb.issue(sa + SA * sizeof(T), d.B, kext, lane);
        };
#pragma unroll
        for (int c = 0; c < STAGES - 1; ++c) {
            if (c < nch) issue(c);
            cp_async_commit();
        }
        for (int c = 0; c < nch; ++c) {
            // the stage of chunk c + STAGES - 1 held chunk c - 1, computed last iteration
            if (c + STAGES - 1 < nch) issue(c + STAGES - 1);
            cp_async_commit();
            cp_async_wait<STAGES - 1>();   // chunk c has landed
            __syncwarp();
            const T *As = stage + (c % STAGES) * ST;
            const T *Bs = As + SA;
            if (c + 1 < nch || (ke - kb) % KC == 0) {
#pragma unroll
                for (int kk = 0; kk < KC; ++kk) {
                    T a[TM], b[TN];
                    lds_vec<T, TM>(a, As + kk * PA + lr * TM);
                    lds_vec<T, TN>(b, Bs + kk * PB + lc * TN);
                    fma_tile<T, TM, TN>(a, b, acc);
                }
            } else {
                // the range's last chunk: only its rows of k that exist (the rest is zero
                // padding, and skipping it is warp-uniform, so it saves pipe time)
                const int kext = (ke - kb) % KC;
#pragma unroll 1
                for (int kk = 0; kk < kext; ++kk) {
                    T a[TM], b[TN];
                    lds_vec<T, TM>(a, As + kk * PA + lr * TM);
                    lds_vec<T, TN>(b, Bs + kk * PB + lc * TN);
                    fma_tile<T, TM, TN>(a, b, acc);
                }
            }
            __syncwarp();   // the stage is refilled two iterations later
        }
        cp_async_wait<0>();
    }

    if (d.splits > 1) {
        // store this k-range's partial sums (accumulator by accumulator, lanes adjacent, so
        // that every warp access is one run); the last of the tile's splits to arrive adds
        // them all in k-range order and finishes the tile
        T *part = gp.partial + d.part_off;
        T *mine = part + ((int64_t)tile * d.splits + s) * (BM * BN) + lane;
#pragma unroll
        for (int ii = 0; ii < TM; ++ii)
#pragma unroll
            for (int jj = 0; jj < TN; ++jj) __stcg(mine + (ii * TN + jj) * 32, acc[ii][jj]);
        __threadfence();
        __syncwarp();
        int last = 0;
        if (lane == 0) last = atomicAdd(gp.counters + d.ctr_off + tile, 1) == d.splits - 1;
        last = __shfl_sync(0xffffffffu, last, 0);
        if (!last) return;
        __threadfence();
        for (int t = 0; t < d.splits; ++t) {
            const T *src = part + ((int64_t)tile * d.splits + t) * (BM * BN) + lane;
#pragma unroll
            for (int ii = 0; ii < TM; ++ii)
#pragma unroll
                for (int jj = 0; jj < TN; ++jj) {
                    const T v = __ldcg(src + (ii * TN + jj) * 32);
                    acc[ii][jj] = (t == 0) ? v : acc[ii][jj] + v;
                }
        }
    }
    // The epilogue goes through the warp's stage (free now: every chunk has landed and been
    // used): C's tile is copied in with lanes along its rows, whole columns at a time (every
    // warp access one or two runs of consecutive elements, all in flight together), updated
    // there by each lane from its accumulators, and written back the way it came in.
    constexpr int CPITCH = BM + 1;
    constexpr int CPI = 32 / BM;   // columns per warp access
    constexpr int NC = BN / CPI;   // accesses per lane
    static_assert(BN * CPITCH <= WarpStage<T>::ELEMS, "the C tile fits the warp's stage");
    const bool read_c = d.beta != T(0);
    const int rr = lane % BM, cj = lane / BM;
    const int row = i * BM + rr;
    const bool row_ok = row < d.m;
    T *crow = d.C + row;
    if (read_c) {
        const uint32_t st0 = smem_addr(stage);
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            const int c = q * CPI + cj, col = j * BN + c;
            const bool ok = row_ok && col < d.n;
            cp_async_elem<sizeof(T)>(st0 + (uint32_t)(c * CPITCH + rr) * sizeof(T),
                                     ok ? crow + (int64_t)col * d.ldc : d.C, ok);
        }
        cp_async_commit();
        cp_async_wait<0>();
        __syncwarp();
    }
#pragma unroll
    for (int ii = 0; ii < TM; ++ii)
#pragma unroll
        for (int jj = 0; jj < TN; ++jj) {
            T &e = stage[(lc * TN + jj) * CPITCH + lr * TM + ii];
            T v = d.alpha * acc[ii][jj];
            if (read_c) v = fma(d.beta, e, v);
            e = v;
        }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < NC; ++q) {
        const int c = q * CPI + cj, col = j * BN + c;
        if (row_ok && col < d.n) crow[(int64_t)col * d.ldc] = stage[c * CPITCH + rr];
    }
    __syncwarp();   // the stage is refilled by the next unit
}

template <typename T> __global__ void prepare_kernel(const GroupParams<T> gp)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= gp.count) return;
    const int g = gp.order ? gp.order[r] : r;
    const char ta = gp.transa[g], tb = gp.transb[g];
    const int m = gp.m[g], n = gp.n[g], k = gp.k[g];
    const bool an = (ta == 'N' || ta == 'n'), bn = (tb == 'N' || tb == 'n');
    const int64_t rows_a = an ? m : k, rows_b = bn ? k : n;
    const int64_t lda = gp.lda[g], ldb = gp.ldb[g], ldc = gp.ldc[g];
    GroupDesc<T> d;
    d.A = gp.A[g];
    d.B = gp.B[g];
    d.C = gp.C[g];
    d.lda = lda;
    d.ldb = ldb;
    d.ldc = ldc;
    d.m = m;
    d.n = n;
    d.k = k;
    d.alpha = gp.alpha[g];
    d.beta = gp.beta[g];
    d.order = (an ? 1 : 0) | (bn ? 0 : 2);
    const bool bad = !trans_ok(ta) || !trans_ok(tb) || m < 0 || n < 0 || k < 0 ||
                     lda < (rows_a > 1 ? rows_a : 1) || ldb < (rows_b > 1 ? rows_b : 1) ||
                     ldc < (m > 1 ? m : 1);
    const bool use_ab = !(d.alpha == T(0) || k == 0);
    // reference-BLAS quick return: nothing to do when m or n is 0, or when C stays C
    const bool nothing = bad || m == 0 || n == 0 || (!use_ab && d.beta == T(1));
    if (bad) atomicOr(gp.status, STATUS_BAD_PROBLEM);
    const int code = gp.plan ? gp.plan[g] : gp.uniform_shape;
    int shape = code & 0xff, splits = (code >> 8) & 0xff;
    if (shape < 0 || shape >= NUM_SHAPES) shape = 0;
    const int es = static_cast<int>(sizeof(T));
    const int bm = shape_bm(es, shape), bn_ = shape_bn(es, shape);
    constexpr int KC = Pipe<T>::KC;
    const int chunks = use_ab ? (k + KC - 1) / KC : 0;
    splits = max(1, min(min(splits, MAX_SPLITS), max(1, chunks)));
    d.shape = shape;
    d.mt = (m + bm - 1) / bm;
    d.nt = (n + bn_ - 1) / bn_;
    d.splits = splits;
    d.ks = use_ab ? ((chunks + splits - 1) / splits) * KC : 0;
    if (use_ab) d.splits = splits = (chunks + d.ks / KC - 1) / (d.ks / KC);   // no empty split
    d.ctr_off = 0;
    d.part_off = 0;
    gp.desc[r] = d;
    const int tiles = nothing ? 0 : d.mt * d.nt;
    gp.units[r] = tiles * splits;
    gp.stiles[r] = splits > 1 ? tiles : 0;
    gp.pelems[r] = splits > 1 ? (int64_t)tiles * splits * bm * bn_ : 0;
}

// The three counts of a rank that the launch scans together.
struct Counts {
    int units, stiles;
    int64_t pelems;
    __device__ Counts operator+(const Counts &o) const
    {
        return Counts{units + o.units, stiles + o.stiles, pelems + o.pelems};
    }
};

__device__ __forceinline__ Counts shfl_up(const Counts &v, int off)
{
    return Counts{__shfl_up_sync(0xffffffffu, v.units, off),
                  __shfl_up_sync(0xffffffffu, v.stiles, off),
                  static_cast<int64_t>(__shfl_up_sync(
                      0xffffffffu, static_cast<long long>(v.pelems), off))};
}

__device__ __forceinline__ Counts warp_inclusive(Counts v, int lane)
{
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const Counts x = shfl_up(v, off);
        if (lane >= off) v = v + x;
    }
    return v;
}

// Exclusive prefix of v over the 1024 threads of the CTA (thread order); *total gets the sum.
// wsum is 33 entries of shared memory, free again when the call returns.
__device__ Counts block_exclusive(const Counts &v, Counts *wsum, Counts *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const Counts inc = warp_inclusive(v, lane);
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const Counts w = wsum[lane];
        const Counts winc = warp_inclusive(w, lane);
        wsum[lane] = Counts{winc.units - w.units, winc.stiles - w.stiles, winc.pelems - w.pelems};
        if (lane == 31) wsum[32] = winc;
    }
    __syncthreads();
    const Counts base = wsum[warp];
    *total = wsum[32];
    __syncthreads();
    return Counts{base.units + inc.units - v.units, base.stiles + inc.stiles - v.stiles,
                  base.pelems + inc.pelems - v.pelems};
}

// One CTA of 1024 threads turns the per-rank counts into the unit prefix sums the GEMM
// kernel searches and gives each split problem its arrival counters and partial-sum space,
// 1024 ranks at a time (coalesced loads, warp-shuffle scans).  With a plan, a split problem
// whose space would pass the workspace's capacity runs unsplit instead: the requested space
// before a rank only grows with the rank, so the kept problems are exactly those before the
// first cut and their places do not move.
template <typename T> __global__ void __launch_bounds__(1024) scan_kernel(const GroupParams<T> gp)
{
    __shared__ Counts wsum[33];
    const int count = gp.count;
    const int tid = threadIdx.x;
    constexpr int KC = Pipe<T>::KC;
    Counts carry{0, 0, 0}, req_carry{0, 0, 0};
    // the next 1024 ranks' counts load while these are scanned
    Counts next{0, 0, 0};
    if (tid < count) next = Counts{gp.units[tid], gp.stiles[tid], gp.pelems[tid]};
    for (int base = 0; base < count; base += 1024) {
        const int r = base + tid;
        Counts v = next;
        if (r + 1024 < count)
            next = Counts{gp.units[r + 1024], gp.stiles[r + 1024], gp.pelems[r + 1024]};
        if (gp.plan != nullptr) {
            Counts tot;
            const Counts before = block_exclusive(v, wsum, &tot) + req_carry;
            req_carry = req_carry + tot;
            if (r < count && v.stiles > 0 &&
                (before.pelems + v.pelems > gp.partial_capacity ||
                 before.stiles + v.stiles > gp.max_split_tiles)) {
                GroupDesc<T> &d = gp.desc[r];
                d.splits = 1;
                d.ks = ((d.k + KC - 1) / KC) * KC;
                v = Counts{v.stiles, 0, 0};   // its tiles, unsplit
            }
        }
        Counts tot;
        const Counts before = block_exclusive(v, wsum, &tot) + carry;
        carry = carry + tot;
        if (r < count) {
            GroupDesc<T> &d = gp.desc[r];
            d.ctr_off = before.stiles;
            d.part_off = before.pelems;
            gp.prefix[r] = before.units;
        }
    }
    if (tid == 0) gp.prefix[count] = carry.units;
    for (int q = tid; q < carry.stiles; q += 1024) gp.counters[q] = 0;
}

template <typename T>
__global__ void __launch_bounds__(Launch<T>::WARPS * 32, Launch<T>::MIN_BLOCKS)
    grouped_kernel(const GroupParams<T> gp)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T *stage = reinterpret_cast<T *>(smem_raw) + warp * WarpStage<T>::ELEMS;
    int *coarse = reinterpret_cast<int *>(smem_raw + (size_t)Launch<T>::WARPS *
                                                          WarpStage<T>::ELEMS * sizeof(T));
    const int count = gp.count;
    // every COARSE-th entry of the prefix sums, for a look-up in two short searches
    const int ncoarse = count / COARSE + 1;
    const bool use_coarse = ncoarse <= COARSE_MAX;
    if (use_coarse)
        for (int t = threadIdx.x; t < ncoarse; t += blockDim.x) coarse[t] = gp.prefix[t * COARSE];
    __syncthreads();
    const int total = gp.prefix[count];
    const int nwarps = gridDim.x * Launch<T>::WARPS;
    const int w = blockIdx.x * Launch<T>::WARPS + warp;
    // units are dealt in bands of nwarps, alternately forwards and backwards (the processing
    // order puts the costliest units first, so every warp gets a similar sum)
    for (int band = 0;; ++band) {
        const int u = band * nwarps + ((band & 1) ? nwarps - 1 - w : w);
        if (band * nwarps >= total) break;
        if (u >= total) continue;
        // rank of unit u: the last r with prefix[r] <= u (ranks without units share their
        // successor's prefix, so the last is the one that has the unit)
        int lo, first;
        if (use_coarse) {
            int clo = 0, chi = ncoarse - 1;
            while (clo < chi) {
                const int mid = (clo + chi + 1) >> 1;
                if (coarse[mid] <= u) clo = mid;
                else chi = mid - 1;
            }
            // one warp-wide read of the COARSE (= 32) entries that follow
            const int r = clo * COARSE + lane;
            const int pr = r < count ? __ldg(gp.prefix + r) : INT_MAX;
            const unsigned le = __ballot_sync(0xffffffffu, pr <= u);
            const int last = 31 - __clz(le);
            lo = clo * COARSE + last;
            first = __shfl_sync(0xffffffffu, pr, last);
        } else {
            int a = 0, b = count - 1;
            while (a < b) {
                const int mid = (a + b + 1) >> 1;
                if (__ldg(gp.prefix + mid) <= u) a = mid;
                else b = mid - 1;
            }
            lo = a;
            first = __ldg(gp.prefix + lo);
        }
        const GroupDesc<T> d = gp.desc[lo];
        const int local = u - first;
        const int tile = local / d.splits, s = local % d.splits;
        switch (d.shape) {
        case 0: warp_tile<T, 0>(gp, d, tile, s, stage, lane); break;
        case 1: warp_tile<T, 1>(gp, d, tile, s, stage, lane); break;
        case 2: warp_tile<T, 2>(gp, d, tile, s, stage, lane); break;
        case 3: warp_tile<T, 3>(gp, d, tile, s, stage, lane); break;
        default: warp_tile<T, 4>(gp, d, tile, s, stage, lane); break;
        }
        __syncwarp();
    }
}

template <typename T> int grid_size()
{
    static int grid = 0;
    if (grid == 0) {
        cudaFuncSetAttribute(grouped_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(Launch<T>::SMEM));
        int per = 0, dev = 0, sms = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, grouped_kernel<T>,
                                                      Launch<T>::WARPS * 32, Launch<T>::SMEM);
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        grid = (per > 0 ? per : 1) * sms;
    }
    return grid;
}

}  // namespace grp

template <typename T> cudaError_t launch_grouped_impl(const GroupParams<T> &gp, cudaStream_t s)
{
    const int threads = 128;
    grp::prepare_kernel<T><<<(gp.count + threads - 1) / threads, threads, 0, s>>>(gp);
    grp::scan_kernel<T><<<1, 1024, 0, s>>>(gp);
    grp::grouped_kernel<T><<<grp::grid_size<T>(), grp::Launch<T>::WARPS * 32,
                             grp::Launch<T>::SMEM, s>>>(gp);
    return cudaGetLastError();
}

size_t grouped_desc_bytes(int count, int es)
{
    return es == 8 ? sizeof(GroupDesc<double>) * (size_t)count
                   : sizeof(GroupDesc<float>) * (size_t)count;
}

template <> cudaError_t launch_grouped<double>(const GroupParams<double> &gp, cudaStream_t s)
{
    return launch_grouped_impl<double>(gp, s);
}

template <> cudaError_t launch_grouped<float>(const GroupParams<float> &gp, cudaStream_t s)
{
    return launch_grouped_impl<float>(gp, s);
}

}  // namespace gfip
