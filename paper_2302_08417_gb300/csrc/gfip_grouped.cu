// gfip_grouped.cu -- many independent GEMMs of uneven sizes in one persistent launch.
//
// The small-to-large unification of GEMMFIP (Sec. 1 and Sec. 3: one code path whatever the
// problem size) read for a batch on a GPU: every problem C_g := alpha_g op(A_g) op(B_g) +
// beta_g C_g, with its own sizes, operand orders and leading dimensions, runs inside ONE
// persistent launch.  The unit of work is a warp: each warp computes one small tile of one
// problem at a time, with a double-buffered k-chunk pipeline of its own (element copies of the
// raw strided operands into a private slice of shared memory, zero-filled at fringes, Sec. 2.2)
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
//   grouped  persistent warps stride over the global unit list, largest problems first when
//            the caller orders them so
#include <cstdint>
#include <type_traits>

#include "gfip_grouped.h"
#include "gfip_kernels.cuh"

namespace gfip {

constexpr unsigned int STATUS_BAD_PROBLEM = 0x4u;  // mirrors GFIP_STATUS_BAD_PROBLEM

namespace grp {

constexpr int KC = 8;           // k rows per chunk
constexpr int STAGES = 3;       // chunk stages per warp: two chunks in flight while one computes
constexpr int MAX_SPLITS = 8;

// Warp tile shapes (GFIP_GROUP_TILE_DEFAULT / SMALL / TINY), the same for both element types:
// BM x BN per warp, TM x TN per lane, lanes BM/TM along m by BN/TN along n.  Small warp tiles
// keep registers and shared memory per warp low, so that an SM holds many warps, each with
// chunks in flight: these problems are bound by memory latency, not by arithmetic.
template <typename T, int SHAPE> struct Shape;
template <typename T> struct Shape<T, 0> { static constexpr int BM = 32, BN = 32, TM = 8, TN = 4; };
template <typename T> struct Shape<T, 1> { static constexpr int BM = 32, BN = 16, TM = 8, TN = 2; };
template <typename T> struct Shape<T, 2> { static constexpr int BM = 16, BN = 16, TM = 4, TN = 2; };

__host__ __device__ constexpr int shape_bm(int es, int shape)
{
    return (void)es, shape == 2 ? 16 : 32;
}
__host__ __device__ constexpr int shape_bn(int es, int shape)
{
    return (void)es, shape == 0 ? 32 : 16;
}

// Shared-memory pitch of a chunk row: 16 bytes of padding spread the transposing copies over
// the banks and keep every fragment read 16-byte aligned.
template <typename T> __host__ __device__ constexpr int pitch(int bx)
{
    return bx + 16 / static_cast<int>(sizeof(T));
}

// Per-warp shared memory: STAGES chunk stages of the largest shape (32 x 32).
template <typename T> struct WarpStage {
    static constexpr int STAGE = KC * (pitch<T>(32) + pitch<T>(32));
    static constexpr int ELEMS = STAGES * STAGE;
};

// CTA of independent warps; FP32: 12 warps, two CTAs per SM (24 warps, 80 registers a
// thread); FP64: 8 warps, two CTAs per SM (16 warps, 128 registers).  Each CTA also keeps a
// coarse copy of the unit prefix sums (every COARSE-th entry) for the unit look-up.
constexpr int COARSE = 32;
constexpr int COARSE_MAX = 512;    // entries kept in shared memory (batches up to 16384)
template <typename T> struct Launch {
    static constexpr int WARPS = std::is_same<T, float>::value ? 12 : 8;
    static constexpr int MIN_BLOCKS = 2;
    static constexpr size_t SMEM =
        (size_t)WARPS * WarpStage<T>::ELEMS * sizeof(T) + COARSE_MAX * sizeof(int);
};

__device__ __forceinline__ bool trans_ok(char t)
{
    return t == 'N' || t == 'n' || t == 'T' || t == 't' || t == 'C' || t == 'c';
}

// Element copies of one k chunk (rows k0 .. k0 + KC - 1, of which kend - k0 exist) of a
// BX-wide operand tile at x0 into the stage (row kk at kk * P); element (x, kk) of op(X)
// sits at g[(x0+x) + (k0+kk)*ld] when contig, else at g[(k0+kk) + (x0+x)*ld].
template <typename T, int BX>
__device__ __forceinline__ void load_chunk(uint32_t sdst, const T *g, int64_t ld, bool contig,
                                           int x0, int x_ext, int k0, int kend, int lane)
{
    constexpr int P = pitch<T>(BX);
    constexpr int N = BX * KC / 32;
    if (contig) {
#pragma unroll 4
        for (int r = 0; r < N; ++r) {
            const int e = lane + 32 * r;
            const int x = e % BX, kk = e / BX;
            const bool ok = (x0 + x < x_ext) && (k0 + kk < kend);
            const T *src = ok ? g + (int64_t)(x0 + x) + (int64_t)(k0 + kk) * ld : g;
            cp_async_elem<sizeof(T)>(sdst + (kk * P + x) * sizeof(T), src, ok);
        }
    } else {
#pragma unroll 4
        for (int r = 0; r < N; ++r) {
            const int e = lane + 32 * r;
            const int kk = e % KC, x = e / KC;
            const bool ok = (x0 + x < x_ext) && (k0 + kk < kend);
            const T *src = ok ? g + (int64_t)(k0 + kk) + (int64_t)(x0 + x) * ld : g;
            cp_async_elem<sizeof(T)>(sdst + (kk * P + x) * sizeof(T), src, ok);
        }
    }
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
    constexpr int LR = BM / TM;
    static_assert(LR * (BN / TN) == 32, "a tile shape must spread over 32 lanes");
    constexpr int PA = pitch<T>(BM), PB = pitch<T>(BN);
    constexpr int SA = KC * PA, SB = KC * PB;   // elements per stage of A and of B
    const int i = tile % d.mt, j = tile / d.mt;
    const int lr = lane % LR, lc = lane / LR;
    T acc[TM][TN];
#pragma unroll
    for (int ii = 0; ii < TM; ++ii)
#pragma unroll
        for (int jj = 0; jj < TN; ++jj) acc[ii][jj] = T(0);

    if (d.ks > 0) {
        const int kb = s * d.ks, ke = min(d.k, kb + d.ks);
        const int nch = (ke - kb + KC - 1) / KC;
        const bool acon = d.order & 1, bcon = (d.order >> 1) & 1;
        const uint32_t s0 = smem_addr(stage);
        constexpr int ST = WarpStage<T>::STAGE;
        auto issue = [&](int c) {
            const uint32_t sa = s0 + (uint32_t)((c % STAGES) * ST) * sizeof(T);
            load_chunk<T, BM>(sa, d.A, d.lda, acon, i * BM, d.m, kb + c * KC, ke, lane);
            load_chunk<T, BN>(sa + SA * sizeof(T), d.B, d.ldb, bcon, j * BN, d.n, kb + c * KC,
                              ke, lane);
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

    const int row0 = i * BM + lr * TM, col0 = j * BN + lc * TN;
    if (d.splits > 1) {
        // store this k-range's partial sums; the last of the tile's splits to arrive adds
        // them all in k-range order and finishes the tile
        T *part = gp.partial + d.part_off;
        T *mine = part + ((int64_t)tile * d.splits + s) * (BM * BN) + lane * (TM * TN);
#pragma unroll
        for (int ii = 0; ii < TM; ++ii)
#pragma unroll
            for (int jj = 0; jj < TN; ++jj) __stcg(mine + ii * TN + jj, acc[ii][jj]);
        __threadfence();
        __syncwarp();
        int last = 0;
        if (lane == 0) last = atomicAdd(gp.counters + d.ctr_off + tile, 1) == d.splits - 1;
        last = __shfl_sync(0xffffffffu, last, 0);
        if (!last) return;
        __threadfence();
        for (int t = 0; t < d.splits; ++t) {
            const T *src = part + ((int64_t)tile * d.splits + t) * (BM * BN) + lane * (TM * TN);
#pragma unroll
            for (int ii = 0; ii < TM; ++ii)
#pragma unroll
                for (int jj = 0; jj < TN; ++jj) {
                    const T v = __ldcg(src + ii * TN + jj);
                    acc[ii][jj] = (t == 0) ? v : acc[ii][jj] + v;
                }
        }
    }
    const bool read_c = d.beta != T(0);
#pragma unroll
    for (int jj = 0; jj < TN; ++jj) {
        const int col = col0 + jj;
        if (col >= d.n) continue;
        T *ccol = d.C + (int64_t)col * d.ldc;
        T c[TM];
#pragma unroll
        for (int ii = 0; ii < TM; ++ii)
            c[ii] = (read_c && row0 + ii < d.m) ? ccol[row0 + ii] : T(0);
#pragma unroll
        for (int ii = 0; ii < TM; ++ii) {
            if (row0 + ii >= d.m) continue;
            T v = d.alpha * acc[ii][jj];
            if (read_c) v = fma(d.beta, c[ii], v);
            ccol[row0 + ii] = v;
        }
    }
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
    if (shape < 0 || shape > 2) shape = 0;
    const int es = static_cast<int>(sizeof(T));
    const int bm = shape_bm(es, shape), bn_ = shape_bn(es, shape);
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
    gp.desc[g] = d;
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

// Exclusive prefix sums of the counts of ranks 0..count-1, in place, over one CTA of 1024
// threads (each scanning a contiguous run of ranks); returns the totals.
template <typename T>
__device__ Counts scan_counts(const GroupParams<T> &gp, Counts *part)
{
    const int count = gp.count;
    const int tid = threadIdx.x;
    const int per = (count + 1023) / 1024;
    const int lo = min(count, tid * per), hi = min(count, lo + per);
    Counts sum{0, 0, 0};
    for (int q = lo; q < hi; ++q) sum = sum + Counts{gp.units[q], gp.stiles[q], gp.pelems[q]};
    part[tid] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const Counts x = tid >= off ? part[tid - off] : Counts{0, 0, 0};
        __syncthreads();
        part[tid] = part[tid] + x;
        __syncthreads();
    }
    Counts run{part[tid].units - sum.units, part[tid].stiles - sum.stiles,
               part[tid].pelems - sum.pelems};
    for (int q = lo; q < hi; ++q) {
        const Counts c{gp.units[q], gp.stiles[q], gp.pelems[q]};
        gp.units[q] = run.units;
        gp.stiles[q] = run.stiles;
        gp.pelems[q] = run.pelems;
        run = run + c;
    }
    const Counts total = part[1023];
    __syncthreads();
    return total;
}

template <typename T> __global__ void __launch_bounds__(1024) scan_kernel(const GroupParams<T> gp)
{
    __shared__ Counts part[1024];
    const int count = gp.count;
    const int tid = threadIdx.x;
    constexpr int ES = static_cast<int>(sizeof(T));
    if (gp.plan != nullptr) {
        // where each split problem's partial sums and counters would start, in processing
        // order; a problem whose range would pass the workspace's capacity runs unsplit (a
        // clean cut: both prefixes only grow).  units[] keeps the per-rank unit counts.
        int *keep_units = gp.prefix;   // scratch: the unscanned unit counts
        for (int r = tid; r < count; r += 1024) keep_units[r] = gp.units[r];
        __syncthreads();
        scan_counts<T>(gp, part);
        for (int r = tid; r < count; r += 1024) {
            GroupDesc<T> &d = gp.desc[gp.order ? gp.order[r] : r];
            const int tiles = keep_units[r] / d.splits;
            if (d.splits > 1) {
                const int64_t pe = (int64_t)tiles * d.splits * shape_bm(ES, d.shape) *
                                   shape_bn(ES, d.shape);
                if (gp.pelems[r] + pe > gp.partial_capacity ||
                    gp.stiles[r] + tiles > gp.max_split_tiles) {
                    d.splits = 1;
                    d.ks = ((d.k + KC - 1) / KC) * KC;
                }
            }
            gp.units[r] = tiles * d.splits;
            gp.stiles[r] = d.splits > 1 ? tiles : 0;
            gp.pelems[r] = d.splits > 1 ? (int64_t)tiles * d.splits * shape_bm(ES, d.shape) *
                                              shape_bn(ES, d.shape)
                                        : 0;
        }
        __syncthreads();
    }
    const Counts total = scan_counts<T>(gp, part);
    for (int r = tid; r < count; r += 1024) {
        GroupDesc<T> &d = gp.desc[gp.order ? gp.order[r] : r];
        d.ctr_off = gp.stiles[r];
        d.part_off = gp.pelems[r];
        gp.prefix[r] = gp.units[r];
    }
    if (tid == 0) gp.prefix[count] = total.units;
    for (int q = tid; q < total.stiles; q += 1024) gp.counters[q] = 0;
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
    for (int u = blockIdx.x * Launch<T>::WARPS + warp; u < total; u += nwarps) {
        // rank of unit u: the last r with prefix[r] <= u
        int lo = 0, hi = count - 1;
        if (use_coarse) {
            int clo = 0, chi = ncoarse - 1;
            while (clo < chi) {
                const int mid = (clo + chi + 1) >> 1;
                if (coarse[mid] <= u) clo = mid;
                else chi = mid - 1;
            }
            lo = clo * COARSE;
            hi = min(count - 1, lo + COARSE - 1);
        }
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(gp.prefix + mid) <= u) lo = mid;
            else hi = mid - 1;
        }
        const int g = gp.order ? __ldg(gp.order + lo) : lo;
        const GroupDesc<T> d = gp.desc[g];
        const int local = u - __ldg(gp.prefix + lo);
        const int tile = local / d.splits, s = local % d.splits;
        switch (d.shape) {
        case 0: warp_tile<T, 0>(gp, d, tile, s, stage, lane); break;
        case 1: warp_tile<T, 1>(gp, d, tile, s, stage, lane); break;
        default: warp_tile<T, 2>(gp, d, tile, s, stage, lane); break;
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
