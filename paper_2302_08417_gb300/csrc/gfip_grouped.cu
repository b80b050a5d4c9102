// gfip_grouped.cu -- many independent GEMMs of uneven sizes in one persistent launch.
//
// The small-to-large unification of GEMMFIP (Sec. 1 and Sec. 3: one code path whatever the
// problem size) read for a GPU: a batch of problems, each C_g := alpha_g op(A_g) op(B_g) +
// beta_g C_g with its own sizes, operand orders and leading dimensions, runs as ONE launch of
// the same tile core as the single GEMM.  Everything the launch needs is derived on the
// device from the caller's device arrays, so a call enqueues three kernels and never reads
// anything back: it can be captured in a CUDA graph and replayed.
//
//   prepare  one thread per problem: validates the arguments (an invalid problem gets no
//            tiles and raises GFIP_STATUS_BAD_PROBLEM), packs a descriptor, counts its tiles
//   scan     one CTA: exclusive prefix sum of the tile counts and the total
//   grouped  persistent CTAs stride over the global tile list; a tile finds its problem by
//            binary search in the prefix sums and runs the data-parallel tile core
//            (raw strided operands, whole k loop, alpha/beta epilogue)
#include <cstdint>
#include <type_traits>

#include "gfip_grouped.h"
#include "gfip_kernels.cuh"

namespace gfip {

constexpr unsigned int STATUS_BAD_PROBLEM = 0x4u;  // mirrors GFIP_STATUS_BAD_PROBLEM

// FP32 tile for small problems: 64 x 64 x 32 on 64 threads (8 x 8 per thread).
struct TileCfgF32Small {
    static constexpr int BM = 64, BN = 64, BK = 32, THREADS = 64, NCM = 2, NCN = 2, STAGES = 3;
    static constexpr int MIN_BLOCKS = 4, UNROLL = 8;
};

__device__ __forceinline__ bool trans_ok(char t)
{
    return t == 'N' || t == 'n' || t == 'T' || t == 't' || t == 'C' || t == 'c';
}

template <typename T, int BM, int BN, int BK>
__global__ void grouped_prepare_kernel(const GroupParams<T> gp)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= gp.count) return;
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
    d.kt = use_ab ? (k + BK - 1) / BK : 0;
    d.mt = (m + BM - 1) / BM;
    gp.desc[g] = d;
    gp.prefix[g] = nothing ? 0 : d.mt * ((n + BN - 1) / BN);
}

// In-place exclusive prefix sum of prefix[0..count) with the total in prefix[count]; one CTA
// of 1024 threads, each scanning a contiguous run.
__global__ void __launch_bounds__(1024) grouped_scan_kernel(int *prefix, int count)
{
    __shared__ int part[1024];
    const int tid = threadIdx.x;
    const int per = (count + 1023) / 1024;
    const int lo = min(count, tid * per), hi = min(count, lo + per);
    int sum = 0;
    for (int g = lo; g < hi; ++g) sum += prefix[g];
    part[tid] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int v = tid >= off ? part[tid - off] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    int run = part[tid] - sum;   // exclusive start of this thread's run
    for (int g = lo; g < hi; ++g) {
        const int c = prefix[g];
        prefix[g] = run;
        run += c;
    }
    if (tid == 1023) prefix[count] = part[1023];
}

template <typename T, typename Cfg, bool AC, bool BC>
__device__ __forceinline__ void grouped_tile(const GroupDesc<T> &d, GemmSmem<T, Cfg> &sm,
                                             int i, int j)
{
    using K = Kernel<T, AC, BC, Cfg>;
    GemmParams<T> p{};
    p.A = d.A;
    p.B = d.B;
    p.C = d.C;
    p.lda = d.lda;
    p.ldb = d.ldb;
    p.ldc = d.ldc;
    p.m = d.m;
    p.n = d.n;
    p.k = d.k;
    p.alpha = d.alpha;
    p.beta = d.beta;
    p.mt = d.mt;
    p.kt = d.kt;
    p.mode_a = MODE_RAW;
    p.mode_b = MODE_RAW;
    typename K::AccT acc;
    // fringe shortcuts for every grouped tile; the half-height micro-tile only where the
    // registers allow it (FP64, the 64-thread FP32 tile), not in the 128-register FP32 tile
    constexpr int FRINGE = (std::is_same<T, double>::value || Cfg::THREADS <= 64) ? 2 : 1;
    K::template run_segment<FRINGE>(p, sm, i, j, 0, d.kt, acc, 0u);
    K::epilogue(p, i, j, acc);
}

template <typename T, typename Cfg>
__global__ void __launch_bounds__(Cfg::THREADS, Cfg::MIN_BLOCKS)
    grouped_kernel(const GroupDesc<T> *desc, const int *prefix, int count)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    GemmSmem<T, Cfg> &sm = *reinterpret_cast<GemmSmem<T, Cfg> *>(smem_raw);
    const int total = prefix[count];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        // problem of tile t: the last g with prefix[g] <= t
        int lo = 0, hi = count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        const GroupDesc<T> d = desc[lo];
        const int local = t - prefix[lo];
        const int i = local % d.mt, j = local / d.mt;
        switch (d.order) {
        case 0: grouped_tile<T, Cfg, false, false>(d, sm, i, j); break;
        case 1: grouped_tile<T, Cfg, true, false>(d, sm, i, j); break;
        case 2: grouped_tile<T, Cfg, false, true>(d, sm, i, j); break;
        default: grouped_tile<T, Cfg, true, true>(d, sm, i, j); break;
        }
        __syncthreads();
    }
}

template <typename T, typename Cfg> int grouped_grid()
{
    static int grid = 0;
    if (grid == 0) {
        const size_t smem = sizeof(GemmSmem<T, Cfg>);
        cudaFuncSetAttribute(grouped_kernel<T, Cfg>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem));
        int per = 0, dev = 0, sms = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, grouped_kernel<T, Cfg>, Cfg::THREADS,
                                                      smem);
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        grid = (per > 0 ? per : 1) * sms;
    }
    return grid;
}

template <typename T, typename Cfg>
cudaError_t launch_grouped_cfg(const GroupParams<T> &gp, cudaStream_t s)
{
    const int threads = 128;
    grouped_prepare_kernel<T, Cfg::BM, Cfg::BN, Cfg::BK>
        <<<(gp.count + threads - 1) / threads, threads, 0, s>>>(gp);
    grouped_scan_kernel<<<1, 1024, 0, s>>>(gp.prefix, gp.count);
    grouped_kernel<T, Cfg><<<grouped_grid<T, Cfg>(), Cfg::THREADS, sizeof(GemmSmem<T, Cfg>), s>>>(
        gp.desc, gp.prefix, gp.count);
    return cudaGetLastError();
}

template <> cudaError_t launch_grouped<double>(const GroupParams<double> &gp, int tile, cudaStream_t s)
{
    (void)tile;   // one FP64 tile: the DFMA-bound 32 x 32 tile already suits small problems
    return launch_grouped_cfg<double, TileCfg<double>>(gp, s);
}

template <> cudaError_t launch_grouped<float>(const GroupParams<float> &gp, int tile, cudaStream_t s)
{
    if (tile == GROUP_TILE_SMALL) return launch_grouped_cfg<float, TileCfgF32Small>(gp, s);
    return launch_grouped_cfg<float, TileCfg<float>>(gp, s);
}

}  // namespace gfip
