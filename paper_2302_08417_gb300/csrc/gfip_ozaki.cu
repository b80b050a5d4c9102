// gfip_ozaki.cu -- FP64 GEMM emulated on the tcgen05 tensor cores with exact BF16 digit
// products (the Ozaki splitting scheme: Ozaki, Ogita, Oishi, Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix multiplication
// and its applications", Numer. Algorithms 59 (2012); here with BF16 digits and FP32
// accumulation).
//
// Splitting (a pack-time transform, like the slicing that the GEMMFIP paper's future work,
// Sec. 5, folds into packing): every row i of op(A) gets an exponent e_i with
// max_p |a_ip| < 2^e_i, and every element becomes exactly
//     a_ip = 2^(e_i + 1) * (sum_{s=1..S} d_s * 2^(-6 s) + r),   |d_s| <= 32,
// with integer digits d_s (exact in BF16) and |r| <= 2^(-6 S - 1) (the scaled element is below
// 1/2, so even the first digit is at most 32).  Columns of op(B) are split the same way with
// exponents f_j.  A product of two digits is an integer of at most 2^10, so a sum of up to
// 16384 of them is an integer of at most 2^24 and the tensor cores' FP32 accumulation of such
// a k-chunk is exact.  The product is recombined in FP64:
//     C_ij = alpha * 2^(e_i + f_j + 2) * sum_{s+t <= S+1} 2^(-6(s+t)) * sum_chunks D_st
//            + beta * C_ij,
// dropping the digit pairs with s + t > S + 1 (triangular truncation).
//
// Kernel layout (one CTA per 128 x 128 tile of C, 10 warps).  A "job" is one digit pair
// (s, t) over one k-chunk, accumulated exactly in one 128-column FP32 accumulator; jobs with
// the same A digit s run two at a time ("steps"), so a stage holds one A-digit tile and two
// B-digit tiles and feeds two MMAs:
//   warp 0      producer: bulk-copies the digit tiles (16 KB each, stored already in the
//               swizzled shared-memory layout the MMA reads) into a 4-stage ring;
//   warp 1      allocates tensor memory and issues tcgen05.mma (one thread) into four
//               128-column FP32 accumulators, two filling while two drain;
//   warps 2-9   drain a finished accumulator with tcgen05.ld and add it, scaled, into FP64
//               registers (64 values per thread), then write C.
// Every mbarrier wait is bounded by a global-timer budget; on a timeout the kernel raises a
// status bit, the roles skip their remaining work, the producer waits for its copies in
// flight, and tensor memory is released before exit.
#include <cstdint>

#include <cuda_bf16.h>

#include "gfip_internal.h"

namespace gfip {

namespace oz {

constexpr int TM = 128;              // tile rows (M of the MMA) and digit-tile rows
constexpr int TN = 128;              // tile cols (N of the MMA)
constexpr int KB = 64;               // k per digit tile: 64 BF16 = one 128-byte row
constexpr int TILE_BYTES = TM * KB * 2;  // 16 KB per digit tile (A and B alike)
constexpr int STAGES = 4;
constexpr int THREADS = 320;
constexpr int EPI_WARPS = 8;
constexpr int BETA_BITS = 6;         // bits per digit
constexpr int KC_BLOCKS = 16384 / KB; // k-blocks per exactly accumulated chunk
constexpr int NACC = 4;              // 128-column FP32 accumulators in tensor memory
constexpr uint32_t TMEM_COLS = NACC * TN;
constexpr unsigned STATUS_TIMEOUT = 0x2u;  // mirrors GFIP_STATUS_MMA_TIMEOUT
constexpr long long WAIT_POLLS = 1ll << 32;  // backstop on polls, should the timer stall

struct Smem {
    uint8_t a[STAGES][TILE_BYTES];      // 1024-byte aligned (swizzle atoms)
    uint8_t b[STAGES][2][TILE_BYTES];   // the step's one or two B-digit tiles
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    uint64_t tfull[NACC];
    uint64_t tempty[NACC];
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
};

__device__ __forceinline__ bool aborted(const Smem &sm)
{
    return *(volatile const int *)&sm.abort != 0;
}

__device__ __forceinline__ uint32_t saddr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    return done != 0;
}

// Waits for the phase with the given parity to complete; gives up after budget_ns of the
// global timer, or when another role has aborted.  Returns false if it gave up; a timeout
// sets the CTA's abort flag and the status bit.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, Smem &sm,
                                          unsigned *status, unsigned long long budget_ns)
{
    const uint32_t a = saddr(bar);
    const unsigned long long t0 = global_ns();
    for (long long it = 0; it < WAIT_POLLS; ++it) {
        if (mbar_try(a, parity)) return true;
        if (aborted(sm)) return false;
        if ((it & 63) == 63 && global_ns() - t0 > budget_ns) break;
    }
    *(volatile int *)&sm.abort = 1;
    atomicOr(status, STATUS_TIMEOUT);
    return false;
}

// The same wait, used while draining after an abort: ignores the abort flag and raises
// nothing; returns false if the budget ran out.
__device__ __forceinline__ bool mbar_wait_drain(uint64_t *bar, uint32_t parity,
                                                unsigned long long budget_ns)
{
    const uint32_t a = saddr(bar);
    const unsigned long long t0 = global_ns();
    for (long long it = 0; it < WAIT_POLLS; ++it) {
        if (mbar_try(a, parity)) return true;
        if ((it & 63) == 63 && global_ns() - t0 > budget_ns) break;
    }
    return false;
}

// 16 KB global -> shared bulk copy (TMA engine), completing on an mbarrier.
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes,
                                          uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(saddr(dst)), "l"(src), "r"(bytes), "r"(saddr(bar))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile in the 128-byte swizzle layout: 8-row
// groups of 128-byte rows, 1024 bytes apart (stride byte offset); descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);        // start address
    d |= (uint64_t)1 << 16;                        // leading byte offset (unused here)
    d |= (uint64_t)(1024 >> 4) << 32;              // stride byte offset
    d |= (uint64_t)1 << 46;                        // descriptor version
    d |= (uint64_t)2 << 61;                        // 128-byte swizzle
    return d;
}

// Instruction descriptor: kind::f16 with BF16 A and B, FP32 D, both K-major, M = 128, N = 128.
constexpr uint32_t IDESC = (1u << 4)                      // D: F32
                           | (1u << 7)                    // A: BF16
                           | (1u << 10)                   // B: BF16
                           | ((uint32_t)(TN >> 3) << 17)  // N
                           | ((uint32_t)(TM >> 4) << 24); // M

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            saddr(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 16 consecutive FP32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_wait_ld()
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Byte offset of element (r, c) (r < 128 rows, c < 64 k) in a digit tile: 8-row groups of
// 1024 bytes; inside a group, row r%8 is 128 bytes whose 16-byte chunks are XOR-permuted by r%8.
__device__ __forceinline__ uint32_t digit_off(int r, int c)
{
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((c >> 3) ^ (r & 7))) << 4) +
                      (c & 7) * 2);
}

// ---- splitting ---------------------------------------------------------------------------

// Exponent of each row: e with max_p |x_rp| < 2^e.  Block (rb, ks) covers rows
// rb*128 .. +127 and the ks-th of KS equal k-ranges and writes the exponent of its partial
// maximum (NO_EXP for an all-zero range) to part[ks * rows_pad + r]; row_exp() takes the
// maximum over the KS parts (the exponent of a maximum is the maximum of the exponents).
// Row r of the operand has element (r, p) at X[r + p*ld] when contig_rows, else X[p + r*ld].
constexpr int NO_EXP = -(1 << 20);

// |x| as an integer with the same order as the magnitudes of finite doubles.
__device__ __forceinline__ unsigned long long mag_bits(double x)
{
    return static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7FFFFFFFFFFFFFFFull;
}

// e with |x| < 2^e for the double whose magnitude bits are b (NO_EXP for zero).
__device__ __forceinline__ int exp_of(unsigned long long b)
{
    if (b == 0) return NO_EXP;
    const int ex = static_cast<int>(b >> 52);
    if (ex == 0) return -1074 + 64 - __clzll(static_cast<long long>(b));  // subnormal
    return ex - 1022;   // |x| = 1.f * 2^(ex-1023) < 2^(ex-1022)
}

__global__ void __launch_bounds__(256) row_exponent_kernel(const double *X, int64_t ld,
                                                           int rows, int kdim, int contig_rows,
                                                           int row_blocks, int ks_count,
                                                           int *part)
{
    __shared__ unsigned long long red[256];
    const int tid = threadIdx.x;
    const int rb = blockIdx.x % row_blocks, ks = blockIdx.x / row_blocks;
    const int rows_pad = row_blocks * TM;
    const int kr = (kdim + ks_count - 1) / ks_count;
    const int p0 = ks * kr, p1 = min(kdim, p0 + kr);
    const int r0 = rb * TM;
    if (contig_rows) {
        // two threads per row, consecutive rows in consecutive threads
        const int r = r0 + (tid % TM);
        unsigned long long mx = 0;
        if (r < rows)
            for (int p = p0 + tid / TM; p < p1; p += 2) {
                const unsigned long long b = mag_bits(X[r + (int64_t)p * ld]);
                mx = b > mx ? b : mx;
            }
        red[tid] = mx;
        __syncthreads();
        if (tid < TM) {
            const unsigned long long a = red[tid], b = red[tid + TM];
            part[ks * rows_pad + r0 + tid] = exp_of(a > b ? a : b);
        }
    } else {
        // one warp per row, lanes along the contiguous k
        const int lane = tid & 31, w = tid >> 5;
        for (int rr = w; rr < TM; rr += 8) {
            const int r = r0 + rr;
            unsigned long long m2 = 0;
            if (r < rows)
                for (int p = p0 + lane; p < p1; p += 32) {
                    const unsigned long long b = mag_bits(X[p + (int64_t)r * ld]);
                    m2 = b > m2 ? b : m2;
                }
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long b = __shfl_xor_sync(0xffffffffu, m2, o);
                m2 = b > m2 ? b : m2;
            }
            if (lane == 0) part[ks * rows_pad + r] = exp_of(m2);
        }
    }
}

// Row exponent from the KS partial exponents (0 for an all-zero row).
__device__ __forceinline__ int row_exp(const int *part, int ks_count, int rows_pad, int r)
{
    int e = NO_EXP;
    for (int ks = 0; ks < ks_count; ++ks) e = max(e, part[ks * rows_pad + r]);
    return e == NO_EXP ? 0 : e;
}

// x * 2^-(e+1) as a signed fixed-point number with 63 fractional bits, truncated toward zero
// (|x| < 2^e, so the result is below 2^62 in magnitude).  Integer operations on the IEEE bit
// pattern only.  For an integer x the truncation drops nothing.
__device__ __forceinline__ long long to_fixed(double x, int e)
{
    const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(x));
    const int ex = static_cast<int>((bits >> 52) & 0x7FF);
    long long mant = static_cast<long long>(bits & 0xFFFFFFFFFFFFFull);
    int ee = ex;
    if (ex == 0) ee = 1; else mant |= 1ll << 52;   // x = +-mant * 2^(ee - 1075)
    const int sh = ee - 1075 + 62 - e;              // x * 2^(62 - e) = mant * 2^sh
    long long v;
    if (sh >= 0) v = mant << sh;
    else v = (sh > -64) ? (mant >> -sh) : 0;
    return (bits >> 63) ? -v : v;
}

// Digit tiles of one 128 x 64 block: every element is scaled by 2^-(e_row+1) (below 1/2) and
// split into S base-64 digits by round-to-nearest on a 63-bit fixed-point copy, all in
// integer arithmetic: d_s = round(X / 2^(63-6s)), X -= d_s * 2^(63-6s).  Digit s of all elements
// is staged in shared memory in the swizzled tile layout, then written out with 16-byte
// stores.  Fringe rows and k positions give zero digits.
__global__ void __launch_bounds__(256) split_kernel(const double *X, int64_t ld, int rows,
                                                    int kdim, int contig_rows, int S,
                                                    const int *part, int ks_count,
                                                    uint16_t *tiles, int row_blocks, int kblocks)
{
    __shared__ __align__(1024) uint8_t stage[TILE_BYTES];
    __shared__ int expo[TM];
    const int tid = threadIdx.x;
    const int rb = blockIdx.x % row_blocks, kb = blockIdx.x / row_blocks;
    if (tid < TM) expo[tid] = row_exp(part, ks_count, row_blocks * TM, rb * TM + tid);
    __syncthreads();
    constexpr int PER = TM * KB / 256;   // 32 elements per thread
    long long rem[PER];
    uint32_t off[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        int r, c;
        if (contig_rows) {          // consecutive threads on consecutive rows
            r = tid % TM;
            c = tid / TM + 2 * q;
        } else {                    // consecutive threads on consecutive k
            c = tid % KB;
            r = tid / KB + 4 * q;
        }
        off[q] = digit_off(r, c);
        const int gr = rb * TM + r, gc = kb * KB + c;
        double v = 0.0;
        if (gr < rows && gc < kdim)
            v = contig_rows ? X[gr + (int64_t)gc * ld] : X[gc + (int64_t)gr * ld];
        rem[q] = (gr < rows) ? to_fixed(v, expo[r]) : 0;
    }
    for (int s = 0; s < S; ++s) {
        const int sh = 63 - 6 * (s + 1);   // the digit's weight, >= 3 for S <= 10
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const long long d = (rem[q] + (1ll << (sh - 1))) >> sh;   // round to nearest
            rem[q] -= d << sh;                                       // |rem| <= 2^(sh-1)
            // |d| <= 32: exact in BF16
            *reinterpret_cast<__nv_bfloat16 *>(stage + off[q]) =
                __int2bfloat16_rn(static_cast<int>(d));
        }
        __syncthreads();
        uint4 *dst = reinterpret_cast<uint4 *>(
            tiles + (((int64_t)s * row_blocks + rb) * kblocks + kb) * (TM * KB));
        const uint4 *src = reinterpret_cast<const uint4 *>(stage);
        for (int c = tid; c < TILE_BYTES / 16; c += 256) dst[c] = src[c];
        __syncthreads();
    }
}

// ---- digit-product GEMM with FP64 recombination -----------------------------------------

// Work list of one tile, per k-chunk: jobs (s, t), s = 1..S, t = 1..S+1-s, in that order;
// the jobs of one s form steps of two (the last may be single).
struct Step {
    int s, t0, count, job;   // A digit, first B digit, jobs in the step, job index of the first
};

__device__ __forceinline__ Step step_of(int q, int slices, int pairs, int steps_per_chunk)
{
    const int chunk = q / steps_per_chunk;
    int r = q - chunk * steps_per_chunk;
    int before = 0;   // jobs of smaller s in this chunk
    for (int s = 1; s <= slices; ++s) {
        const int n = slices + 1 - s, g = (n + 1) / 2;
        if (r < g) return Step{s, 1 + 2 * r, min(2, n - 2 * r), chunk * pairs + before + 2 * r};
        r -= g;
        before += n;
    }
    return Step{0, 0, 0, 0};
}

struct Job {
    int s, t;
};

__device__ __forceinline__ Job job_of(int j, int slices, int pairs)
{
    int r = j % pairs;
    for (int s = 1; s <= slices; ++s) {
        const int n = slices + 1 - s;
        if (r < n) return Job{s, 1 + r};
        r -= n;
    }
    return Job{0, 0};
}

__device__ __forceinline__ int steps_per_chunk(int slices)
{
    int g = 0;
    for (int s = 1; s <= slices; ++s) g += (slices + 2 - s) / 2;
    return g;
}

__global__ void __launch_bounds__(THREADS, 1) ozaki_kernel(const OzakiParams p)
{
    extern __shared__ uint8_t smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // CTAs that run at the same time cover a band of GROUP tile-rows, so they share digit
    // panels of A (within the band) and of B (across it) in L2
    constexpr int GROUP = 8;
    const int band = blockIdx.x / (GROUP * p.nt);
    const int in_band = blockIdx.x % (GROUP * p.nt);
    const int rows_in_band = min(GROUP, p.mt - band * GROUP);
    const int ib = band * GROUP + in_band % rows_in_band;
    const int jb = in_band / rows_in_band;
    const int nchunks = (p.kt + KC_BLOCKS - 1) / KC_BLOCKS;
    const int pairs = p.slices * (p.slices + 1) / 2;
    const int spc = steps_per_chunk(p.slices);
    const int nsteps = spc * nchunks;
    const int njobs = pairs * nchunks;

    if (tid == 0) {
        for (int i = 0; i < STAGES; ++i) {
            mbar_init(&sm.full[i], 1);
            mbar_init(&sm.empty[i], 1);
        }
        for (int i = 0; i < NACC; ++i) {
            mbar_init(&sm.tfull[i], 1);
            mbar_init(&sm.tempty[i], EPI_WARPS);
        }
        mbar_init(&sm.drain, 1);
        sm.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         saddr(&sm.tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            long long issued = 0;   // stages handed to the copy engine (or withheld)
            const bool withhold = p.inject_timeout && blockIdx.x == 0;
            for (int q = 0; q < nsteps && !aborted(sm); ++q) {
                const Step x = step_of(q, p.slices, pairs, spc);
                const int k0 = (q / spc) * KC_BLOCKS;
                const int k1 = min(p.kt, k0 + KC_BLOCKS);
                bool ok = true;
                for (int kb = k0; kb < k1; ++kb) {
                    if (!mbar_wait(&sm.empty[stage], phase ^ 1, sm, p.status, p.wait_ns)) {
                        ok = false;
                        break;
                    }
                    if (!(withhold && issued == 0)) {
                        mbar_expect_tx(&sm.full[stage], (1 + x.count) * TILE_BYTES);
                        const uint16_t *ta =
                            p.sa + (((int64_t)(x.s - 1) * p.mt + ib) * p.kt + kb) * (TM * KB);
                        bulk_copy(sm.a[stage], ta, TILE_BYTES, &sm.full[stage]);
                        for (int c = 0; c < x.count; ++c) {
                            const uint16_t *tb =
                                p.sb + (((int64_t)(x.t0 + c - 1) * p.nt + jb) * p.kt + kb) *
                                           (TN * KB);
                            bulk_copy(sm.b[stage][c], tb, TILE_BYTES, &sm.full[stage]);
                        }
                    }
                    ++issued;
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
                if (!ok) break;
            }
            // No bulk copy may still be writing shared memory when the CTA exits: wait for
            // the last STAGES stages handed out (each is in the phase it was issued in; one
            // the consumer already took has completed that phase).  The withheld stage, if
            // any, has nothing in flight.
            for (int d = 1; d <= STAGES && d <= issued; ++d) {
                if (--stage < 0) {
                    stage = STAGES - 1;
                    phase ^= 1;
                }
                if (withhold && issued - d == 0) continue;
                mbar_wait_drain(&sm.full[stage], phase, p.wait_ns);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            for (int q = 0; q < nsteps && !aborted(sm); ++q) {
                const Step x = step_of(q, p.slices, pairs, spc);
                bool ok = true;
                for (int c = 0; c < x.count && ok; ++c) {
                    const int j = x.job + c;
                    ok = mbar_wait(&sm.tempty[j % NACC], ((uint32_t)(j / NACC) & 1u) ^ 1u, sm,
                                   p.status, p.wait_ns);
                }
                if (!ok) break;
                tc_fence_after();
                const int k0 = (q / spc) * KC_BLOCKS;
                const int k1 = min(p.kt, k0 + KC_BLOCKS);
                for (int kb = k0; kb < k1; ++kb) {
                    if (!mbar_wait(&sm.full[stage], phase, sm, p.status, p.wait_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = saddr(sm.a[stage]);
                    for (int c = 0; c < x.count; ++c) {
                        const uint32_t dcol = tmem + (uint32_t)(((x.job + c) % NACC) * TN);
                        const uint32_t b0 = saddr(sm.b[stage][c]);
#pragma unroll
                        for (int kk = 0; kk < KB / 16; ++kk)
                            mma_bf16(dcol, smem_desc(a0 + kk * 32), smem_desc(b0 + kk * 32),
                                     (kb > k0 || kk > 0) ? 1u : 0u);
                    }
                    mma_commit(&sm.empty[stage]);
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
                if (!ok) break;
                for (int c = 0; c < x.count; ++c) mma_commit(&sm.tfull[(x.job + c) % NACC]);
            }
            // all MMAs this thread issued have completed once this commit arrives
            mma_commit(&sm.drain);
            mbar_wait_drain(&sm.drain, 0, p.wait_ns);
        }
    } else {
        // epilogue warps: TMEM lane quarter from warp % 4, column half from (warp - 2) / 4
        const int quarter = warp & 3, half = (warp - 2) >> 2;
        const int row = ib * TM + quarter * 32 + lane;
        double acc[64];
#pragma unroll
        for (int c = 0; c < 64; ++c) acc[c] = 0.0;
        for (int j = 0; j < njobs; ++j) {
            const int buf = j % NACC;
            const uint32_t use = (uint32_t)(j / NACC);
            if (!mbar_wait(&sm.tfull[buf], use & 1, sm, p.status, p.wait_ns)) break;
            tc_fence_after();
            const Job x = job_of(j, p.slices, pairs);
            const double scale = ldexp(1.0, -BETA_BITS * (x.s + x.t));
            const uint32_t taddr =
                tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * TN + half * 64);
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                uint32_t r[16];
                tmem_ld16(taddr + g * 16, r);
                tmem_wait_ld();
#pragma unroll
                for (int c = 0; c < 16; ++c)
                    acc[g * 16 + c] = fma((double)__uint_as_float(r[c]), scale, acc[g * 16 + c]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.tempty[buf]);
        }
        if (!aborted(sm) && row < p.m) {
            const int er = row_exp(p.ea, p.ks_a, p.mt * TM, row) + 2;  // 2^(e_i+1) 2^(f_j+1)
            const bool read_c = (p.beta != 0.0);
#pragma unroll
            for (int c = 0; c < 64; ++c) {
                const int col = jb * TN + half * 64 + c;
                if (col < p.n) {
                    double v =
                        p.alpha * ldexp(acc[c], er + row_exp(p.eb, p.ks_b, p.nt * TN, col));
                    double *cp = p.C + row + (int64_t)col * p.ldc;
                    if (read_c) v = fma(p.beta, *cp, v);
                    *cp = v;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS)
                     : "memory");
}

}  // namespace oz

size_t ozaki_smem_bytes()
{
    return sizeof(oz::Smem) + 1024;
}

cudaError_t launch_ozaki(const OzakiParams &p, cudaStream_t s)
{
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(oz::ozaki_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(ozaki_smem_bytes()));
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int rb_a = p.mt, rb_b = p.nt;
    oz::row_exponent_kernel<<<rb_a * p.ks_a, 256, 0, s>>>(p.A, p.lda, p.m, p.k, p.a_contig_rows,
                                                           rb_a, p.ks_a, p.ea);
    oz::row_exponent_kernel<<<rb_b * p.ks_b, 256, 0, s>>>(p.B, p.ldb, p.n, p.k, p.b_contig_rows,
                                                           rb_b, p.ks_b, p.eb);
    oz::split_kernel<<<rb_a * p.kt, 256, 0, s>>>(p.A, p.lda, p.m, p.k, p.a_contig_rows,
                                                 p.slices, p.ea, p.ks_a, p.sa, rb_a, p.kt);
    oz::split_kernel<<<rb_b * p.kt, 256, 0, s>>>(p.B, p.ldb, p.n, p.k, p.b_contig_rows,
                                                 p.slices, p.eb, p.ks_b, p.sb, rb_b, p.kt);
    oz::ozaki_kernel<<<p.mt * p.nt, oz::THREADS, ozaki_smem_bytes(), s>>>(p);
    return cudaGetLastError();
}

}  // namespace gfip
