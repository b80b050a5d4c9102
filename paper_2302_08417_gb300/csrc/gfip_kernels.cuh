// gfip_kernels.cuh -- device code of the fused-in-packing GEMM (templated on FP64/FP32).
//
// One persistent kernel computes C := alpha*op(A)*op(B) + beta*C for column-major strided
// operands.  Three properties carry the paper's method onto the GPU:
//
//  * Packed layout = shared-memory image (Sec. 2.1, Fig. 2).  An operand tile (BX x BK of
//    op(A) or op(B)) lives in shared memory in a swizzled layout: 128-byte row segments along
//    x, one per k, whose 16-byte chunks are XOR-permuted by (k mod 8).  The packed copy of a
//    tile in global memory is byte-for-byte that image, so a CTA fetches a packed tile with
//    contiguous 16-byte copies and no address arithmetic, and fringes are zero-padded once,
//    when packing (Sec. 2.2).
//
//  * Fused-in packing (Sec. 3.1 Alg. 1, Sec. 3.2).  In MODE_FIP the first CTA that needs a
//    (panel, k-block) claims it with one atomic, reads the raw strided operand, computes with
//    it, and in the same pass writes the tile image to the packed buffer, then publishes it.
//    Every later CTA that needs it loads the packed copy.  A CTA that finds the tile claimed
//    but not yet published reads the raw operand itself and never waits, so there is no
//    inter-CTA wait anywhere in the kernel (Sec. 3.5: each packer packs its own share and
//    only consumers that come later use the packed data).
//
//  * One code path for all sizes.  Tiles are scheduled as data-parallel waves over the
//    persistent CTAs; the tiles of the last, partial wave (plus one full wave) are split
//    evenly along k over all CTAs ("stream-K"), and split tiles are summed in a fixed order
//    by whichever CTA finishes last.  The split points depend only on the problem shape and
//    the grid, so every variant (fused, direct, pack-then-compute) and every pack policy
//    produces identical bits: packing changes where a tile is read from, never its value.
#pragma once

#include <cstdint>

#include "gfip_internal.h"

namespace gfip {

constexpr unsigned int STATUS_BAD_SEGMENT = 0x1u;  // mirrors GFIP_STATUS_BAD_SEGMENT

enum Decision : int { DEC_RAW = 0, DEC_PACKED = 1, DEC_PRODUCE = 2 };

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Element copy global -> shared through L1, zero-filling the destination when !ok.
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

// Offset (in elements) of element (x, kk) inside a BX x BK operand tile.  x runs along m
// (for A) or n (for B), kk along k.  Rows of W = 128/sizeof(T) consecutive x form one
// 128-byte segment per kk; the 16-byte chunks of a segment are XOR-permuted by (kk mod 8).
template <typename T, int BK> __device__ __forceinline__ int tile_off(int x, int kk)
{
    constexpr int W = 128 / static_cast<int>(sizeof(T));
    constexpr int CH = 16 / static_cast<int>(sizeof(T));
    return (x / W) * (BK * W) + kk * W + ((x % W) ^ ((kk & 7) * CH));
}

// Raw strided tile load: element (x, kk) of the BX x BK tile at (x0, k0) of op(X), X = A
// (x = row of op(A)) or B (x = column of op(B)), into shared memory at sdst.  Positions
// outside the X_ext x K_ext operand are zero-filled.  contig_x: element at g[x + kk*ld],
// else at g[kk + x*ld].  Either way consecutive lanes read consecutive addresses, and the
// swizzle keeps the shared-memory writes free of bank conflicts.
template <typename T, int BX, int BK, int THREADS>
__device__ __forceinline__ void load_raw_tile(uint32_t sdst, const T *__restrict__ g, int64_t ld,
                                              int x0, int k0, int x_ext, int k_ext, int contig_x,
                                              int tid)
{
    constexpr int PER = BX * BK / THREADS;
    static_assert(PER * THREADS == BX * BK, "tile must divide over the threads");
    if (contig_x) {
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int e = tid + r * THREADS;
            const int x = e % BX, kk = e / BX;
            const int gx = x0 + x, gk = k0 + kk;
            const bool ok = (gx < x_ext) && (gk < k_ext);
            const T *src = ok ? g + (int64_t)gx + (int64_t)gk * ld : g;
            cp_async_elem<sizeof(T)>(sdst + tile_off<T, BK>(x, kk) * sizeof(T), src, ok);
        }
    } else {
        // a warp covers 4 consecutive x by 8 consecutive k: 4 runs of 8 contiguous elements
        const int lane = tid & 31, w = tid >> 5;
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int b = w + r * (THREADS / 32);
            const int x = (b % (BX / 4)) * 4 + (lane >> 3);
            const int kk = (b / (BX / 4)) * 8 + (lane & 7);
            const int gx = x0 + x, gk = k0 + kk;
            const bool ok = (gx < x_ext) && (gk < k_ext);
            const T *src = ok ? g + (int64_t)gk + (int64_t)gx * ld : g;
            cp_async_elem<sizeof(T)>(sdst + tile_off<T, BK>(x, kk) * sizeof(T), src, ok);
        }
    }
}

// Packed tile load: the packed tile is the shared-memory image, copied in 16-byte pieces.
template <typename T, int BX, int BK, int THREADS>
__device__ __forceinline__ void load_packed_tile(uint32_t sdst, const T *src, int tid)
{
    constexpr int CHUNKS = BX * BK * static_cast<int>(sizeof(T)) / 16;
    const char *s = reinterpret_cast<const char *>(src);
#pragma unroll
    for (int c = tid; c < CHUNKS; c += THREADS) cp_async_16(sdst + c * 16, s + c * 16);
}

// Writes the shared-memory image of a tile to its packed slot (the fused pack store).
template <typename T, int BX, int BK, int THREADS>
__device__ __forceinline__ void store_packed_tile(T *dst, const T *stile, int tid)
{
    constexpr int CHUNKS = BX * BK * static_cast<int>(sizeof(T)) / 16;
    const uint4 *s = reinterpret_cast<const uint4 *>(stile);
    uint4 *d = reinterpret_cast<uint4 *>(dst);
#pragma unroll
    for (int c = tid; c < CHUNKS; c += THREADS) __stcg(d + c, s[c]);
}

// Claims or looks up one (panel, k-block) of a packed operand.  The word holds
// (epoch << 32) | ready.  One atomic max with (epoch << 32) returns the previous value:
// an older epoch means nobody has claimed the tile in this call, so this CTA now owns it and
// packs it; (epoch << 32) | 0 means another CTA is packing it right now (read raw);
// (epoch << 32) | 1 means it is published (read packed).  The fetch and the classification
// are separate so the atomic's latency overlaps the compute of the current k-block.
__device__ __forceinline__ unsigned long long claim_fetch(unsigned long long *word,
                                                          unsigned int epoch)
{
    const unsigned long long tag = static_cast<unsigned long long>(epoch) << 32;
    unsigned long long old;
    asm volatile("atom.acquire.gpu.global.max.u64 %0, [%1], %2;\n"
                 : "=l"(old)
                 : "l"(word), "l"(tag)
                 : "memory");
    return old;
}

__device__ __forceinline__ int claim_classify(unsigned long long old, unsigned int epoch)
{
    const unsigned long long tag = static_cast<unsigned long long>(epoch) << 32;
    if (old == (tag | 1ull)) return DEC_PACKED;
    if (old < tag) return DEC_PRODUCE;
    return DEC_RAW;
}

// Marks a packed tile as published.  Called by thread 0 after a CTA barrier that follows
// every thread's pack stores of that tile.
__device__ __forceinline__ void publish(unsigned long long *word, unsigned int epoch)
{
    const unsigned long long v = (static_cast<unsigned long long>(epoch) << 32) | 1ull;
    __threadfence();
    asm volatile("red.release.gpu.global.max.u64 [%0], %1;\n" ::"l"(word), "l"(v) : "memory");
}

template <typename T> struct GemmSmem {
    using Cfg = TileCfg<T>;
    T a[Cfg::STAGES][Cfg::BM * Cfg::BK];
    T b[Cfg::STAGES][Cfg::BN * Cfg::BK];
    int dec_a[2 * Cfg::STAGES];
    int dec_b[2 * Cfg::STAGES];
    int flag;
};

template <typename T> struct Vec16;
template <> struct Vec16<double> {
    using type = double2;
};
template <> struct Vec16<float> {
    using type = float4;
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

template <typename T> struct Kernel {
    using Cfg = TileCfg<T>;
    static constexpr int BM = Cfg::BM, BN = Cfg::BN, BK = Cfg::BK;
    static constexpr int THREADS = Cfg::THREADS, STAGES = Cfg::STAGES;
    static constexpr int CH = 16 / static_cast<int>(sizeof(T));
    static constexpr int TM = 2 * CH, TN = 2 * CH;  // register micro-tile
    static constexpr int TX = BM / TM;               // threads along m
    static_assert(TX * (BN / TN) == THREADS, "thread grid must cover the tile");
    static constexpr int DEC = 2 * STAGES;

    // Decision for one operand tile under a launch mode, in two steps (see claim_fetch).
    static __device__ __forceinline__ unsigned long long fetch(int mode, unsigned long long *state,
                                                               unsigned int epoch)
    {
        return mode == MODE_FIP ? claim_fetch(state, epoch) : 0ull;
    }
    static __device__ __forceinline__ int classify(int mode, unsigned long long old,
                                                   unsigned int epoch)
    {
        if (mode == MODE_RAW) return DEC_RAW;
        if (mode == MODE_PACKED) return DEC_PACKED;
        return claim_classify(old, epoch);
    }

    static __device__ __forceinline__ void issue(const GemmParams<T> &p, GemmSmem<T> &sm,
                                                 int i, int j, int kb, int q, int tid)
    {
        const int stage = q % STAGES;
        const int da = sm.dec_a[q % DEC], db = sm.dec_b[q % DEC];
        const uint32_t sa = smem_addr(sm.a[stage]), sb = smem_addr(sm.b[stage]);
        if (da == DEC_PACKED)
            load_packed_tile<T, BM, BK, THREADS>(
                sa, p.pack_a + ((int64_t)i * p.kt + kb) * (BM * BK), tid);
        else
            load_raw_tile<T, BM, BK, THREADS>(sa, p.A, p.lda, i * BM, kb * BK, p.m, p.k,
                                              p.a_contig_m, tid);
        if (db == DEC_PACKED)
            load_packed_tile<T, BN, BK, THREADS>(
                sb, p.pack_b + ((int64_t)j * p.kt + kb) * (BN * BK), tid);
        else
            load_raw_tile<T, BN, BK, THREADS>(sb, p.B, p.ldb, j * BN, kb * BK, p.n, p.k,
                                              p.b_contig_n, tid);
    }

    static __device__ __forceinline__ void compute(const T *As, const T *Bs, T (&acc)[TM][TN],
                                                   int tx, int ty)
    {
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[TM], b[TN];
            lds16<T>(a, As + tile_off<T, BK>(tx * CH, kk));
            lds16<T>(a + CH, As + tile_off<T, BK>(BM / 2 + tx * CH, kk));
            lds16<T>(b, Bs + tile_off<T, BK>(ty * CH, kk));
            lds16<T>(b + CH, Bs + tile_off<T, BK>(BN / 2 + ty * CH, kk));
#pragma unroll
            for (int ii = 0; ii < TM; ++ii)
#pragma unroll
                for (int jj = 0; jj < TN; ++jj) acc[ii][jj] = fma(a[ii], b[jj], acc[ii][jj]);
        }
    }

    // Accumulates op(A)[tile rows, kb0*BK : kb1*BK] * op(B)[..., tile cols] into acc, packing
    // operand tiles on the way where this CTA won the claim.
    static __device__ void run_segment(const GemmParams<T> &p, GemmSmem<T> &sm, int t, int kb0,
                                       int kb1, T (&acc)[TM][TN])
    {
        const int tid = threadIdx.x;
        const int tx = tid % TX, ty = tid / TX;
        const int i = t % p.mt, j = t / p.mt;
        const int nkb = kb1 - kb0;

#pragma unroll
        for (int ii = 0; ii < TM; ++ii)
#pragma unroll
            for (int jj = 0; jj < TN; ++jj) acc[ii][jj] = T(0);

        if (tid == 0) {
            unsigned long long oa[STAGES], ob[STAGES];
#pragma unroll
            for (int q = 0; q < STAGES; ++q) {
                if (q < nkb) {
                    oa[q] = fetch(p.mode_a, p.state_a + (int64_t)i * p.kt + kb0 + q, p.epoch);
                    ob[q] = fetch(p.mode_b, p.state_b + (int64_t)j * p.kt + kb0 + q, p.epoch);
                }
            }
#pragma unroll
            for (int q = 0; q < STAGES; ++q) {
                if (q < nkb) {
                    sm.dec_a[q] = classify(p.mode_a, oa[q], p.epoch);
                    sm.dec_b[q] = classify(p.mode_b, ob[q], p.epoch);
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < STAGES - 1; ++q) {
            if (q < nkb) issue(p, sm, i, j, kb0 + q, q, tid);
            cp_async_commit();
        }

        for (int it = 0; it < nkb; ++it) {
            cp_async_wait<STAGES - 2>();
            __syncthreads();
            const int stage = it % STAGES;
            if (tid == 0 && it > 0) {
                if (sm.dec_a[(it - 1) % DEC] == DEC_PRODUCE)
                    publish(p.state_a + (int64_t)i * p.kt + kb0 + it - 1, p.epoch);
                if (sm.dec_b[(it - 1) % DEC] == DEC_PRODUCE)
                    publish(p.state_b + (int64_t)j * p.kt + kb0 + it - 1, p.epoch);
            }
            if (sm.dec_a[it % DEC] == DEC_PRODUCE)
                store_packed_tile<T, BM, BK, THREADS>(
                    p.pack_a + ((int64_t)i * p.kt + kb0 + it) * (BM * BK), sm.a[stage], tid);
            if (sm.dec_b[it % DEC] == DEC_PRODUCE)
                store_packed_tile<T, BN, BK, THREADS>(
                    p.pack_b + ((int64_t)j * p.kt + kb0 + it) * (BN * BK), sm.b[stage], tid);
            const int q = it + STAGES - 1;
            if (q < nkb) issue(p, sm, i, j, kb0 + q, q, tid);
            cp_async_commit();
            // claims for k-block it+STAGES: fetched now, classified after this block's compute
            const bool ahead = (tid == 0) && (it + STAGES < nkb);
            unsigned long long oa = 0, ob = 0;
            if (ahead) {
                oa = fetch(p.mode_a, p.state_a + (int64_t)i * p.kt + kb0 + it + STAGES, p.epoch);
                ob = fetch(p.mode_b, p.state_b + (int64_t)j * p.kt + kb0 + it + STAGES, p.epoch);
            }
            compute(sm.a[stage], sm.b[stage], acc, tx, ty);
            if (ahead) {
                sm.dec_a[(it + STAGES) % DEC] = classify(p.mode_a, oa, p.epoch);
                sm.dec_b[(it + STAGES) % DEC] = classify(p.mode_b, ob, p.epoch);
            }
        }
        cp_async_wait<0>();
        __syncthreads();
        if (tid == 0 && nkb > 0) {
            if (sm.dec_a[(nkb - 1) % DEC] == DEC_PRODUCE)
                publish(p.state_a + (int64_t)i * p.kt + kb0 + nkb - 1, p.epoch);
            if (sm.dec_b[(nkb - 1) % DEC] == DEC_PRODUCE)
                publish(p.state_b + (int64_t)j * p.kt + kb0 + nkb - 1, p.epoch);
        }
    }

    // C[tile] := alpha*acc + beta*C[tile]; C is not read when beta == 0.
    static __device__ void epilogue(const GemmParams<T> &p, int t, const T (&acc)[TM][TN])
    {
        const int tid = threadIdx.x;
        const int tx = tid % TX, ty = tid / TX;
        const int m0 = (t % p.mt) * BM, n0 = (t / p.mt) * BN;
        const bool read_c = (p.beta != T(0));
#pragma unroll
        for (int jj = 0; jj < TN; ++jj) {
            const int col = n0 + ty * CH + (jj % CH) + (jj / CH) * (BN / 2);
            if (col >= p.n) continue;
            T *ccol = p.C + (int64_t)col * p.ldc;
#pragma unroll
            for (int ii = 0; ii < TM; ++ii) {
                const int row = m0 + tx * CH + (ii % CH) + (ii / CH) * (BM / 2);
                if (row >= p.m) continue;
                T v = p.alpha * acc[ii][jj];
                if (read_c) v = fma(p.beta, ccol[row], v);
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
    static __device__ void fixup(const GemmParams<T> &p, GemmSmem<T> &sm, int t, int g,
                                 int slot, T (&acc)[TM][TN])
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
            for (int jj = 0; jj < TN; ++jj) __stcg(mine + (ii * TN + jj) * THREADS + tid, acc[ii][jj]);
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            const unsigned long long tag = static_cast<unsigned long long>(p.epoch) << 32;
            atomicMax(p.tile_count + t, tag);
            const unsigned long long old = atomicAdd(p.tile_count + t, 1ull);
            const long long cnt = static_cast<long long>(old - tag) + 1;
            if ((old >> 32) != p.epoch || cnt > nseg) atomicOr(p.status, STATUS_BAD_SEGMENT);
            sm.flag = (cnt == nseg);
            __threadfence();
        }
        __syncthreads();
        if (sm.flag) {
            for (int gg = g0; gg <= g1; ++gg) {
                const int64_t lo = S * gg / G;
                const int gslot = (lo / p.kt == u) ? 0 : 1;
                const T *src = p.partial + (int64_t)(2 * gg + gslot) * (BM * BN);
#pragma unroll
                for (int ii = 0; ii < TM; ++ii)
#pragma unroll
                    for (int jj = 0; jj < TN; ++jj) {
                        const T v = __ldcg(src + (ii * TN + jj) * THREADS + tid);
                        acc[ii][jj] = (gg == g0) ? v : acc[ii][jj] + v;
                    }
            }
            epilogue(p, t, acc);
        }
        __syncthreads();
    }

    static __device__ void run(const GemmParams<T> &p, GemmSmem<T> &sm)
    {
        const int g = blockIdx.x;
        T acc[TM][TN];
        for (int t = g; t < p.dp_tiles; t += p.grid) {
            run_segment(p, sm, t, 0, p.kt, acc);
            epilogue(p, t, acc);
            __syncthreads();
        }
        if (p.sk_iters > 0) {
            const int64_t lo = p.sk_iters * g / p.grid, hi = p.sk_iters * (g + 1) / p.grid;
            const int first_u = static_cast<int>(lo / p.kt);
            int64_t q = lo;
            while (q < hi) {
                const int u = static_cast<int>(q / p.kt);
                const int t = p.dp_tiles + u;
                const int kb0 = static_cast<int>(q % p.kt);
                const int64_t rest = hi - q;
                const int kb1 = (rest < (int64_t)(p.kt - kb0)) ? kb0 + static_cast<int>(rest) : p.kt;
                run_segment(p, sm, t, kb0, kb1, acc);
                if (kb0 == 0 && kb1 == p.kt) {
                    epilogue(p, t, acc);
                    __syncthreads();
                } else {
                    fixup(p, sm, t, g, (u == first_u) ? 0 : 1, acc);
                }
                q += kb1 - kb0;
            }
        }
    }
};

template <typename T>
__global__ void __launch_bounds__(TileCfg<T>::THREADS, TileCfg<T>::MIN_BLOCKS)
    gemm_kernel(const GemmParams<T> p)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    GemmSmem<T> &sm = *reinterpret_cast<GemmSmem<T> *>(smem_raw);
    Kernel<T>::run(p, sm);
}

// Pack kernel of the pack-then-compute variant: block b packs one (panel, k-block) tile,
// A tiles first, through the same shared-memory staging as the GEMM kernel.
template <typename T>
__global__ void __launch_bounds__(TileCfg<T>::THREADS) pack_kernel(const PackParams<T> p)
{
    using Cfg = TileCfg<T>;
    constexpr int BM = Cfg::BM, BN = Cfg::BN, BK = Cfg::BK, THREADS = Cfg::THREADS;
    constexpr int BX = BM > BN ? BM : BN;
    __shared__ __align__(128) T tile[BX * BK];
    const int tid = threadIdx.x;
    const int64_t a_tiles = (int64_t)p.mt * p.kt;
    const int64_t b = blockIdx.x;
    if (b < a_tiles) {
        const int i = static_cast<int>(b / p.kt), kb = static_cast<int>(b % p.kt);
        load_raw_tile<T, BM, BK, THREADS>(smem_addr(tile), p.A, p.lda, i * BM, kb * BK, p.m, p.k,
                                          p.a_contig_m, tid);
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();
        store_packed_tile<T, BM, BK, THREADS>(p.pack_a + b * (BM * BK), tile, tid);
    } else {
        const int64_t bb = b - a_tiles;
        const int j = static_cast<int>(bb / p.kt), kb = static_cast<int>(bb % p.kt);
        load_raw_tile<T, BN, BK, THREADS>(smem_addr(tile), p.B, p.ldb, j * BN, kb * BK, p.n, p.k,
                                          p.b_contig_n, tid);
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();
        store_packed_tile<T, BN, BK, THREADS>(p.pack_b + bb * (BN * BK), tile, tid);
    }
}

// C := beta*C on the m x n region (beta == 0 writes zeros without reading C).
template <typename T>
__global__ void scale_kernel(T *C, int64_t ldc, int m, int n, T beta)
{
    const int64_t total = (int64_t)m * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t col = e / m, row = e % m;
        T *c = C + row + col * ldc;
        *c = (beta == T(0)) ? T(0) : beta * *c;
    }
}

template <typename T> inline size_t gemm_smem_bytes()
{
    return sizeof(GemmSmem<T>);
}

template <typename T> cudaError_t launch_gemm_impl(const GemmParams<T> &p, cudaStream_t s)
{
    static bool configured = false;
    const size_t smem = gemm_smem_bytes<T>();
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(gemm_kernel<T>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        configured = true;
    }
    gemm_kernel<T><<<p.grid, TileCfg<T>::THREADS, smem, s>>>(p);
    return cudaGetLastError();
}

template <typename T> int gemm_blocks_per_sm_impl()
{
    const size_t smem = gemm_smem_bytes<T>();
    cudaFuncSetAttribute(gemm_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gemm_kernel<T>, TileCfg<T>::THREADS,
                                                      smem) != cudaSuccess)
        return 0;
    return n;
}

template <typename T> cudaError_t launch_pack_impl(const PackParams<T> &p, cudaStream_t s)
{
    const int64_t blocks = (int64_t)(p.mt + p.nt) * p.kt;
    if (blocks <= 0) return cudaSuccess;
    pack_kernel<T><<<static_cast<unsigned int>(blocks), TileCfg<T>::THREADS, 0, s>>>(p);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scale_impl(T *C, int64_t ldc, int m, int n, T beta, cudaStream_t s)
{
    const int64_t total = (int64_t)m * n;
    const int threads = 256;
    int64_t blocks = (total + threads - 1) / threads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    scale_kernel<T><<<static_cast<unsigned int>(blocks), threads, 0, s>>>(C, ldc, m, n, beta);
    return cudaGetLastError();
}

}  // namespace gfip

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
    cudaError_t launch_scale<T>(T * C, int64_t ldc, int m, int n, T beta, cudaStream_t s)     \
    {                                                                                         \
        return launch_scale_impl<T>(C, ldc, m, n, beta, s);                                   \
    }                                                                                         \
    template <> int gemm_blocks_per_sm<T>()                                                   \
    {                                                                                         \
        return gemm_blocks_per_sm_impl<T>();                                                  \
    }                                                                                         \
    }
