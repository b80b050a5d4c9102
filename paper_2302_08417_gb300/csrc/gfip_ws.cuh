// gfip_ws.cuh -- warp-specialised FP32 tile core of the fused-in-packing GEMM.
//
// The FP32 GEMM is bound by the FFMA pipe.  When every thread of a CTA both loads operand
// tiles and computes (the tile core of gfip_kernels.cuh), the element-wise raw loads of the
// first pass, the ready-word look-ups with their acquire fences, and the barrier after every
// k-block all sit in the instruction stream of the FFMA warps: the math pipe idles while the
// warps of a CTA load and synchronise together, and a tile that reads the raw strided operand
// costs the FFMA loop about 10 % more than one that reads a packed copy.  Here the roles are
// split (Sec. 3.2's fused microkernel, with the "load and pack" half given its own warp):
//
//   math warps: wait until a stage is full, run the FFMA2 loop over its BK rows, release
//              the stage; accumulators, alpha/beta epilogue and the split-tile fix-up as in
//              the shared tile core (same micro-tile, same k order, so the same bits)
//   last warp:  producer: per k-block decides raw / packed / produce for each operand (the
//              ready-word look-ups and acquire fences happen here), fills the stage with
//              element copies of the raw strided operand or 128-byte bulk copies of the packed
//              tile (the copy engine), and for a producer tile (Alg. 1: the first tile column
//              packs A, the first tile row packs B) writes the staged tile to the packed buffer
//              with bulk stores once it has arrived, then publishes it
//
// A stage is handed over on mbarriers: `full` completes when the producer's 32 lanes have
// seen their element copies land (cp.async.mbarrier.arrive.noinc) and the bulk copies'
// bytes have arrived (expect_tx); `empty` completes when all math warps are done with it.
// The producer runs up to STAGES k-blocks ahead across tile and segment boundaries, so the
// next tile's first loads overlap the current tile's last k-blocks.  Every wait is bounded by
// a global-timer budget; a timeout raises GFIP_STATUS_WAIT_TIMEOUT (the result is then
// invalid), every role stops, and the producer waits for its copies in flight before exiting.
#pragma once

#include "gfip_kernels.cuh"

namespace gfip {
namespace ws {

// Math micro-tile: NCM 16-byte chunks (4 floats each) along m by 2 along n per thread.  With
// NCM = 4 (16 x 8) a 128 x 128 tile takes 4 math warps; two CTAs of 4 + 1 warps fit an SM
// with up to 168 registers a thread, which the 128 accumulators need.  (8 x 8 on 8 math warps
// would leave 96 registers a thread at two CTAs per SM, and spill.)  Every micro-tile shape
// gives the same bits: each C element is one FMA chain in k order.
#ifndef GFIP_WS_NCM
#define GFIP_WS_NCM 4
#endif
#ifndef GFIP_WS_UNROLL
#define GFIP_WS_UNROLL 8
#endif
struct Cfg {
    static constexpr int BM = 128, BN = 128, BK = 32, NCM = GFIP_WS_NCM, NCN = 2;
    static constexpr int THREADS = BM * BN / (NCM * 4 * NCN * 4);
    static constexpr int UNROLL = GFIP_WS_UNROLL;
    static constexpr int STAGES = 3, MIN_BLOCKS = 2;
};
static_assert(Cfg::BM == TileCfg<float>::BM && Cfg::BN == TileCfg<float>::BN &&
                  Cfg::BK == TileCfg<float>::BK,
              "the packed tiles are shared with the other FP32 kernels");

constexpr int MATH_THREADS = Cfg::THREADS;
constexpr int MATH_WARPS = MATH_THREADS / 32;
constexpr int THREADS = MATH_THREADS + 32;
constexpr int STAGES = Cfg::STAGES;
constexpr unsigned int STATUS_WAIT_TIMEOUT = 0x8u;       // mirrors GFIP_STATUS_WAIT_TIMEOUT
constexpr unsigned long long WAIT_BUDGET_NS = 2000000000ull;
constexpr long long WAIT_POLLS = 1ll << 40;              // the time budget ends every wait

using Lay = TileLayout<float, 128, 32>;   // A and B tiles share one layout
constexpr int TILE_BYTES = 128 * 32 * 4;  // one packed operand tile (16 KB)

struct Smem {
    float a[STAGES][Lay::ELEMS];
    float b[STAGES][Lay::ELEMS];
    unsigned long long full[STAGES];
    unsigned long long empty[STAGES];
    int flag;    // split-tile fix-up: this CTA adds the partial sums
    int abort;   // a wait gave up: every role stops
};

__device__ __forceinline__ bool aborted(const Smem &sm)
{
    return *(volatile const int *)&sm.abort != 0;
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// Arrives on the barrier once every cp.async this thread issued so far has landed; the
// arrival is one of the barrier's expected arrivals (.noinc).
__device__ __forceinline__ void cp_async_arrive(unsigned long long *bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
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

// Waits for the phase of the given parity; gives up after the budget or when another role
// has aborted.  A timeout sets the abort flag and the status bit.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity, Smem &sm,
                                          unsigned int *status)
{
    const uint32_t a = smem_addr(bar);
    if (mbar_try(a, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (long long it = 0; it < WAIT_POLLS; ++it) {
        if (mbar_try(a, parity)) return true;
        if (aborted(sm)) return false;
        if ((it & 63) == 63 && global_ns() - t0 > WAIT_BUDGET_NS) break;
    }
    *(volatile int *)&sm.abort = 1;
    atomicOr(status, STATUS_WAIT_TIMEOUT);
    return false;
}

// The same wait while draining after an abort: ignores the flag, raises nothing.
__device__ __forceinline__ void mbar_wait_drain(unsigned long long *bar, uint32_t parity)
{
    const uint32_t a = smem_addr(bar);
    const unsigned long long t0 = global_ns();
    for (long long it = 0; it < WAIT_POLLS; ++it) {
        if (mbar_try(a, parity)) return;
        if ((it & 63) == 63 && global_ns() - t0 > WAIT_BUDGET_NS) return;
    }
}

// 128-byte bulk copy global -> shared (copy engine), completing on an mbarrier.
__device__ __forceinline__ void bulk_load_row(uint32_t dst, const void *src,
                                              unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], 128, [%2];"
        ::"r"(dst), "l"(src), "r"(smem_addr(bar))
        : "memory");
}

// 128-byte bulk copy shared -> global, tracked in this thread's bulk async-groups.
__device__ __forceinline__ void bulk_store_row(void *dst, uint32_t src)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], 128;" ::"l"(dst),
                 "r"(src)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit()
{
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Waits until at most N of this thread's most recent bulk groups are pending.
template <int N> __device__ __forceinline__ void bulk_wait()
{
    asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}

// Orders this thread's generic-proxy accesses with its later (or earlier) async-proxy
// (bulk copy) accesses of global memory.
__device__ __forceinline__ void fence_proxy_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_shared()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void math_barrier()
{
    asm volatile("bar.sync 1, %0;" ::"n"(MATH_THREADS) : "memory");
}

// The segments one CTA runs, in order: whole tiles of the data-parallel waves, then its share
// of the k-split tiles.  Both roles walk the same sequence with their own cursor.
struct Segment {
    int t, i, j, kb0, kb1;
    int slot;   // which of the CTA's two partial-sum slots a split segment uses
};

struct SegCursor {
    int t;              // next data-parallel tile
    int64_t q, hi;      // next and end split iteration
    int first_u;

    __device__ __forceinline__ void start(const GemmParams<float> &p)
    {
        const int g = blockIdx.x;
        t = g;
        q = p.sk_iters * g / p.grid;
        hi = p.sk_iters * (g + 1) / p.grid;
        first_u = static_cast<int>(q / (p.kt > 0 ? p.kt : 1));
    }

    __device__ __forceinline__ bool next(const GemmParams<float> &p, Segment &s)
    {
        if (t < p.dp_tiles) {
            s.t = t;
            tile_of(p, t, s.i, s.j);
            s.kb0 = 0;
            s.kb1 = p.kt;
            s.slot = 0;
            t += p.grid;
            return true;
        }
        if (p.sk_iters <= 0 || q >= hi) return false;
        const int u = static_cast<int>(q / p.kt);
        s.t = p.dp_tiles + u;
        tile_of(p, s.t, s.i, s.j);
        s.kb0 = static_cast<int>(q % p.kt);
        const int64_t rest = hi - q;
        s.kb1 = (rest < (int64_t)(p.kt - s.kb0)) ? s.kb0 + static_cast<int>(rest) : p.kt;
        s.slot = (u == first_u) ? 0 : 1;
        q += s.kb1 - s.kb0;
        return true;
    }
};

// Element copies of one raw 128 x 32 operand tile by the 32 producer lanes; element (x, kk)
// of the tile at (x0, k0) of op(X) sits at g[(x0+x) + (k0+kk)*ld] (CONTIG) or
// g[(k0+kk) + (x0+x)*ld].  Out-of-range elements are zero-filled (Sec. 2.2).
//   CONTIG: lane covers x = lane + 32 q: a copy instruction reads 128 contiguous bytes and
//           writes 32 consecutive words of one shared-memory row (conflict free).
//   else:   lane covers kk = lane % 8 + 8 r, x = lane / 8 + 4 q: four 32-byte runs along k,
//           written to 32 distinct banks thanks to the padded row pitch.
template <bool CONTIG>
__device__ __forceinline__ void raw_tile(uint32_t sdst, const float *g, int64_t ld, int x0,
                                         int k0, int x_ext, int kleft, int lane)
{
    const bool whole = (x0 + 128 <= x_ext) && (kleft >= 32);
    if (CONTIG) {
        const float *src = g + (int64_t)(x0 + lane) + (int64_t)k0 * ld;
        uint32_t d = sdst + lane * 4;
        uint32_t xok = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (x0 + lane + 32 * q < x_ext) xok |= 1u << q;
#pragma unroll 4
        for (int kk = 0; kk < 32; ++kk) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const bool ok = whole || (((xok >> q) & 1u) && kk < kleft);
                cp_async_elem<4>(d + q * Lay::SEG * 4, ok ? src + 32 * q : g, ok);
            }
            src += ld;
            d += Lay::P * 4;
        }
    } else {
        const int kl = lane & 7, xl = lane >> 3;
        const float *src = g + (int64_t)(k0 + kl) + (int64_t)(x0 + xl) * ld;
        const int64_t step = 4 * ld;
#pragma unroll 4
        for (int q = 0; q < 32; ++q) {
            const int x = xl + 4 * q;
            const uint32_t d = sdst + ((x >> 5) * Lay::SEG + (x & 31) + kl * Lay::P) * 4;
            const bool xin = x0 + x < x_ext;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const bool ok = whole || (xin && kl + 8 * r < kleft);
                cp_async_elem<4>(d + 8 * r * Lay::P * 4, ok ? src + 8 * r : g, ok);
            }
            src += step;
        }
    }
}

// Bulk copies of one packed tile (128 rows of 128 bytes) into the padded stage layout; lane
// takes rows lane + 32 q, i.e. 128-byte segment q, k row `lane`.
__device__ __forceinline__ void packed_tile(uint32_t sdst, const float *tile, int lane,
                                            unsigned long long *bar)
{
#pragma unroll
    for (int q = 0; q < 4; ++q)
        bulk_load_row(sdst + (q * Lay::SEG + lane * Lay::P) * 4, tile + (q * 32 + lane) * 32, bar);
}

// Bulk stores of a staged tile into its packed slot (the fused pack store).
__device__ __forceinline__ void store_tile(float *tile, uint32_t ssrc, int lane)
{
#pragma unroll
    for (int q = 0; q < 4; ++q)
        bulk_store_row(tile + (q * 32 + lane) * 32, ssrc + (q * Lay::SEG + lane * Lay::P) * 4);
}

template <bool ACONTIG, bool BCONTIG> struct WsKernel {
    using K = Kernel<float, ACONTIG, BCONTIG, Cfg>;   // micro-tile, epilogue, split fix-up math
    static constexpr int TM = K::TM, TN = K::TN, TX = K::TX, NCM = K::NCM;

    // What the producer did with one stage: which operand tiles it must pack and publish.
    struct Meta {
        int prod;      // bit 0: pack A, bit 1: pack B
        int i, j, kb;
        int last;      // bit 0 (1): kb ends a whole A (B) panel this CTA produced
    };

    static __device__ __forceinline__ float *pack_slot_a(const GemmParams<float> &p, int i, int kb)
    {
        return p.pack_a + ((int64_t)i * p.kt + kb) * (128 * 32);
    }
    static __device__ __forceinline__ float *pack_slot_b(const GemmParams<float> &p, int j, int kb)
    {
        return p.pack_b + ((int64_t)j * p.kt + kb) * (128 * 32);
    }

    // Publishes the packed tiles of one stage (lane 0, after every lane's bulk stores of it
    // have completed and each lane has fenced the async proxy): ready words per k-block, and
    // the panel words when a whole panel is done.
    static __device__ __forceinline__ void publish_meta(const GemmParams<float> &p, const Meta &m,
                                                        unsigned int epoch)
    {
        if (!m.prod) return;
        if (m.prod & 1) publish(p.state_a + (int64_t)m.i * p.kt + m.kb, epoch);
        if (m.prod & 2) publish(p.state_b + (int64_t)m.j * p.kt + m.kb, epoch);
        if (m.last & 1) publish(p.state_a + (int64_t)p.mt * p.kt + m.i, epoch);
        if (m.last & 2) publish(p.state_b + (int64_t)p.nt * p.kt + m.j, epoch);
    }

    static __device__ void producer(const GemmParams<float> &p, Smem &sm)
    {
        const int lane = threadIdx.x & 31;
        unsigned int epoch = 0u;
        if (lane == 0) epoch = *(volatile unsigned int *)p.launch_count + 1u;
        epoch = __shfl_sync(0xffffffffu, epoch, 0);
        const unsigned long long ready = ready_value(epoch);
        Meta meta[STAGES];
        long long q = 0;          // k-blocks filled so far (stage q % STAGES)
        bool ok = true;

        // the stage of k-block `d` has arrived: write its packed tiles (bulk stores)
        auto store_stage = [&](long long d) {
            const Meta &m = meta[d % STAGES];
            if (m.prod) {
                const int st = static_cast<int>(d % STAGES);
                if (!mbar_wait(&sm.full[st], static_cast<uint32_t>((d / STAGES) & 1), sm,
                               p.status)) {
                    ok = false;
                    return;
                }
                fence_proxy_shared();
                if (m.prod & 1) store_tile(pack_slot_a(p, m.i, m.kb), smem_addr(sm.a[st]), lane);
                if (m.prod & 2) store_tile(pack_slot_b(p, m.j, m.kb), smem_addr(sm.b[st]), lane);
            }
            bulk_commit();   // one group per k-block (empty when nothing is packed)
        };

        SegCursor cur;
        cur.start(p);
        Segment sg;
        while (ok && !aborted(sm) && cur.next(p, sg)) {
            const int i = sg.i, j = sg.j, kb0 = sg.kb0, kb1 = sg.kb1;
            const bool prod_a = p.mode_a == MODE_FIP && j == 0 && p.a_produces;
            const bool prod_b = p.mode_b == MODE_FIP && i == 0 && p.b_produces;
            // a panel its producer finished whole needs no per-k-block look-ups
            bool full_a = false, full_b = false;
            if (lane == 0) {
                full_a = p.mode_a == MODE_FIP && !prod_a &&
                         ld_relaxed(p.state_a + (int64_t)p.mt * p.kt + i) == ready;
                full_b = p.mode_b == MODE_FIP && !prod_b &&
                         ld_relaxed(p.state_b + (int64_t)p.nt * p.kt + j) == ready;
            }
            full_a = __shfl_sync(0xffffffffu, full_a, 0);
            full_b = __shfl_sync(0xffffffffu, full_b, 0);
            if (full_a || full_b) {
                fence_acquire();
                fence_proxy_global();
            }
            for (int kb = kb0; kb < kb1; ++kb) {
                const int st = static_cast<int>(q % STAGES);
                if (q >= STAGES) {
                    // the stage's previous k-block is done: math released it, and its pack
                    // stores (issued a k-block after it arrived) have been read; publish them
                    if (!mbar_wait(&sm.empty[st], static_cast<uint32_t>(((q / STAGES) - 1) & 1),
                                   sm, p.status)) {
                        ok = false;
                        break;
                    }
                }
                // decisions (Sec. 3.2's four cases, per operand)
                int da = 0, db = 0;   // 0 raw, 1 packed, 2 produce
                if (lane == 0) {
                    da = (p.mode_a == MODE_PACKED) ? 1 : 0;
                    db = (p.mode_b == MODE_PACKED) ? 1 : 0;
                    bool acq = false;
                    if (p.mode_a == MODE_FIP) {
                        if (prod_a) da = 2;
                        else if (full_a) da = 1;
                        else if (ld_relaxed(p.state_a + (int64_t)i * p.kt + kb) == ready) {
                            da = 1;
                            acq = true;
                        }
                    }
                    if (p.mode_b == MODE_FIP) {
                        if (prod_b) db = 2;
                        else if (full_b) db = 1;
                        else if (ld_relaxed(p.state_b + (int64_t)j * p.kt + kb) == ready) {
                            db = 1;
                            acq = true;
                        }
                    }
                    if (acq) {
                        fence_acquire();
                        fence_proxy_global();
                    }
                    // copy-engine bytes this stage waits for, with this lane's arrival
                    mbar_arrive_expect_tx(&sm.full[st], (da == 1 ? TILE_BYTES : 0) +
                                                            (db == 1 ? TILE_BYTES : 0));
                }
                da = __shfl_sync(0xffffffffu, da, 0);
                db = __shfl_sync(0xffffffffu, db, 0);
                const int kleft = p.k - kb * 32;
                const uint32_t sa = smem_addr(sm.a[st]), sb = smem_addr(sm.b[st]);
                if (da == 1)
                    packed_tile(sa, pack_slot_a(p, i, kb), lane, &sm.full[st]);
                else
                    raw_tile<ACONTIG>(sa, p.A, p.lda, i * 128, kb * 32, p.m, kleft, lane);
                if (db == 1)
                    packed_tile(sb, pack_slot_b(p, j, kb), lane, &sm.full[st]);
                else
                    raw_tile<BCONTIG>(sb, p.B, p.ldb, j * 128, kb * 32, p.n, kleft, lane);
                cp_async_arrive(&sm.full[st]);
                Meta &m = meta[st];
                m.prod = (da == 2 ? 1 : 0) | (db == 2 ? 2 : 0);
                m.i = i;
                m.j = j;
                m.kb = kb;
                m.last = (kb == kb1 - 1 && kb0 == 0 && kb1 == p.kt) ? m.prod : 0;
                // the previous k-block has had a k-block's time to arrive: pack it now; then
                // every group but the newest has completed, so the k-block before it (whose
                // stage is the next to be refilled) is published
                if (q >= 1) {
                    store_stage(q - 1);
                    if (!ok) break;
                    bulk_wait<1>();
                    fence_proxy_global();
                    __syncwarp();
                    if (q >= 2 && lane == 0) publish_meta(p, meta[(q - 2) % STAGES], epoch);
                }
                ++q;
            }
        }
        // the last k-block's pack stores, then everything published
        if (ok && q >= 1 && !aborted(sm)) store_stage(q - 1);
        bulk_wait<0>();
        fence_proxy_global();
        __syncwarp();
        if (ok && !aborted(sm) && lane == 0) {
            if (q >= 2) publish_meta(p, meta[(q - 2) % STAGES], epoch);
            if (q >= 1) publish_meta(p, meta[(q - 1) % STAGES], epoch);
        }
        if (aborted(sm)) {
            // nothing may still write shared memory when the CTA exits
            asm volatile("cp.async.wait_all;" ::: "memory");
            for (long long d = q - 1; d >= 0 && d >= q - STAGES; --d)
                mbar_wait_drain(&sm.full[d % STAGES], static_cast<uint32_t>((d / STAGES) & 1));
        }
    }

    // C[tile] := alpha*acc + beta*C[tile] (C not read when beta == 0), the operations of the
    // shared tile core's epilogue, taking C four rows (one 16-byte chunk) at a time so that
    // few registers are live beside the 128 accumulators.
    static __device__ void epilogue(const GemmParams<float> &p, int i, int j,
                                    const float (&acc)[TM][TN])
    {
        constexpr int CH = 4;
        const int tid = threadIdx.x;
        const int tx = tid % TX, ty = tid / TX;
        const bool read_c = (p.beta != 0.f);
#pragma unroll
        for (int jj = 0; jj < TN; ++jj) {
            const int col = j * 128 + ty * CH + (jj % CH) + (jj / CH) * (128 / K::NCN);
            if (col >= p.n) continue;
            float *ccol = p.C + (int64_t)col * p.ldc;
#pragma unroll
            for (int c = 0; c < TM / CH; ++c) {
                const int row0 = i * 128 + tx * CH + c * (128 / NCM);
                float cv[CH];
#pragma unroll
                for (int r = 0; r < CH; ++r)
                    cv[r] = (read_c && row0 + r < p.m) ? ccol[row0 + r] : 0.f;
#pragma unroll
                for (int r = 0; r < CH; ++r) {
                    if (row0 + r >= p.m) continue;
                    float v = p.alpha * acc[c * CH + r][jj];
                    if (read_c) v = fmaf(p.beta, cv[r], v);
                    ccol[row0 + r] = v;
                }
            }
        }
    }

    // Split-tile fix-up (as in the shared tile core, with the math warps' named barrier).
    static __device__ void fixup(const GemmParams<float> &p, Smem &sm, int t, int i, int j,
                                 int slot, float (&acc)[TM][TN], unsigned int epoch)
    {
        const int tid = threadIdx.x;
        const int g = blockIdx.x;
        const int64_t S = p.sk_iters;
        const int G = p.grid;
        const int u = t - p.dp_tiles;
        const int g0 = K::cta_of((int64_t)u * p.kt, S, G);
        const int g1 = K::cta_of((int64_t)(u + 1) * p.kt - 1, S, G);
        const int nseg = g1 - g0 + 1;
        float *mine = p.partial + (int64_t)(2 * g + slot) * (128 * 128);
#pragma unroll
        for (int ii = 0; ii < TM; ++ii)
#pragma unroll
            for (int jj = 0; jj < TN; ++jj)
                __stcg(mine + (ii * TN + jj) * MATH_THREADS + tid, acc[ii][jj]);
        math_barrier();
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
        math_barrier();
        if (sm.flag) {
            // the segments' partial sums added in k order, CHK values at a time (the
            // accumulators already hold all the registers a thread can spare)
            constexpr int NV = TM * TN, CHK = 16;
            float *flat = &acc[0][0];
#pragma unroll
            for (int c0 = 0; c0 < NV; c0 += CHK) {
                for (int gs = g0; gs <= g1; ++gs) {
                    const int64_t lo = S * gs / G;
                    const int gslot = (lo / p.kt == u) ? 0 : 1;
                    const float *src = p.partial + (int64_t)(2 * gs + gslot) * (128 * 128);
                    float v[CHK];
#pragma unroll
                    for (int e = 0; e < CHK; ++e)
                        v[e] = __ldcg(src + (c0 + e) * MATH_THREADS + tid);
#pragma unroll
                    for (int e = 0; e < CHK; ++e)
                        flat[c0 + e] = (gs == g0) ? v[e] : flat[c0 + e] + v[e];
                }
            }
            epilogue(p, i, j, acc);
        }
        math_barrier();
    }

    static __device__ void math(const GemmParams<float> &p, Smem &sm)
    {
        const int tid = threadIdx.x;
        const int tx = tid % TX, ty = tid / TX;
        unsigned int epoch = 0u;
        if (tid == 0) epoch = *(volatile unsigned int *)p.launch_count + 1u;
        float acc[TM][TN];
        int st = 0;          // stage of the next k-block
        uint32_t ph = 0;     // parity of that stage's next full phase
        SegCursor cur;
        cur.start(p);
        Segment sg;
        bool ok = true;
        while (ok && cur.next(p, sg)) {
            const int i = sg.i, j = sg.j, kb0 = sg.kb0, kb1 = sg.kb1;
#pragma unroll
            for (int ii = 0; ii < TM; ++ii)
#pragma unroll
                for (int jj = 0; jj < TN; ++jj) acc[ii][jj] = 0.f;
            // the segment that ends the tile's k loop will read C: warm L2 with it now
            if (kb1 == p.kt && p.beta != 0.f) {
                constexpr int PER_COL = 128 / 32;
                for (int e = tid; e < 128 * PER_COL; e += MATH_THREADS) {
                    const int col = j * 128 + e / PER_COL, row = i * 128 + (e % PER_COL) * 32;
                    if (col < p.n && row < p.m)
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(p.C + row +
                                                                       (int64_t)col * p.ldc));
                }
            }
            for (int kb = kb0; kb < kb1; ++kb) {
                if (!mbar_wait(&sm.full[st], ph, sm, p.status)) {
                    ok = false;
                    break;
                }
                K::template compute<NCM>(sm.a[st], sm.b[st], acc, tx, ty, 32);
                __syncwarp();
                if ((tid & 31) == 0) mbar_arrive(&sm.empty[st]);
                if (++st == STAGES) {
                    st = 0;
                    ph ^= 1u;
                }
            }
            if (!ok) break;
            if (kb0 == 0 && kb1 == p.kt)
                epilogue(p, i, j, acc);
            else
                fixup(p, sm, sg.t, i, j, sg.slot, acc, epoch);
        }
    }
};

// The launch's epoch tags its ready words and arrival counters exactly as in gemm_kernel:
// every role reads the launch counter at start, and the last CTA to finish advances it.
template <bool ACONTIG, bool BCONTIG>
__global__ void __launch_bounds__(THREADS, 2) ws_gemm_kernel(const GemmParams<float> p)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&sm.full[s], 33);             // 32 lanes' copy arrivals + expect_tx
            mbar_init(&sm.empty[s], MATH_WARPS);
        }
        sm.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (warp == MATH_WARPS)
        WsKernel<ACONTIG, BCONTIG>::producer(p, sm);
    else
        WsKernel<ACONTIG, BCONTIG>::math(p, sm);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(p.done_count, 1u) == gridDim.x - 1) {
            const unsigned int epoch = *(volatile unsigned int *)p.launch_count + 1u;
            *(volatile unsigned int *)p.done_count = 0u;
            *(volatile unsigned int *)p.launch_count = epoch;
            __threadfence();
        }
    }
}

inline size_t smem_bytes()
{
    return sizeof(Smem);
}

template <bool AC, bool BC> cudaError_t configure()
{
    static bool configured = false;
    if (configured) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(ws_gemm_kernel<AC, BC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem_bytes()));
    if (e == cudaSuccess) configured = true;
    return e;
}

template <bool AC, bool BC> cudaError_t launch_t(const GemmParams<float> &p, cudaStream_t s)
{
    cudaError_t e = configure<AC, BC>();
    if (e != cudaSuccess) return e;
    ws_gemm_kernel<AC, BC><<<p.grid, THREADS, smem_bytes(), s>>>(p);
    return cudaGetLastError();
}

template <bool AC, bool BC> int blocks_per_sm_one()
{
    if (configure<AC, BC>() != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, ws_gemm_kernel<AC, BC>, THREADS,
                                                      smem_bytes()) != cudaSuccess)
        return 0;
    return n;
}

}  // namespace ws
}  // namespace gfip
