// gfip_ws.cuh -- warp-specialised FP32 tile core of the fused-in-packing GEMM.
//
// The FP32 GEMM is bound by the FFMA pipe.  When every thread of a CTA both loads operand
// tiles and computes (the tile core of gfip_kernels.cuh), the element-wise raw loads of the
// first pass, the ready-word look-ups with their acquire fences, and the barrier after every
// k-block all sit in the instruction stream of the FFMA warps: the math pipe idles while the
// warps of a CTA load and synchronise together, and a tile that reads the raw strided operand
// costs the FFMA loop about 10 % more than one that reads a packed copy.  Here the roles are
// split (Sec. 3.2's fused microkernel, with the "load and pack" half given warps of its own):
//
//   warps 0-3  math: wait until a stage is full, run the FFMA2 loop over its 32 k rows,
//              release the stage; accumulators, alpha/beta epilogue and the split-tile fix-up
//              (each C element is one FMA chain in k order, as in the shared tile core, so
//              every variant and both tile cores give the same bits)
//   warp 4     producer of op(A) tiles, warp 5 producer of op(B) tiles: per k-block each
//              decides raw / packed / produce for its operand (the ready-word look-ups and
//              acquire fences happen here), fills its half of the stage with element copies of
//              the raw strided operand or ONE 16 KB bulk copy of the packed tile (the copy
//              engine), and for a producer tile (Alg. 1: the first tile column packs A, the
//              first tile row packs B) writes the staged tile to the packed buffer with one
//              bulk store once it has arrived, then publishes it
//
// Stage layout (and packed layout): a 128 x 32 operand tile is four 128-byte-wide segments
// of x (m for A, n for B), each 32 rows (one per k) of 32 floats, rows 128 bytes apart with no
// padding; the 16-byte chunk c of row kk is stored at chunk position c ^ (kk % 8).  The XOR
// swizzle keeps both the raw copies (a warp writes 8 rows x 4 x, or 32 x of one row) and the
// math warps' 16-byte fragment reads free of bank conflicts, and makes the packed tile in HBM
// the exact 16 KB shared-memory image, moved by one bulk copy each way.
//
// A stage is handed over on mbarriers: `full` completes when both producers' 32 lanes have
// seen their element copies land (cp.async.mbarrier.arrive.noinc) and the bulk copies' bytes
// have arrived (expect_tx); `empty` completes when all math warps are done with it.  The
// producers run up to STAGES k-blocks ahead across tile and segment boundaries, so the next
// tile's first loads overlap the current tile's last k-blocks.  Every wait is bounded by a
// global-timer budget; a timeout raises GFIP_STATUS_WAIT_TIMEOUT (the result is then
// invalid), every role stops, and each producer waits for its copies in flight before exiting.
#pragma once

#include "gfip_kernels.cuh"

namespace gfip {
namespace ws {

// Math micro-tile: 16 x 8 per thread (4 chunks of 4 floats along m, 2 along n), so a
// 128 x 128 tile takes one warpgroup of 4 math warps.  A CTA holds one SM: two math
// warpgroups, each running the tiles of one "virtual CTA" of the shared schedule (ids
// 2 * block and 2 * block + 1, so the grid, the split points and the bits are those of the
// other FP32 kernels at two CTAs per SM), and one producer warpgroup (op(A) and op(B)
// producers of each math warpgroup).  Registers: launched at 168 a thread (384 x 168 = 64512),
// the producers drop to 56 and the math warpgroups rise to 224 (128 x 56 + 256 x 224 =
// 64512), room for 128 accumulators and double-buffered fragments.
struct Cfg {
    static constexpr int BM = 128, BN = 128, BK = 32, NCM = 4, NCN = 2;
    static constexpr int THREADS = BM * BN / (NCM * 4 * NCN * 4);
    static constexpr int UNROLL = 8;
    static constexpr int STAGES = 3, MIN_BLOCKS = 1;
};
static_assert(Cfg::BM == TileCfg<float>::BM && Cfg::BN == TileCfg<float>::BN &&
                  Cfg::BK == TileCfg<float>::BK,
              "the tile grid and its schedule are shared with the other FP32 kernels");

constexpr int MATH_THREADS = Cfg::THREADS;     // 128: one warpgroup per virtual CTA
constexpr int MATH_WARPS = MATH_THREADS / 32;  // 4
constexpr int VCTA = 2;                        // virtual CTAs (math warpgroups) per CTA
constexpr int THREADS = (VCTA + 1) * 128;      // + the producer warpgroup
constexpr int LAUNCH_REGS = 168, PRODUCER_REGS = 56, MATH_REGS = 224;
static_assert(128 * PRODUCER_REGS + VCTA * 128 * MATH_REGS == THREADS * LAUNCH_REGS,
              "the register split must add up to the launch's registers exactly");
constexpr int STAGES = Cfg::STAGES;
constexpr int TILE_FLOATS = 128 * 32;
constexpr int TILE_BYTES = TILE_FLOATS * 4;    // one operand tile, packed or staged (16 KB)
constexpr unsigned int STATUS_WAIT_TIMEOUT = 0x8u;       // mirrors GFIP_STATUS_WAIT_TIMEOUT
constexpr unsigned long long WAIT_BUDGET_NS = 2000000000ull;
constexpr long long WAIT_POLLS = 1ll << 40;              // the time budget ends every wait

// Float offset of element (x, kk) of a tile in the swizzled layout.
__host__ __device__ constexpr int swz(int x, int kk)
{
    return (x >> 5) * 1024 + kk * 32 + ((((x & 31) >> 2) ^ (kk & 7)) << 2) + (x & 3);
}

// The stage ring of one math warpgroup.
struct __align__(128) Ring {
    float a[STAGES][TILE_FLOATS];
    float b[STAGES][TILE_FLOATS];
    unsigned long long full[STAGES];
    unsigned long long empty[STAGES];
    int flag;    // split-tile fix-up: this virtual CTA adds the partial sums
};

struct __align__(128) Smem {
    Ring ring[VCTA];
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

// Bulk copy global -> shared (copy engine), completing on an mbarrier.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes,
                                          unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Bulk copy shared -> global, tracked in this thread's bulk async-groups.
__device__ __forceinline__ void bulk_store(void *dst, uint32_t src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                 "r"(src), "r"(bytes)
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

// Orders this thread's generic-proxy accesses with its async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_shared()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Named barrier of one math warpgroup (ids 1 and 2; 0 is __syncthreads).
__device__ __forceinline__ void math_barrier(int ring)
{
    asm volatile("bar.sync %0, %1;" ::"r"(1 + ring), "n"(MATH_THREADS) : "memory");
}

// The segments one (virtual) CTA g runs, in order: whole tiles of the data-parallel waves,
// then its share of the k-split tiles.  Every role walks the same sequence with its own cursor.
struct Segment {
    int t, i, j, kb0, kb1;
    int slot;   // which of the CTA's two partial-sum slots a split segment uses
};

struct SegCursor {
    int t;              // next data-parallel tile
    int64_t q, hi;      // next and end split iteration
    int first_u;

    __device__ __forceinline__ void start(const GemmParams<float> &p, int g)
    {
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

// Element copies of one raw 128 x 32 operand tile by 32 lanes into the swizzled layout;
// element (x, kk) of the tile at (x0, k0) of op(X) sits at g[(x0+x) + (k0+kk)*ld] (CONTIG) or
// g[(k0+kk) + (x0+x)*ld].  Out-of-range elements are zero-filled (Sec. 2.2).
//   CONTIG: lane covers x = lane + 32 q: one copy instruction reads 128 contiguous bytes of
//           a column and writes 32 distinct banks of one row.
//   else:   lane covers kk = lane % 8 + 8 r, x = lane / 8 + 4 q: four 32-byte runs along k,
//           written to 8 rows whose swizzled chunks fall in distinct banks.
// A tile that lies wholly inside the operand takes the copies without per-element checks.
template <bool CONTIG>
__device__ __forceinline__ void raw_tile(uint32_t sdst, const float *g, int64_t ld, int x0,
                                         int k0, int x_ext, int kleft, int lane)
{
    const bool whole = (x0 + 128 <= x_ext) && (kleft >= 32);
    if (CONTIG) {
        const float *src = g + (int64_t)(x0 + lane) + (int64_t)k0 * ld;
        // row kk: chunk lane/4 goes to chunk (lane/4) ^ (kk % 8); bytes within it lane % 4
        const uint32_t rowbase = sdst + (lane & 3) * 4;
        if (whole) {
#pragma unroll 8
            for (int kk = 0; kk < 32; ++kk) {
                const uint32_t d = rowbase + kk * 128 + ((((lane >> 2) ^ (kk & 7))) << 4);
#pragma unroll
                for (int q = 0; q < 4; ++q) cp_async_elem<4>(d + q * 4096, src + 32 * q, true);
                src += ld;
            }
        } else {
            uint32_t xok = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (x0 + lane + 32 * q < x_ext) xok |= 1u << q;
#pragma unroll 4
            for (int kk = 0; kk < 32; ++kk) {
                const uint32_t d = rowbase + kk * 128 + ((((lane >> 2) ^ (kk & 7))) << 4);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const bool ok = ((xok >> q) & 1u) && kk < kleft;
                    cp_async_elem<4>(d + q * 4096, ok ? src + 32 * q : g, ok);
                }
                src += ld;
            }
        }
    } else {
        const int kl = lane & 7, xl = lane >> 3;
        const float *src = g + (int64_t)(k0 + kl) + (int64_t)(x0 + xl) * ld;
        const int64_t step = 4 * ld;
        // element (xl + 4 q, kl + 8 r): segment q / 8, row kl + 8 r, chunk (q % 8) ^ kl, word xl
        const uint32_t base = sdst + (kl * 32 + xl) * 4;
        if (whole) {
#pragma unroll 8
            for (int q = 0; q < 32; ++q) {
                const uint32_t d = base + (q >> 3) * 4096 + (((q & 7) ^ kl) << 4);
#pragma unroll
                for (int r = 0; r < 4; ++r) cp_async_elem<4>(d + r * 1024, src + 8 * r, true);
                src += step;
            }
        } else {
#pragma unroll 4
            for (int q = 0; q < 32; ++q) {
                const uint32_t d = base + (q >> 3) * 4096 + (((q & 7) ^ kl) << 4);
                const bool xin = x0 + xl + 4 * q < x_ext;
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const bool ok = xin && kl + 8 * r < kleft;
                    cp_async_elem<4>(d + r * 1024, ok ? src + 8 * r : g, ok);
                }
                src += step;
            }
        }
    }
}

template <bool ACONTIG, bool BCONTIG> struct WsKernel {
    using K = Kernel<float, ACONTIG, BCONTIG, Cfg>;   // FFMA2 micro-tile update, split bookkeeping
    static constexpr int TM = K::TM, TN = K::TN, TX = K::TX, NCM = K::NCM, NCN = K::NCN;
    static_assert(TM == 16 && TN == 8 && TX == 8, "fragment addressing assumes 16 x 8 on 8 x 16");

    // What a producer did with one stage of its operand.
    struct Meta {
        int prod;     // this stage's tile is to be packed and published
        int panel, kb;
        int last;     // kb ends a whole panel this CTA produced
    };

    // ---- producer warps ------------------------------------------------------------------
    // OPB: false = the op(A) producer, true = the op(B) producer of ring r (virtual CTA g).
    template <bool OPB>
    static __device__ void producer(const GemmParams<float> &p, Smem &sm, Ring &rg, int g)
    {
        constexpr bool CONTIG = OPB ? BCONTIG : ACONTIG;
        const int lane = threadIdx.x & 31;
        const int mode = OPB ? p.mode_b : p.mode_a;
        const float *X = OPB ? p.B : p.A;
        const int64_t ld = OPB ? p.ldb : p.lda;
        const int x_ext = OPB ? p.n : p.m;
        const int npanels = OPB ? p.nt : p.mt;
        unsigned long long *state = OPB ? p.state_b : p.state_a;
        float *pack = OPB ? p.pack_b : p.pack_a;
        const bool produces = OPB ? p.b_produces : p.a_produces;

        unsigned int epoch = 0u;
        if (lane == 0) epoch = *(volatile unsigned int *)p.launch_count + 1u;
        const unsigned long long ready = ready_value(epoch);   // meaningful in lane 0 only
        Meta meta[STAGES];
        long long q = 0;          // k-blocks filled so far (stage q % STAGES)
        bool ok = true;

        auto buf = [&](int st) -> uint32_t {
            return smem_addr(OPB ? rg.b[st] : rg.a[st]);
        };
        auto slot = [&](int panel, int kb) -> float * {
            return pack + ((int64_t)panel * p.kt + kb) * TILE_FLOATS;
        };
        // lane 0: once the stage of k-block d has arrived, write its packed tile (one bulk
        // store); one bulk group is committed per k-block, empty when nothing is packed
        auto store_stage = [&](long long d) {
            const Meta &m = meta[d % STAGES];
            const int st = static_cast<int>(d % STAGES);
            if (m.prod) {
                if (!mbar_wait(&rg.full[st], static_cast<uint32_t>((d / STAGES) & 1), sm,
                               p.status)) {
                    ok = false;
                    return;
                }
                fence_proxy_shared();
                bulk_store(slot(m.panel, m.kb), buf(st), TILE_BYTES);
            }
            bulk_commit();
        };
        // lane 0: the packed tile of a stage whose bulk store has completed becomes visible
        auto publish_meta = [&](const Meta &m) {
            if (!m.prod) return;
            publish(state + (int64_t)m.panel * p.kt + m.kb, epoch);
            if (m.last) publish(state + (int64_t)npanels * p.kt + m.panel, epoch);
        };

        SegCursor cur;
        cur.start(p, g);
        Segment sg;
        while (ok && !aborted(sm) && cur.next(p, sg)) {
            const int panel = OPB ? sg.j : sg.i;
            const int other = OPB ? sg.i : sg.j;
            // a panel that no later tile reuses is neither packed nor looked up (reused_a/_b)
            const int emode =
                (mode == MODE_FIP && !(OPB ? reused_b(p, panel) : reused_a(p, panel))) ? MODE_RAW
                                                                                        : mode;
            const bool prod = emode == MODE_FIP && other == 0 && produces;
            // a panel its producer finished whole needs no per-k-block look-ups
            bool full = false;
            if (lane == 0 && emode == MODE_FIP && !prod) {
                full = ld_relaxed(state + (int64_t)npanels * p.kt + panel) == ready;
                if (full) {
                    fence_acquire();
                    fence_proxy_global();
                }
            }
            for (int kb = sg.kb0; kb < sg.kb1; ++kb) {
                const int st = static_cast<int>(q % STAGES);
                if (q >= STAGES &&
                    !mbar_wait(&rg.empty[st], static_cast<uint32_t>(((q / STAGES) - 1) & 1), sm,
                               p.status)) {
                    ok = false;
                    break;
                }
                // decision (Sec. 3.2's cases, for this operand): 0 raw, 1 packed, 2 produce
                int d = 0;
                if (lane == 0) {
                    if (emode == MODE_PACKED) {
                        d = 1;
                    } else if (emode == MODE_FIP) {
                        if (prod) {
                            d = 2;
                        } else if (full) {
                            d = 1;
                        } else if (ld_relaxed(state + (int64_t)panel * p.kt + kb) == ready) {
                            d = 1;
                            fence_acquire();
                            fence_proxy_global();
                        }
                    }
                    // this lane's arrival, with the copy-engine bytes the stage waits for
                    mbar_arrive_expect_tx(&rg.full[st], d == 1 ? TILE_BYTES : 0);
                    if (d == 1) bulk_load(buf(st), slot(panel, kb), TILE_BYTES, &rg.full[st]);
                }
                d = __shfl_sync(0xffffffffu, d, 0);
                if (d != 1)
                    raw_tile<CONTIG>(buf(st), X, ld, panel * 128, kb * 32, x_ext, p.k - kb * 32,
                                     lane);
                cp_async_arrive(&rg.full[st]);
                Meta &m = meta[st];
                m.prod = (d == 2);
                m.panel = panel;
                m.kb = kb;
                m.last = (d == 2) && kb == sg.kb1 - 1 && sg.kb0 == 0 && sg.kb1 == p.kt;
                // the previous k-block has had a k-block's time to arrive: pack it now; then
                // every bulk group but the newest has completed, so the k-block before it
                // (whose stage is the next to be refilled) is published
                if (q >= 1 && lane == 0) {
                    store_stage(q - 1);
                    if (ok) {
                        bulk_wait<1>();
                        fence_proxy_global();
                        if (q >= 2) publish_meta(meta[(q - 2) % STAGES]);
                    }
                }
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) break;
                ++q;
            }
        }
        if (lane == 0) {
            if (ok && q >= 1 && !aborted(sm)) store_stage(q - 1);
            bulk_wait<0>();
            fence_proxy_global();
            if (ok && !aborted(sm)) {
                if (q >= 2) publish_meta(meta[(q - 2) % STAGES]);
                if (q >= 1) publish_meta(meta[(q - 1) % STAGES]);
            }
        }
        __syncwarp();
        if (aborted(sm)) {
            // nothing may still write shared memory when the CTA exits
            asm volatile("cp.async.wait_all;" ::: "memory");
            if (lane == 0)
                for (long long d = q - 1; d >= 0 && d >= q - STAGES; --d)
                    mbar_wait_drain(&rg.full[d % STAGES], static_cast<uint32_t>((d / STAGES) & 1));
        }
    }

    // ---- math warps ------------------------------------------------------------------------
    // Fragments of one k row.  Thread (tx, ty): A chunks c = 0..3 in segment c at chunk
    // position tx; B chunks c = 0..1 in segment ty / 8 + 2 c at chunk position ty % 8.  In row
    // kk the chunk position is XORed with kk % 8, which only touches address bits 4-6 (rows
    // are 128 bytes, segments 4 KB): the row's byte offset is (base ^ (U << 4)) + U * 128 for
    // row U of an 8-row group whose row 0 sits at base.
    template <int U>
    static __device__ __forceinline__ void load_row(const char *sa, const char *sb, uint32_t oa,
                                                    uint32_t ob, float (&a)[TM], float (&b)[TN])
    {
        const char *pa = sa + ((oa ^ (U << 4)) + U * 128);
        const char *pb = sb + ((ob ^ (U << 4)) + U * 128);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float4 v = *reinterpret_cast<const float4 *>(pa + c * 4096);
            a[4 * c + 0] = v.x;
            a[4 * c + 1] = v.y;
            a[4 * c + 2] = v.z;
            a[4 * c + 3] = v.w;
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const float4 v = *reinterpret_cast<const float4 *>(pb + c * 8192);
            b[4 * c + 0] = v.x;
            b[4 * c + 1] = v.y;
            b[4 * c + 2] = v.z;
            b[4 * c + 3] = v.w;
        }
    }

    // Row U of an 8-row group: the fragments of the next row are loaded first (double
    // buffering), then row U's FFMA2 block.
    template <int U>
    static __device__ __forceinline__ void step(const char *sa, const char *sb, uint32_t oa,
                                                uint32_t ob, bool more, float (&a)[2][TM],
                                                float (&b)[2][TN], float (&acc)[TM][TN])
    {
        if constexpr (U < 7)
            load_row<U + 1>(sa, sb, oa, ob, a[(U + 1) & 1], b[(U + 1) & 1]);
        else if (more)
            load_row<0>(sa, sb, oa + 8 * 128, ob + 8 * 128, a[0], b[0]);
        K::template fma_block<TM>(a[U & 1], b[U & 1], acc);
    }

    // acc += A^T B over the 32 k rows of one stage.
    static __device__ __forceinline__ void compute(const float *sa_, const float *sb_,
                                                   float (&acc)[TM][TN], int tx, int ty)
    {
        const char *sa = reinterpret_cast<const char *>(sa_);
        const char *sb = reinterpret_cast<const char *>(sb_);
        uint32_t oa = tx * 16;
        uint32_t ob = (ty >> 3) * 4096 + (ty & 7) * 16;
        float a[2][TM], b[2][TN];
        load_row<0>(sa, sb, oa, ob, a[0], b[0]);
#pragma unroll 1
        for (int k0 = 0; k0 < 32; k0 += 8) {
            const bool more = k0 + 8 < 32;
            step<0>(sa, sb, oa, ob, more, a, b, acc);
            step<1>(sa, sb, oa, ob, more, a, b, acc);
            step<2>(sa, sb, oa, ob, more, a, b, acc);
            step<3>(sa, sb, oa, ob, more, a, b, acc);
            step<4>(sa, sb, oa, ob, more, a, b, acc);
            step<5>(sa, sb, oa, ob, more, a, b, acc);
            step<6>(sa, sb, oa, ob, more, a, b, acc);
            step<7>(sa, sb, oa, ob, more, a, b, acc);
            oa += 8 * 128;
            ob += 8 * 128;
        }
    }

    // C[tile] := alpha*acc + beta*C[tile] (C not read when beta == 0), the operations of the
    // shared tile core's epilogue.  C is read two columns (32 values) at a time, all loads
    // issued before any store, so a tile's epilogue costs four round trips to L2 (where the
    // prefetch at segment start has put C), not one per 4-row chunk.
    static __device__ void epilogue(const GemmParams<float> &p, int i, int j, int tid,
                                    const float (&acc)[TM][TN])
    {
        constexpr int CH = 4;
        const int tx = tid % TX, ty = tid / TX;
        const bool read_c = (p.beta != 0.f);
#pragma unroll
        for (int j0 = 0; j0 < TN; j0 += 2) {
            float cv[2][TM];
#pragma unroll
            for (int d = 0; d < 2; ++d) {
                const int jj = j0 + d;
                const int col = j * 128 + ty * CH + (jj % CH) + (jj / CH) * (128 / NCN);
                const float *ccol = p.C + (int64_t)col * p.ldc;
#pragma unroll
                for (int ii = 0; ii < TM; ++ii) {
                    const int row = i * 128 + tx * CH + (ii % CH) + (ii / CH) * (128 / NCM);
                    cv[d][ii] = (read_c && col < p.n && row < p.m) ? ccol[row] : 0.f;
                }
            }
#pragma unroll
            for (int d = 0; d < 2; ++d) {
                const int jj = j0 + d;
                const int col = j * 128 + ty * CH + (jj % CH) + (jj / CH) * (128 / NCN);
                if (col >= p.n) continue;
                float *ccol = p.C + (int64_t)col * p.ldc;
#pragma unroll
                for (int ii = 0; ii < TM; ++ii) {
                    const int row = i * 128 + tx * CH + (ii % CH) + (ii / CH) * (128 / NCM);
                    if (row >= p.m) continue;
                    float v = p.alpha * acc[ii][jj];
                    if (read_c) v = fmaf(p.beta, cv[d][ii], v);
                    ccol[row] = v;
                }
            }
        }
    }

    // The last virtual CTA of a split tile: adds the segments' partial-sum tiles in k order and
    // applies the epilogue, with coalesced float4 loads, 8 per thread in flight (this thread's
    // share: float4 f = tid + 128 r of the tile, r = 0..31, i.e. column f / 32, rows 4 (f % 32)).
    static __device__ __forceinline__ void reduce_split_tile(const GemmParams<float> &p, int i,
                                                             int j, int u, int g0, int g1,
                                                             int tid)
    {
        const int64_t S = p.sk_iters;
        const int G = p.grid;
        constexpr int PART = 8;
        const bool read_c = (p.beta != 0.f);
#pragma unroll 1
        for (int r0 = 0; r0 < 32; r0 += PART) {
            float4 sum[PART];
            for (int gs = g0; gs <= g1; ++gs) {
                const int64_t lo = S * gs / G;
                const int gslot = (lo / p.kt == u) ? 0 : 1;
                const float4 *src = reinterpret_cast<const float4 *>(
                    p.partial + (int64_t)(2 * gs + gslot) * (128 * 128));
                float4 v[PART];
#pragma unroll
                for (int r = 0; r < PART; ++r) v[r] = __ldcg(src + tid + 128 * (r0 + r));
#pragma unroll
                for (int r = 0; r < PART; ++r) {
                    if (gs == g0) {
                        sum[r] = v[r];
                    } else {
                        sum[r].x += v[r].x;
                        sum[r].y += v[r].y;
                        sum[r].z += v[r].z;
                        sum[r].w += v[r].w;
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < PART; ++r) {
                const int f = tid + 128 * (r0 + r);
                const int col = j * 128 + f / 32, row0 = i * 128 + 4 * (f % 32);
                if (col >= p.n) continue;
                float *ccol = p.C + (int64_t)col * p.ldc;
                const float sv[4] = {sum[r].x, sum[r].y, sum[r].z, sum[r].w};
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    if (row0 + w >= p.m) continue;
                    float v = p.alpha * sv[w];
                    if (read_c) v = fmaf(p.beta, ccol[row0 + w], v);
                    ccol[row0 + w] = v;
                }
            }
        }
    }

    // Split-tile fix-up.  Every segment stores its partial sums as a column-major 128 x 128
    // tile (float4 stores of 4 consecutive rows); the virtual CTA that arrives last adds the
    // segments' tiles in k order (the order of the shared tile core, so the same bits).
    static __device__ void fixup(const GemmParams<float> &p, Ring &rg, int ring, int g, int t,
                                 int i, int j, int slot, const float (&acc)[TM][TN],
                                 unsigned int epoch, int tid)
    {
        const int tx = tid % TX, ty = tid / TX;
        const int64_t S = p.sk_iters;
        const int G = p.grid;
        const int u = t - p.dp_tiles;
        const int g0 = K::cta_of((int64_t)u * p.kt, S, G);
        const int g1 = K::cta_of((int64_t)(u + 1) * p.kt - 1, S, G);
        const int nseg = g1 - g0 + 1;
        float *mine = p.partial + (int64_t)(2 * g + slot) * (128 * 128);
#pragma unroll
        for (int jj = 0; jj < TN; ++jj) {
            const int col = ty * 4 + (jj % 4) + (jj / 4) * (128 / NCN);
#pragma unroll
            for (int c = 0; c < NCM; ++c)
                __stcg(reinterpret_cast<float4 *>(mine + col * 128 + tx * 4 + c * (128 / NCM)),
                       make_float4(acc[c * 4 + 0][jj], acc[c * 4 + 1][jj], acc[c * 4 + 2][jj],
                                   acc[c * 4 + 3][jj]));
        }
        math_barrier(ring);
        if (tid == 0) {
            __threadfence();
            const unsigned long long tag = static_cast<unsigned long long>(epoch) << 32;
            atomicMax(p.tile_count + t, tag);
            const unsigned long long old = atomicAdd(p.tile_count + t, 1ull);
            const long long cnt = static_cast<long long>(old - tag) + 1;
            if ((old >> 32) != epoch || cnt > nseg) atomicOr(p.status, STATUS_BAD_SEGMENT);
            rg.flag = (cnt == nseg);
            __threadfence();
        }
        math_barrier(ring);
        if (rg.flag) reduce_split_tile(p, i, j, u, g0, g1, tid);
        math_barrier(ring);
    }

    static __device__ void math(const GemmParams<float> &p, Smem &sm, Ring &rg, int ring, int g)
    {
        const int tid = threadIdx.x & (MATH_THREADS - 1);
        const int tx = tid % TX, ty = tid / TX;
        unsigned int epoch = 0u;
        if (tid == 0) epoch = *(volatile unsigned int *)p.launch_count + 1u;
        float acc[TM][TN];
        int st = 0;          // stage of the next k-block
        uint32_t ph = 0;     // parity of that stage's next full phase
        SegCursor cur;
        cur.start(p, g);
        Segment sg;
        bool ok = true;
        while (ok && cur.next(p, sg)) {
            const int i = sg.i, j = sg.j;
#pragma unroll
            for (int ii = 0; ii < TM; ++ii)
#pragma unroll
                for (int jj = 0; jj < TN; ++jj) acc[ii][jj] = 0.f;
            // the segment that ends the tile's k loop will read C: warm L2 with it now
            if (sg.kb1 == p.kt && p.beta != 0.f) {
                constexpr int PER_COL = 128 / 32;
                for (int e = tid; e < 128 * PER_COL; e += MATH_THREADS) {
                    const int col = j * 128 + e / PER_COL, row = i * 128 + (e % PER_COL) * 32;
                    if (col < p.n && row < p.m)
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(p.C + row +
                                                                       (int64_t)col * p.ldc));
                }
            }
            for (int kb = sg.kb0; kb < sg.kb1; ++kb) {
                if (!mbar_wait(&rg.full[st], ph, sm, p.status)) {
                    ok = false;
                    break;
                }
                compute(rg.a[st], rg.b[st], acc, tx, ty);
                __syncwarp();
                if ((tid & 31) == 0) mbar_arrive(&rg.empty[st]);
                if (++st == STAGES) {
                    st = 0;
                    ph ^= 1u;
                }
            }
            if (!ok) break;
            if (sg.kb0 == 0 && sg.kb1 == p.kt)
                epilogue(p, i, j, tid, acc);
            else
                fixup(p, rg, ring, g, sg.t, i, j, sg.slot, acc, epoch, tid);
        }
    }
};

// One CTA per SM: warpgroups 0 and 1 are the math warpgroups of virtual CTAs 2 * block and
// 2 * block + 1 (a virtual id at or past the grid has no work), warpgroup 2 holds their
// producers (warp 8 + 2 r: op(A) of ring r, warp 9 + 2 r: op(B)).  The launch's epoch tags its
// ready words and arrival counters exactly as in gemm_kernel: every role reads the launch
// counter at start, and the last CTA to finish advances it.
template <bool ACONTIG, bool BCONTIG>
__global__ void __launch_bounds__(THREADS, 1) ws_gemm_kernel(const GemmParams<float> p)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    const int warp = threadIdx.x >> 5;
    const int wg = warp >> 2;
    if (threadIdx.x == 0) {
        for (int r = 0; r < VCTA; ++r)
            for (int s = 0; s < STAGES; ++s) {
                mbar_init(&sm.ring[r].full[s], 2 * 33);   // A and B producers: 32 lanes + tx
                mbar_init(&sm.ring[r].empty[s], MATH_WARPS);
            }
        sm.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (wg == VCTA) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(PRODUCER_REGS));
        const int w = warp - 4 * VCTA;          // 0..3
        const int r = w >> 1;
        const int g = VCTA * blockIdx.x + r;
        if (g < p.grid) {
            if (w & 1)
                WsKernel<ACONTIG, BCONTIG>::template producer<true>(p, sm, sm.ring[r], g);
            else
                WsKernel<ACONTIG, BCONTIG>::template producer<false>(p, sm, sm.ring[r], g);
        }
    } else {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(MATH_REGS));
        const int g = VCTA * blockIdx.x + wg;
        if (g < p.grid) WsKernel<ACONTIG, BCONTIG>::math(p, sm, sm.ring[wg], wg, g);
    }
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

// Pack kernel of the pack-then-compute variant for this tile core: one warp per (panel,
// k-block) tile, A tiles first; raw copies into shared memory in the swizzled layout, then
// the 16 KB image to the packed buffer with 16-byte stores.
constexpr int PACK_WARPS = 4;

template <bool ACONTIG, bool BCONTIG>
__global__ void __launch_bounds__(PACK_WARPS * 32) ws_pack_kernel(const PackParams<float> p)
{
    extern __shared__ __align__(128) unsigned char pack_smem[];
    float (*tile)[TILE_FLOATS] = reinterpret_cast<float (*)[TILE_FLOATS]>(pack_smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t a_tiles = (int64_t)p.mt * p.kt;
    const int64_t total = a_tiles + (int64_t)p.nt * p.kt;
    const int64_t b = (int64_t)blockIdx.x * PACK_WARPS + warp;
    if (b >= total) return;
    float *dst;
    const uint32_t s = smem_addr(tile[warp]);
    if (b < a_tiles) {
        const int i = static_cast<int>(b / p.kt), kb = static_cast<int>(b % p.kt);
        raw_tile<ACONTIG>(s, p.A, p.lda, i * 128, kb * 32, p.m, p.k - kb * 32, lane);
        dst = p.pack_a + b * TILE_FLOATS;
    } else {
        const int64_t bb = b - a_tiles;
        const int j = static_cast<int>(bb / p.kt), kb = static_cast<int>(bb % p.kt);
        raw_tile<BCONTIG>(s, p.B, p.ldb, j * 128, kb * 32, p.n, p.k - kb * 32, lane);
        dst = p.pack_b + bb * TILE_FLOATS;
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncwarp();
    const uint4 *src = reinterpret_cast<const uint4 *>(tile[warp]);
    uint4 *d = reinterpret_cast<uint4 *>(dst);
#pragma unroll 8
    for (int c = lane; c < TILE_BYTES / 16; c += 32) __stcg(d + c, src[c]);
}

inline size_t smem_bytes()
{
    return sizeof(Smem);
}

constexpr size_t PACK_SMEM = (size_t)PACK_WARPS * TILE_BYTES;

// The register split of the warpgroups (setmaxnreg) assumes the kernel is launched with
// exactly LAUNCH_REGS registers a thread: with fewer, the math warpgroups' increase could never
// be granted.  A build where the compiler chose another count is refused here.
template <bool AC, bool BC> cudaError_t configure()
{
    static bool configured = false;
    if (configured) return cudaSuccess;
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, ws_gemm_kernel<AC, BC>);
    if (e != cudaSuccess) return e;
    if (fa.numRegs != LAUNCH_REGS) return cudaErrorInvalidConfiguration;
    e = cudaFuncSetAttribute(ws_gemm_kernel<AC, BC>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem_bytes()));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ws_pack_kernel<AC, BC>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(PACK_SMEM));
    if (e == cudaSuccess) configured = true;
    return e;
}

template <bool AC, bool BC> cudaError_t launch_t(const GemmParams<float> &p, cudaStream_t s)
{
    cudaError_t e = configure<AC, BC>();
    if (e != cudaSuccess) return e;
    ws_gemm_kernel<AC, BC><<<(p.grid + VCTA - 1) / VCTA, THREADS, smem_bytes(), s>>>(p);
    return cudaGetLastError();
}

template <bool AC, bool BC> cudaError_t launch_pack_t(const PackParams<float> &p, cudaStream_t s)
{
    const int64_t tiles = (int64_t)(p.mt + p.nt) * p.kt;
    if (tiles <= 0) return cudaSuccess;
    cudaError_t e = configure<AC, BC>();
    if (e != cudaSuccess) return e;
    const unsigned int blocks = static_cast<unsigned int>((tiles + PACK_WARPS - 1) / PACK_WARPS);
    ws_pack_kernel<AC, BC><<<blocks, PACK_WARPS * 32, PACK_SMEM, s>>>(p);
    return cudaGetLastError();
}

// Virtual CTAs per SM (the unit of the shared schedule): VCTA per resident CTA.
template <bool AC, bool BC> int blocks_per_sm_one()
{
    if (configure<AC, BC>() != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, ws_gemm_kernel<AC, BC>, THREADS,
                                                      smem_bytes()) != cudaSuccess)
        return 0;
    return n * VCTA;
}

}  // namespace ws
}  // namespace gfip
