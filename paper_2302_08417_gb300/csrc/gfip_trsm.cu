// gfip_trsm.cu -- the panel solves of the blocked triangular solve (TRSM).
//
// TRSM runs as a sequence over panels of op(A)'s diagonal (see gfip_api.cu): each step solves
// one panel of at most TRSM_PANEL unknowns for every right-hand side with the kernel below,
// then the fused GEMM kernel subtracts the panel's contribution from the unknowns still to be
// solved.  The kernel solves a panel by column-oriented substitution: once unknown d is known
// (divided by its diagonal entry), every unknown below it loses its multiple at once; per
// chunk of columns the chain updates only its own 32-row group, and the later groups are
// updated afterwards, off the chain.  A warp holds one or two right-hand sides, one element
// per lane and 32-row group, in registers; the panel's triangle streams through shared memory
// in chunks of columns, double-buffered and shared by the CTA's warps, the next chunk loaded
// into registers while this one is solved.  Only the entries a triangular solve reads are
// read: never the other triangle, nor a unit diagonal.
#include <cstdint>

#include "gfip_internal.h"

namespace gfip {
namespace trsm {

// Right-hand sides per warp: FP32 two (8 warps a CTA: the two chains interleave within the
// warp; 6 % faster at 2048 x 2048 than one a warp in 16 warps), FP64 one (its registers do
// not hold two, and it is bound by its DFMA pipe): the shortest chain per right-hand side.
// FP64 runs between 8 and 16 warps a CTA, as many as spread the right-hand sides over all SMs
// (2048 of them on 152 SMs: 14 a CTA, 147 CTAs, 11 % faster than 16 a CTA on 128 SMs).
template <typename T> struct Shape {
    static constexpr int RPW = sizeof(T) == 4 ? 2 : 1;
    static constexpr int MIN_WARPS = 8 / RPW, MAX_WARPS = 16 / RPW;
    // staging slots a thread takes per half chunk: one with 512 threads, more with fewer
    // (the kernel is compiled for each)
    static constexpr int MAX_SLOTS = TRSM_PANEL / (MIN_WARPS * 32);
};
constexpr int ROWS = TRSM_PANEL / 32;     // 32-row groups of a panel: registers per vector
constexpr int CW = 16;                    // triangle columns per staged chunk
constexpr int HALF = CW / 2;              // columns staged together
static_assert(TRSM_PANEL % 32 == 0 && 32 % CW == 0, "a 32-row group is whole chunks");
static_assert(ROWS == 16, "the group update below is written out for 16 groups");
// A chunk buffer holds one row of CW triangle entries per unknown of the panel, rows padded to
// PADW elements: a lane reads its row 16 bytes at a time, and the 8 lanes of one shared-memory
// wavefront (rows 80 or 144 bytes apart) fall on distinct banks.
template <typename T> __host__ __device__ constexpr int padw() { return CW + 16 / (int)sizeof(T); }
template <typename T> __host__ __device__ constexpr size_t buf_elems() { return (size_t)TRSM_PANEL * padw<T>(); }
// two chunk buffers, two diagonals and two reciprocal diagonals
template <typename T> constexpr size_t smem_bytes() { return sizeof(T) * (2 * buf_elems<T>() + 4 * CW); }

// 16-byte shared-memory accesses of a row (float4 / double2)
__device__ __forceinline__ void ld16(const float *s, float (&v)[4])
{
    const float4 t = *reinterpret_cast<const float4 *>(s);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld16(const double *s, double (&v)[2])
{
    const double2 t = *reinterpret_cast<const double2 *>(s);
    v[0] = t.x; v[1] = t.y;
}
__device__ __forceinline__ void st16(float *s, const float *v)
{
    *reinterpret_cast<float4 *>(s) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st16(double *s, const double *v)
{
    *reinterpret_cast<double2 *>(s) = make_double2(v[0], v[1]);
}

// The panel's system in solve order: unknown q of the local lower triangular system is row
// lower_t ? q : pw - 1 - q of the block, so an upper triangular block is solved by the same
// forward loop.  t(r, c) = op(A)[k0 + r, k0 + c] (side 'L') or op(A)[k0 + c, k0 + r] (side
// 'R', transpose_t), op(A)[i, j] = A[i + j lda] ('N') or A[j + i lda] ('T').  Every case is
// linear in (q, d): t(q, d) sits at A0[q sq + d sd], the three set on the host
// (launch_trsm_panel); one of |sq|, |sd| is 1.
struct Panel {
    const void *A0;
    int64_t sq, sd;
    int along_q;        // |sq| == 1: a column of the local system is contiguous
    int lower_t, unit;
    int pw;
    __device__ __forceinline__ int row(int q) const { return lower_t ? q : pw - 1 - q; }
};

// Staging of chunk [d0, d0 + CW) of the strictly lower part of the local system: row q of
// the buffer holds t(q, d0 + dd) at buf[q PADW + dd] for q > d0 + dd, zero elsewhere, for the
// rows of the chunk's 32-row group and after (qlo <= q < qhi), and the chunk's diagonal
// (unless unit) with its reciprocals.  A chunk is staged in two halves of HALF columns,
// each a half's loads into registers issued ahead of the work they hide behind and stored to
// shared memory after it.  Where columns are contiguous in A (along_q) a thread stages rows
// (q = qlo + tid + i NT) and stores each row's half with 16-byte stores; otherwise a thread
// keeps one column (dd = tid % CW) and stages every (NT / CW)-th row, so that a warp's loads
// run along A's rows either way.  A warp whose rows all lie past qhi skips its slot.
template <typename T, int SLOTS> struct Stage {
    T v[SLOTS][HALF];
    T diag;
};

template <int SLOTS>
__device__ __forceinline__ int stage_row(const Panel &p, int qlo, int hf, int i, int j, int e)
{
    // row of slot (i, j) of half hf for thread e (e = tid, or tid & ~31 for the warp's first)
    const int nt = blockDim.x;
    if (p.along_q) return qlo + e + i * nt;
    return qlo + e / CW + ((hf * HALF + j) * SLOTS + i) * (nt / CW);
}

template <typename T, int SLOTS>
__device__ __forceinline__ void stage_load(const Panel &p, int d0, int hf, int tid,
                                           Stage<T, SLOTS> &st)
{
    const T *A0 = static_cast<const T *>(p.A0);
    const int qlo = d0 & ~31, qhi = (p.pw + 31) & ~31, pw = p.pw;
    const int wfirst = tid & ~31;
    if (p.along_q) {
#pragma unroll
        for (int i = 0; i < SLOTS; ++i) {
            if (stage_row<SLOTS>(p, qlo, hf, i, 0, wfirst) >= qhi) continue;   // warp-uniform
            const int q = stage_row<SLOTS>(p, qlo, hf, i, 0, tid);
            const int da = d0 + hf * HALF;
            const T *src = A0 + (int64_t)q * p.sq + (int64_t)da * p.sd;
#pragma unroll
            for (int j = 0; j < HALF; ++j) {
                st.v[i][j] = (q > da + j && q < pw) ? *src : T(0);
                src += p.sd;
            }
        }
    } else {
        const int d = d0 + (tid % CW);
#pragma unroll
        for (int j = 0; j < HALF; ++j)
#pragma unroll
            for (int i = 0; i < SLOTS; ++i) {
                if (stage_row<SLOTS>(p, qlo, hf, i, j, wfirst) >= qhi) continue;
                const int q = stage_row<SLOTS>(p, qlo, hf, i, j, tid);
                st.v[i][j] = (q > d && q < pw) ? A0[(int64_t)q * p.sq + (int64_t)d * p.sd] : T(0);
            }
    }
    if (hf == 0 && tid < CW) {
        const int d = d0 + tid;
        st.diag = (!p.unit && d < pw) ? A0[(int64_t)d * (p.sq + p.sd)] : T(1);
    }
}

template <typename T, int SLOTS>
__device__ __forceinline__ void stage_store(const Panel &p, int d0, int hf, int tid,
                                            const Stage<T, SLOTS> &st, T *buf, T *dg, T *dr)
{
    constexpr int PADW = padw<T>(), V = 16 / (int)sizeof(T);
    const int qlo = d0 & ~31, qhi = (p.pw + 31) & ~31;
    const int wfirst = tid & ~31;
    if (p.along_q) {
#pragma unroll
        for (int i = 0; i < SLOTS; ++i) {
            if (stage_row<SLOTS>(p, qlo, hf, i, 0, wfirst) >= qhi) continue;
            const int q = stage_row<SLOTS>(p, qlo, hf, i, 0, tid);
            if (q < qhi) {
                T *row = buf + q * PADW + hf * HALF;
#pragma unroll
                for (int j = 0; j < HALF; j += V) st16(row + j, &st.v[i][j]);
            }
        }
    } else {
        const int dd = tid % CW;
#pragma unroll
        for (int j = 0; j < HALF; ++j)
#pragma unroll
            for (int i = 0; i < SLOTS; ++i) {
                if (stage_row<SLOTS>(p, qlo, hf, i, j, wfirst) >= qhi) continue;
                const int q = stage_row<SLOTS>(p, qlo, hf, i, j, tid);
                if (q < qhi) buf[q * PADW + dd] = st.v[i][j];
            }
    }
    if (hf == 0 && tid < CW) {
        dg[tid] = st.diag;
        dr[tid] = p.unit ? T(1) : T(1) / st.diag;
    }
}

// b / t from r = RN(1 / t): the product corrected by one exact residual step (an FMA gives
// b - t q0 exactly), which lands on the correctly rounded quotient or next to it; a
// non-finite result takes the division itself (its IEEE special values).
template <typename T> __device__ __noinline__ T divide(T b, T t) { return b / t; }

template <typename T> __device__ __forceinline__ T quotient(T b, T t, T r)
{
    const T q0 = b * r;
    const T q = fma(fma(-t, q0, b), r, q0);
    // a zero, infinite or NaN t (r infinite, zero or NaN) or a non-finite b makes q
    // non-finite; the division then gives the IEEE result (a call, so that it is never
    // evaluated on the common path)
    if (__builtin_expect(!isfinite(q), 0)) return divide(b, t);
    return q;
}

// b[R][w] -= sum over the chunk's columns dd, in order, of t(32 R + lane, d0 + dd) x[dd][w]:
// this lane's element of group R of every right-hand side (row = this lane's buffer row in
// group 0), the row read 16 bytes at a time.
template <typename T, int R, int RPW>
__device__ __forceinline__ void update_group(T (&b)[ROWS][RPW], const T *row,
                                             const T (&x)[CW][RPW])
{
    constexpr int PADW = padw<T>(), V = 16 / (int)sizeof(T);
    const T *r = row + 32 * R * PADW;
#pragma unroll
    for (int d4 = 0; d4 < CW; d4 += V) {
        T t[V];
        ld16(r + d4, t);
#pragma unroll
        for (int j = 0; j < V; ++j)
#pragma unroll
            for (int w = 0; w < RPW; ++w) b[R][w] = fma(-t[j], x[d4 + j][w], b[R][w]);
    }
}

template <typename T, int SLOTS>
__global__ void __launch_bounds__(Shape<T>::MAX_WARPS * 32, 1)
    panel_kernel(T *B, int64_t vstride, int64_t estride, int nvec, const Panel p)
{
    constexpr int RPW = Shape<T>::RPW;
    constexpr int PADW = padw<T>(), V = 16 / (int)sizeof(T);
    constexpr size_t BUF = buf_elems<T>();
    const int rpc = (blockDim.x >> 5) * RPW;   // right-hand sides of this CTA
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *bufs = reinterpret_cast<T *>(smem_raw);
    T *dgs = bufs + 2 * BUF;     // [2][CW] diagonal entries
    T *drs = dgs + 2 * CW;       // [2][CW] their reciprocals
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int pw = p.pw;

    // element q of right-hand side w (this warp's) is b[q / 32][w] on lane q % 32; element i
    // of vector v sits at B[v vstride + i estride]
    T b[ROWS][RPW];
    int vec[RPW];
#pragma unroll
    for (int w = 0; w < RPW; ++w) vec[w] = blockIdx.x * rpc + warp * RPW + w;
#pragma unroll
    for (int r = 0; r < ROWS; ++r)
#pragma unroll
        for (int w = 0; w < RPW; ++w) {
            const int q = 32 * r + lane;
            b[r][w] = (q < pw && vec[w] < nvec)
                          ? B[(int64_t)vec[w] * vstride + (int64_t)p.row(q) * estride]
                          : T(0);
        }

    {
        Stage<T, SLOTS> st;
        stage_load<T, SLOTS>(p, 0, 0, tid, st);
        stage_store<T, SLOTS>(p, 0, 0, tid, st, bufs, dgs, drs);
        stage_load<T, SLOTS>(p, 0, 1, tid, st);
        stage_store<T, SLOTS>(p, 0, 1, tid, st, bufs, dgs, drs);
    }
    // The groups run in a loop, not unrolled (the code stays small enough for the instruction
    // cache): the group being solved moves into cur[] and back; the later groups are
    // updated through a switch that enters at the first of them.  One barrier a chunk: the
    // one that publishes chunk ch also ends every warp's reads of the buffer restaged next.
    int ch = 0;   // chunks begun
#pragma unroll 1
    for (int r = 0; r < ROWS; ++r) {
        if (32 * r >= pw) break;
        T cur[RPW];
#pragma unroll
        for (int rr = 0; rr < ROWS; ++rr)
            if (rr == r) {
#pragma unroll
                for (int w = 0; w < RPW; ++w) cur[w] = b[rr][w];
            }
        const T *lrow = nullptr;   // this lane's row of group 0 in the current buffer
#pragma unroll 1
        for (int h = 0; h < 32 / CW; ++h) {
            const int d0 = 32 * r + h * CW;
            if (d0 >= pw) break;
            __syncthreads();      // chunk ch is in shared memory
            const T *tb = bufs + (ch & 1) * BUF;
            const T *dg = dgs + (ch & 1) * CW, *dr = drs + (ch & 1) * CW;
            lrow = tb + lane * PADW;
            const bool more = d0 + CW < pw;   // a next chunk to stage meanwhile
            T *nbuf = bufs + ((ch + 1) & 1) * BUF;
            T *ndg = dgs + ((ch + 1) & 1) * CW, *ndr = drs + ((ch + 1) & 1) * CW;
            Stage<T, SLOTS> st;
            if (more) stage_load<T, SLOTS>(p, d0 + CW, 0, tid, st);
            const int dn = min(CW, pw - d0);
            // this lane's row of the chunk (its entries left of the diagonal: FP32 reads it
            // whole ahead of the chain, FP64, short of registers, an entry a step), and, for
            // the lane whose unknown is in the chunk, its diagonal entry and reciprocal
            const int ln = lane - h * CW;   // this lane's unknown within the chunk, if in range
            const T *crow = lrow + 32 * r * PADW;
            constexpr bool PRELOAD = sizeof(T) == 4;
            T trow[CW];
            if (PRELOAD) {
#pragma unroll
                for (int d4 = 0; d4 < CW; d4 += V) {
                    T v[V];
                    ld16(crow + d4, v);
#pragma unroll
                    for (int j = 0; j < V; ++j) trow[d4 + j] = v[j];
                }
            }
            const bool inch = ln >= 0 && ln < CW;
            const int lc = ln < 0 ? 0 : (ln >= CW ? CW - 1 : ln);
            const T t = dg[lc], rt = dr[lc];
            // the chunk's unknowns one after another; each updates only the later unknowns
            // of its own 32-row group here (the chain's latency is the solve's floor).
            // A whole chunk first takes the short form: every lane forms the quotient of its
            // own element (by its own diagonal entry; lanes outside the chunk, and a unit
            // diagonal, by 1), the owner's is broadcast, and every lane subtracts its multiple
            // with its row's entry, which is zero on and above the diagonal, so that the
            // chunk's unknowns keep their last right-hand side and take their quotient once
            // the chunk is done (the one the owner broadcast: the same operands).  A
            // non-finite quotient in any lane makes the chunk run again in the exact form
            // below (owner-only quotients, the division for special values), as does a short
            // last chunk.  With finite values both forms give the same bits.  FP64 keeps the
            // exact form: its extra multiply-adds would load the DFMA pipe that bounds it.
            bool exact = sizeof(T) == 8 || dn < CW;
            if (!exact) {
                const T tl = inch ? t : T(1), rl = inch ? rt : T(1);
                T cur0[RPW];
                T acc = T(0);   // stays zero while every quotient is finite
#pragma unroll
                for (int w = 0; w < RPW; ++w) cur0[w] = cur[w];
#pragma unroll
                for (int dd = 0; dd < CW; ++dd)
#pragma unroll
                    for (int w = 0; w < RPW; ++w) {
                        const T q0 = cur[w] * rl;
                        const T qv = fma(fma(-tl, q0, cur[w]), rl, q0);
                        acc = fma(qv, T(0), acc);
                        const T x = __shfl_sync(0xffffffffu, qv, h * CW + dd);
                        cur[w] = fma(-(PRELOAD ? trow[dd] : crow[dd]), x, cur[w]);
                    }
                if (__any_sync(0xffffffffu, !(acc == T(0)))) {
                    exact = true;
#pragma unroll
                    for (int w = 0; w < RPW; ++w) cur[w] = cur0[w];
                } else if (inch) {
#pragma unroll
                    for (int w = 0; w < RPW; ++w) {
                        const T q0 = cur[w] * rl;
                        cur[w] = fma(fma(-tl, q0, cur[w]), rl, q0);
                    }
                }
            }
            if (exact) {
#pragma unroll
                for (int dd = 0; dd < CW; ++dd) {
                    if (dd >= dn) break;
#pragma unroll
                    for (int w = 0; w < RPW; ++w) {
                        T bc = cur[w];
                        if (!p.unit && ln == dd) bc = quotient(bc, t, rt);
                        const T x = __shfl_sync(0xffffffffu, bc, h * CW + dd);
                        if (ln == dd) cur[w] = x;
                        if (ln > dd) cur[w] = fma(-(PRELOAD ? trow[dd] : crow[dd]), x, cur[w]);
                    }
                }
            }
            if (more) {
                stage_store<T, SLOTS>(p, d0 + CW, 0, tid, st, nbuf, ndg, ndr);
                stage_load<T, SLOTS>(p, d0 + CW, 1, tid, st);
            }
            // then the chunk's unknowns leave the later groups, in the same order (the
            // multiply-adds of every element still run in increasing column order), free of
            // the chain: every group and right-hand side an independent accumulation.  The
            // chunk's solved unknowns are gathered once; a group's update is then straight-line
            // code over the chunk's columns, entered at the first later group and falling
            // through the rest (no instruction for a group that is done).  Columns past the
            // panel (a short last chunk) hold zeros in the staged triangle and take zero
            // unknowns here, so they change nothing.
            T xs[CW][RPW];
#pragma unroll
            for (int dd = 0; dd < CW; ++dd)
#pragma unroll
                for (int w = 0; w < RPW; ++w) {
                    const T x = __shfl_sync(0xffffffffu, cur[w], h * CW + dd);
                    xs[dd][w] = dd < dn ? x : T(0);
                }
            switch (r) {
#define GFIP_TRSM_GROUP(R)                                                                  \
    case R - 1:                                                                             \
        if (32 * R < pw) update_group<T, R, RPW>(b, lrow, xs);                              \
        [[fallthrough]];
                GFIP_TRSM_GROUP(1) GFIP_TRSM_GROUP(2) GFIP_TRSM_GROUP(3)
                GFIP_TRSM_GROUP(4) GFIP_TRSM_GROUP(5) GFIP_TRSM_GROUP(6)
                GFIP_TRSM_GROUP(7) GFIP_TRSM_GROUP(8) GFIP_TRSM_GROUP(9)
                GFIP_TRSM_GROUP(10) GFIP_TRSM_GROUP(11) GFIP_TRSM_GROUP(12)
                GFIP_TRSM_GROUP(13) GFIP_TRSM_GROUP(14) GFIP_TRSM_GROUP(15)
#undef GFIP_TRSM_GROUP
            default: break;
            }
            if (more) stage_store<T, SLOTS>(p, d0 + CW, 1, tid, st, nbuf, ndg, ndr);
            ++ch;
        }
#pragma unroll
        for (int rr = 0; rr < ROWS; ++rr)
            if (rr == r) {
#pragma unroll
                for (int w = 0; w < RPW; ++w) b[rr][w] = cur[w];
            }
    }

#pragma unroll
    for (int r = 0; r < ROWS; ++r)
#pragma unroll
        for (int w = 0; w < RPW; ++w) {
            const int q = 32 * r + lane;
            if (q < pw && vec[w] < nvec)
                B[(int64_t)vec[w] * vstride + (int64_t)p.row(q) * estride] = b[r][w];
        }
}

}  // namespace trsm

template <typename T>
cudaError_t launch_trsm_panel_impl(T *B, int64_t vstride, int64_t estride, int nvec,
                                   const T *A, int64_t lda, int a_trans, int k0, int pw,
                                   int lower_t, int transpose_t, int unit, cudaStream_t s)
{
    if (nvec <= 0 || pw <= 0) return cudaSuccess;
    if (pw > TRSM_PANEL) return cudaErrorInvalidValue;
    using S = trsm::Shape<T>;
    static bool configured = false;
    if (!configured) {
        for (auto *k : {trsm::panel_kernel<T, 1>, trsm::panel_kernel<T, 2>,
                        trsm::panel_kernel<T, S::MAX_SLOTS>}) {
            const cudaError_t e =
                cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(trsm::smem_bytes<T>()));
            if (e != cudaSuccess) return e;
        }
        configured = true;
    }
    trsm::Panel p;
    // t(q, d): row index i and column index j of op(A) are k0 + r0 + sgn q and k0 + r0 + sgn d
    // (swapped for side 'R'); op(A)[i, j] is element i + j lda ('N') or j + i lda ('T')
    const int64_t ci = a_trans ? lda : 1, cj = a_trans ? 1 : lda;
    const int64_t cq = transpose_t ? cj : ci, cd = transpose_t ? ci : cj;
    const int sgn = lower_t ? 1 : -1;
    p.A0 = A + (int64_t)(k0 + (lower_t ? 0 : pw - 1)) * (cq + cd);
    p.sq = sgn * cq;
    p.sd = sgn * cd;
    p.along_q = cq == 1;
    p.lower_t = lower_t;
    p.unit = unit;
    p.pw = pw;
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    const int want = (nvec + sms * S::RPW - 1) / (sms * S::RPW);
    const int warps = sizeof(T) == 4 ? S::MAX_WARPS
                      : want < S::MIN_WARPS ? S::MIN_WARPS
                                            : (want > S::MAX_WARPS ? S::MAX_WARPS : want);
    const int rpc = warps * S::RPW;
    const int blocks = (nvec + rpc - 1) / rpc;
    if (warps * 32 >= TRSM_PANEL)
        trsm::panel_kernel<T, 1><<<blocks, warps * 32, trsm::smem_bytes<T>(), s>>>(
            B, vstride, estride, nvec, p);
    else if (warps * 64 >= TRSM_PANEL)
        trsm::panel_kernel<T, 2><<<blocks, warps * 32, trsm::smem_bytes<T>(), s>>>(
            B, vstride, estride, nvec, p);
    else
        trsm::panel_kernel<T, S::MAX_SLOTS><<<blocks, warps * 32, trsm::smem_bytes<T>(), s>>>(
            B, vstride, estride, nvec, p);
    return cudaGetLastError();
}

template <>
cudaError_t launch_trsm_panel<double>(double *B, int64_t vstride, int64_t estride, int nvec,
                                      const double *A, int64_t lda, int a_trans, int k0, int pw,
                                      int lower_t, int transpose_t, int unit, cudaStream_t s)
{
    return launch_trsm_panel_impl<double>(B, vstride, estride, nvec, A, lda, a_trans, k0, pw,
                                          lower_t, transpose_t, unit, s);
}

template <>
cudaError_t launch_trsm_panel<float>(float *B, int64_t vstride, int64_t estride, int nvec,
                                     const float *A, int64_t lda, int a_trans, int k0, int pw,
                                     int lower_t, int transpose_t, int unit, cudaStream_t s)
{
    return launch_trsm_panel_impl<float>(B, vstride, estride, nvec, A, lda, a_trans, k0, pw,
                                         lower_t, transpose_t, unit, s);
}

}  // namespace gfip
