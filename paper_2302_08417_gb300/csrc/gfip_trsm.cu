// gfip_trsm.cu -- the panel solves of the blocked triangular solve (TRSM).
//
// TRSM runs as a sequence over panels of op(A)'s diagonal (see gfip_api.cu): each step solves
// one panel of at most TRSM_PANEL unknowns for every right-hand side with the kernel below,
// then the fused GEMM kernel subtracts the panel's contribution from the unknowns still to be
// solved.  The kernel solves a panel by column-oriented substitution: once unknown d is known
// (divided by its diagonal entry), every unknown below it loses its multiple at once; per
// chunk of columns the chain updates only its own 32-row group, and the later groups are
// updated afterwards, off the chain.  A warp holds one right-hand side, one element per lane
// and 32-row group, in registers; the panel's triangle streams through shared memory in
// chunks of columns, double-buffered and shared by the CTA's warps, the next chunk loaded
// into registers while this one is solved.  Only the entries a triangular solve reads are
// read: never the other triangle, nor a unit diagonal.
#include <cstdint>

#include "gfip_internal.h"

namespace gfip {
namespace trsm {

// One right-hand side per warp: a warp's substitution chain is as short as it gets, and the
// CTA's warps interleave their chains (two per warp, 8 warps a CTA, measured 11 % slower at
// 2048 x 2048 in FP32).
// FP32 CTAs run 16 warps.  FP64, bound by its DFMA pipe, runs between 8 and 16, as many as
// spread the right-hand sides over all SMs (2048 of them on 152 SMs: 14 a CTA, 147 CTAs,
// 11 % faster than 16 a CTA on 128 SMs; the same shape made FP32 5 % slower).
#ifndef GFIP_TRSM_RPW
#define GFIP_TRSM_RPW 1
#endif
constexpr int RPW = GFIP_TRSM_RPW;   // (overridable at build time for measurements)
constexpr int MIN_WARPS = 8 / RPW, MAX_WARPS = 16 / RPW;
// loads a staging part takes a thread: one with 16 warps, two with fewer (the kernel is
// compiled for both)
constexpr int MAX_SLOTS = TRSM_PANEL / (MIN_WARPS * 32);
constexpr int ROWS = TRSM_PANEL / 32;     // 32-row groups of a panel: registers per vector
constexpr int CW = 16;                    // triangle columns per staged chunk
constexpr size_t BUF = (size_t)CW * TRSM_PANEL;   // elements of one chunk buffer
static_assert(TRSM_PANEL % 32 == 0 && 32 % CW == 0, "a 32-row group is whole chunks");
static_assert(ROWS == 16, "the group update below is written out for 16 groups");
// two chunk buffers, two diagonals and two reciprocal diagonals
template <typename T> constexpr size_t smem_bytes() { return sizeof(T) * (2 * BUF + 4 * CW); }

// The panel's system in solve order: unknown q of the local lower triangular system is row
// lower_t ? q : pw - 1 - q of the block, so an upper triangular block is solved by the same
// forward loop.  t(r, c) = op(A)[k0 + r, k0 + c] (side 'L') or op(A)[k0 + c, k0 + r] (side
// 'R', transpose_t), op(A)[i, j] = A[i + j lda] ('N') or A[j + i lda] ('T').  Every case is
// linear in (q, d): t(q, d) sits at A[o0 + sgn (q cq + d cd)], the four numbers set on the
// host (launch_trsm_panel).
struct Panel {
    const void *A;
    int64_t o0, cq, cd;
    int sgn;            // +1 lower, -1 upper (rows counted from the block's end)
    int lower_t, unit;
    int k0, pw;
    __device__ __forceinline__ int row(int q) const { return lower_t ? q : pw - 1 - q; }
    template <typename T> __device__ __forceinline__ const T *at(int q, int d) const
    {
        return static_cast<const T *>(A) + o0 + sgn * ((int64_t)q * cq + (int64_t)d * cd);
    }
    // along q the copies run along memory (|cq| == 1)
    __device__ __forceinline__ bool along_q() const { return cq == 1; }
};

// Staging of chunk [d0, d0 + CW) of the strictly lower part of the local system:
// buf[dd * TRSM_PANEL + q] = t(q, d0 + dd) for q > d0 + dd, zero elsewhere (rows from the
// chunk's 32-row group on), and its diagonal (unless unit).  A chunk is CW parts: where A is
// contiguous along q a part is one column of the chunk, otherwise a slice of its rows, so
// that a warp's loads are consecutive in A either way; a part is at most SLOTS elements per
// thread.  Plain loads into registers, issued a chunk ahead and stored to shared memory
// after the work they hide behind (element copies through cp.async cost more issue slots).
constexpr int HALF = CW / 2;   // parts loaded together
template <typename T, int SLOTS> struct Stage {
    T v[HALF][SLOTS];
    T diag;
};

template <typename T>
__device__ __forceinline__ void stage_slot(const Panel &p, int d0, int part, int i, int tid,
                                           int &q, int &dd)
{
    const int qlo = d0 & ~31, qhi = (p.pw + 31) & ~31;
    const int e = tid + blockDim.x * i;
    if (p.along_q()) {
        dd = part;
        q = qlo + e;
        if (q >= qhi) q = -1;
    } else {
        const int rows = (qhi - qlo) / CW;
        dd = e % CW;
        const int qo = e / CW;
        q = qo < rows ? qlo + part * rows + qo : -1;
    }
}

template <typename T, int SLOTS>
__device__ __forceinline__ void stage_load(const Panel &p, int d0, int part0, int tid,
                                           Stage<T, SLOTS> &st)
{
#pragma unroll
    for (int k = 0; k < HALF; ++k)
#pragma unroll
        for (int i = 0; i < SLOTS; ++i) {
            int q, dd;
            stage_slot<T>(p, d0, part0 + k, i, tid, q, dd);
            const int d = d0 + dd;
            st.v[k][i] = (q > d && q < p.pw) ? *p.at<T>(q, d) : T(0);
        }
    if (part0 == 0 && tid < CW) {
        const int d = d0 + tid;
        st.diag = (!p.unit && d < p.pw) ? *p.at<T>(d, d) : T(1);
    }
}

template <typename T, int SLOTS>
__device__ __forceinline__ void stage_store(const Panel &p, int d0, int part0, int tid,
                                            const Stage<T, SLOTS> &st, T *buf, T *dg)
{
#pragma unroll
    for (int k = 0; k < HALF; ++k)
#pragma unroll
        for (int i = 0; i < SLOTS; ++i) {
            int q, dd;
            stage_slot<T>(p, d0, part0 + k, i, tid, q, dd);
            if (q >= 0) buf[dd * TRSM_PANEL + q] = st.v[k][i];
        }
    if (part0 == 0 && tid < CW) dg[tid] = st.diag;
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
// this lane's element of group R of every right-hand side (col = the chunk's staged column 0
// at the group's first row).
template <typename T, int R, int RPW>
__device__ __forceinline__ void update_group(T (&b)[ROWS][RPW], const T *col,
                                             const T (&x)[CW][RPW])
{
#pragma unroll
    for (int dd = 0; dd < CW; ++dd) {
        const T tq = col[dd * TRSM_PANEL];
#pragma unroll
        for (int w = 0; w < RPW; ++w) b[R][w] = fma(-tq, x[dd][w], b[R][w]);
    }
}

template <typename T, int SLOTS>
__global__ void __launch_bounds__(MAX_WARPS * 32, 1)
    panel_kernel(T *B, int64_t vstride, int64_t estride, int nvec, const Panel p)
{
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
        stage_store<T, SLOTS>(p, 0, 0, tid, st, bufs, dgs);
        stage_load<T, SLOTS>(p, 0, HALF, tid, st);
        stage_store<T, SLOTS>(p, 0, HALF, tid, st, bufs, dgs);
    }
    // The groups run in a loop, not unrolled (the code stays small enough for the instruction
    // cache): the group being solved moves into cur[] and back; the later groups are
    // updated in an unrolled loop over all groups, skipping the ones not after it.
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
#pragma unroll 1
        for (int h = 0; h < 32 / CW; ++h) {
            const int d0 = 32 * r + h * CW;
            if (d0 >= pw) break;
            __syncthreads();      // chunk ch is in shared memory
            const T *tb = bufs + (ch & 1) * BUF;
            const T *dg = dgs + (ch & 1) * CW;
            T *dr = drs + (ch & 1) * CW;
            if (tid < CW) dr[tid] = p.unit ? T(1) : T(1) / dg[tid];
            __syncthreads();
            const bool more = d0 + CW < pw;   // a next chunk to stage meanwhile
            T *nbuf = bufs + ((ch + 1) & 1) * BUF;
            T *ndg = dgs + ((ch + 1) & 1) * CW;
            Stage<T, SLOTS> st;
            if (more) stage_load<T, SLOTS>(p, d0 + CW, 0, tid, st);
            const int dn = min(CW, pw - d0);
            // the chunk's unknowns one after another; each updates only the later unknowns
            // of its own 32-row group here (the chain's latency is the solve's floor)
            for (int dd = 0; dd < dn; ++dd) {
                const int owner = h * CW + dd;   // the lane holding unknown d0 + dd
                const T t = dg[dd], rt = dr[dd];
                const T tq = tb[dd * TRSM_PANEL + 32 * r + lane];
#pragma unroll
                for (int w = 0; w < RPW; ++w) {
                    T bc = cur[w];
                    if (!p.unit && lane == owner) bc = quotient(bc, t, rt);
                    const T x = __shfl_sync(0xffffffffu, bc, owner);
                    if (lane == owner) cur[w] = x;
                    if (lane > owner) cur[w] = fma(-tq, x, cur[w]);
                }
            }
            if (more) {
                stage_store<T, SLOTS>(p, d0 + CW, 0, tid, st, nbuf, ndg);
                stage_load<T, SLOTS>(p, d0 + CW, HALF, tid, st);
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
            const T *col = tb + lane;
            switch (r) {
#define GFIP_TRSM_GROUP(R)                                                                  \
    case R - 1:                                                                             \
        if (32 * R < pw) update_group<T, R, RPW>(b, col + 32 * R, xs);                     \
        [[fallthrough]];
                GFIP_TRSM_GROUP(1) GFIP_TRSM_GROUP(2) GFIP_TRSM_GROUP(3)
                GFIP_TRSM_GROUP(4) GFIP_TRSM_GROUP(5) GFIP_TRSM_GROUP(6)
                GFIP_TRSM_GROUP(7) GFIP_TRSM_GROUP(8) GFIP_TRSM_GROUP(9)
                GFIP_TRSM_GROUP(10) GFIP_TRSM_GROUP(11) GFIP_TRSM_GROUP(12)
                GFIP_TRSM_GROUP(13) GFIP_TRSM_GROUP(14) GFIP_TRSM_GROUP(15)
#undef GFIP_TRSM_GROUP
            default: break;
            }
            if (more) stage_store<T, SLOTS>(p, d0 + CW, HALF, tid, st, nbuf, ndg);
            __syncthreads();   // this buffer is restaged during the next chunk
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
    static bool configured = false;
    if (!configured) {
        for (auto *k : {trsm::panel_kernel<T, 1>, trsm::panel_kernel<T, 2>,
                        trsm::panel_kernel<T, trsm::MAX_SLOTS>}) {
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
    p.cq = transpose_t ? cj : ci;
    p.cd = transpose_t ? ci : cj;
    p.sgn = lower_t ? 1 : -1;
    p.o0 = (int64_t)(k0 + (lower_t ? 0 : pw - 1)) * (p.cq + p.cd);
    p.A = A;
    p.lower_t = lower_t;
    p.unit = unit;
    p.k0 = k0;
    p.pw = pw;
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    const int want = (nvec + sms * trsm::RPW - 1) / (sms * trsm::RPW);
    const int warps = sizeof(T) == 4 ? trsm::MAX_WARPS
                      : want < trsm::MIN_WARPS
                          ? trsm::MIN_WARPS
                          : (want > trsm::MAX_WARPS ? trsm::MAX_WARPS : want);
    const int rpc = warps * trsm::RPW;
    const int blocks = (nvec + rpc - 1) / rpc;
    if (warps * 32 >= TRSM_PANEL)
        trsm::panel_kernel<T, 1><<<blocks, warps * 32, trsm::smem_bytes<T>(), s>>>(
            B, vstride, estride, nvec, p);
    else if (warps * 64 >= TRSM_PANEL)
        trsm::panel_kernel<T, 2><<<blocks, warps * 32, trsm::smem_bytes<T>(), s>>>(
            B, vstride, estride, nvec, p);
    else
        trsm::panel_kernel<T, trsm::MAX_SLOTS><<<blocks, warps * 32, trsm::smem_bytes<T>(), s>>>(
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
