// peak_probe.cu -- measures the arithmetic peaks the GEMM roofline is taken against:
// FP64 DFMA, FP64 mma.sync (DMMA) shapes, FP32 FFMA, and the SM clock seen meanwhile.
// Prints one JSON object on stdout.  Standalone executable; not part of the library.
//
// Each kernel runs independent multiply-add chains (no memory traffic in the timed loop)
// and writes one value per thread at the end so the compiler keeps the arithmetic.
#include <cstdio>
#include <cstdlib>
#include <cuda_runtime.h>

#define CK(x)                                                                          \
    do {                                                                               \
        cudaError_t e_ = (x);                                                          \
        if (e_ != cudaSuccess) {                                                       \
            fprintf(stderr, "CUDA error %s at %s:%d\n", cudaGetErrorString(e_), __FILE__, \
                    __LINE__);                                                         \
            exit(1);                                                                   \
        }                                                                              \
    } while (0)

constexpr int CHAINS = 16;

__device__ __forceinline__ void span_mark(int which);

__global__ void dfma_kernel(double *out, int iters, double a, double b)
{
    span_mark(0);
    double acc[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) acc[c] = threadIdx.x * 1e-9 + c;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) acc[c] = fma(acc[c], a, b);
    }
    double s = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += acc[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    span_mark(1);
}

__global__ void ffma_kernel(float *out, int iters, float a, float b)
{
    float acc[CHAINS * 2];
#pragma unroll
    for (int c = 0; c < CHAINS * 2; ++c) acc[c] = threadIdx.x * 1e-6f + c;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < CHAINS * 2; ++c) acc[c] = fmaf(acc[c], a, b);
    }
    float s = 0;
#pragma unroll
    for (int c = 0; c < CHAINS * 2; ++c) s += acc[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// mma.sync m8n8k4 f64: A 8x4 (1 elem/thread), B 4x8 (1 elem/thread), C 8x8 (2 elems/thread)
__global__ void dmma_m8n8k4_kernel(double *out, int iters, double a, double b)
{
    double acc[4][2];
#pragma unroll
    for (int c = 0; c < 4; ++c) { acc[c][0] = threadIdx.x; acc[c][1] = c; }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 "
                         "{%0, %1}, {%2}, {%3}, {%0, %1};\n"
                         : "+d"(acc[c][0]), "+d"(acc[c][1])
                         : "d"(a), "d"(b));
        }
    }
    double s = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) s += acc[c][0] + acc[c][1];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// mma.sync m16n8k4 f64: A 16x4 (2/thread), B 4x8 (1/thread), C 16x8 (4/thread)
__global__ void dmma_m16n8k4_kernel(double *out, int iters, double a, double b)
{
    double acc[4][4];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[c][r] = threadIdx.x + r + c;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            asm volatile("mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 "
                         "{%0, %1, %2, %3}, {%4, %5}, {%6}, {%0, %1, %2, %3};\n"
                         : "+d"(acc[c][0]), "+d"(acc[c][1]), "+d"(acc[c][2]), "+d"(acc[c][3])
                         : "d"(a), "d"(b), "d"(b));
        }
    }
    double s = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) s += acc[c][0] + acc[c][1] + acc[c][2] + acc[c][3];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// mma.sync m16n8k16 f64: A 16x16 (8/thread), B 16x8 (4/thread), C 16x8 (4/thread)
__global__ void dmma_m16n8k16_kernel(double *out, int iters, double a, double b)
{
    double acc[2][4];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[c][r] = threadIdx.x + r + c;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            asm volatile("mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 "
                         "{%0, %1, %2, %3}, {%4, %5, %6, %7, %8, %9, %10, %11}, "
                         "{%12, %13, %14, %15}, {%0, %1, %2, %3};\n"
                         : "+d"(acc[c][0]), "+d"(acc[c][1]), "+d"(acc[c][2]), "+d"(acc[c][3])
                         : "d"(a), "d"(a), "d"(a), "d"(a), "d"(a), "d"(a), "d"(a), "d"(a),
                           "d"(b), "d"(b), "d"(b), "d"(b));
        }
    }
    double s = 0;
#pragma unroll
    for (int c = 0; c < 2; ++c) s += acc[c][0] + acc[c][1] + acc[c][2] + acc[c][3];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Thread 0 of block 0 records %clock64 and %globaltimer at its start and end, so that each
// rate can be put against the SM clock it actually ran at.
__device__ unsigned long long g_span[4];
__device__ __forceinline__ void span_mark(int which)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        g_span[2 * which] = clock64();
        g_span[2 * which + 1] = t;
    }
}

// FP64 work of two kinds in one loop: ND independent DFMA chains per thread and NM
// independent m8n8k4 DMMA chains per warp.  With both, the time shows whether the two share
// one pipe (times add) or run on separate ones (the longer one hides the other).  SPLIT puts
// the DFMA chains on even warps and the DMMA chains on odd ones instead.
template <int ND, int NM, bool SPLIT>
__global__ void fp64_mix_kernel(double *out, int iters, double a, double b)
{
    span_mark(0);
    const bool do_d = !SPLIT || ((threadIdx.x >> 5) & 1) == 0;
    const bool do_m = !SPLIT || ((threadIdx.x >> 5) & 1) == 1;
    double acc[ND > 0 ? ND : 1];
    double macc[NM > 0 ? NM : 1][2];
#pragma unroll
    for (int c = 0; c < (ND > 0 ? ND : 1); ++c) acc[c] = threadIdx.x * 1e-9 + c;
#pragma unroll
    for (int c = 0; c < (NM > 0 ? NM : 1); ++c) { macc[c][0] = threadIdx.x; macc[c][1] = c; }
    if (do_d && ND > 0) {
        if (!SPLIT && NM > 0) {
            for (int it = 0; it < iters; ++it) {
#pragma unroll
                for (int c = 0; c < ND; ++c) acc[c] = fma(acc[c], a, b);
#pragma unroll
                for (int c = 0; c < NM; ++c)
                    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 "
                                 "{%0, %1}, {%2}, {%3}, {%0, %1};\n"
                                 : "+d"(macc[c][0]), "+d"(macc[c][1])
                                 : "d"(a), "d"(b));
            }
        } else {
            for (int it = 0; it < iters; ++it) {
#pragma unroll
                for (int c = 0; c < ND; ++c) acc[c] = fma(acc[c], a, b);
            }
        }
    } else if (do_m && NM > 0) {
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int c = 0; c < NM; ++c)
                asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 "
                             "{%0, %1}, {%2}, {%3}, {%0, %1};\n"
                             : "+d"(macc[c][0]), "+d"(macc[c][1])
                             : "d"(a), "d"(b));
        }
    }
    double s = 0;
#pragma unroll
    for (int c = 0; c < (ND > 0 ? ND : 1); ++c) s += acc[c];
#pragma unroll
    for (int c = 0; c < (NM > 0 ? NM : 1); ++c) s += macc[c][0] + macc[c][1];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    span_mark(1);
}

// Reads %clock64 and %globaltimer across a busy loop to estimate the SM clock.
__global__ void clock_kernel(unsigned long long *out, int iters, double a)
{
    unsigned long long c0 = clock64(), t0, t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    double x = threadIdx.x;
    for (int i = 0; i < iters; ++i) x = fma(x, a, 1e-9);
    unsigned long long c1 = clock64();
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    if (threadIdx.x == 0) {
        out[2 * blockIdx.x] = c1 - c0;
        out[2 * blockIdx.x + 1] = t1 - t0;
    }
    if (x == 12345.0) out[0] = 0;
}

template <typename K>
static double time_ms(K launch, int reps)
{
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    launch();
    CK(cudaDeviceSynchronize());
    float best = 1e30f;
    for (int r = 0; r < reps; ++r) {
        CK(cudaEventRecord(e0));
        launch();
        CK(cudaEventRecord(e1));
        CK(cudaEventSynchronize(e1));
        float ms;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) best = ms;
    }
    CK(cudaGetLastError());
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

int main(int argc, char **argv)
{
    int dev = 0;
    CK(cudaSetDevice(dev));
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, dev));
    int sms = prop.multiProcessorCount;
    int clk_khz = 0;
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
    int iters = argc > 1 ? atoi(argv[1]) : 4096;

    const int threads = 256;
    const int blocks = sms * 8;
    size_t n = (size_t)blocks * threads;
    double *dout;
    CK(cudaMalloc(&dout, n * sizeof(double) * 2));
    unsigned long long *cout;
    CK(cudaMalloc(&cout, 2 * sizeof(unsigned long long) * sms));

    double dfma_ms = time_ms([&] { dfma_kernel<<<blocks, threads>>>(dout, iters, 1.0000001, 1e-7); }, 5);
    double dfma_tf = 2.0 * CHAINS * (double)iters * n / (dfma_ms * 1e-3) / 1e12;

    double ffma_ms = time_ms([&] { ffma_kernel<<<blocks, threads>>>((float *)dout, iters * 8, 1.0000001f, 1e-7f); }, 5);
    double ffma_tf = 2.0 * CHAINS * 2 * (double)iters * 8 * n / (ffma_ms * 1e-3) / 1e12;

    // warps in flight: blocks*threads/32 ; each mma does 2*M*N*K flops per warp
    double warps = (double)n / 32.0;
    double d884_ms = time_ms([&] { dmma_m8n8k4_kernel<<<blocks, threads>>>(dout, iters, 1.0000001, 1e-7); }, 5);
    double d884_tf = 2.0 * 8 * 8 * 4 * 4.0 * iters * warps / (d884_ms * 1e-3) / 1e12;
    double d1684_ms = time_ms([&] { dmma_m16n8k4_kernel<<<blocks, threads>>>(dout, iters, 1.0000001, 1e-7); }, 5);
    double d1684_tf = 2.0 * 16 * 8 * 4 * 4.0 * iters * warps / (d1684_ms * 1e-3) / 1e12;
    double d16816_ms = time_ms([&] { dmma_m16n8k16_kernel<<<blocks, threads>>>(dout, iters / 4, 1.0000001, 1e-7); }, 5);
    double d16816_tf = 2.0 * 16 * 8 * 16 * 2.0 * (iters / 4) * warps / (d16816_ms * 1e-3) / 1e12;

    // SM clock over the last timed launch, from block 0's first thread (MHz)
    auto span_mhz = [&]() {
        unsigned long long sp[4];
        CK(cudaMemcpyFromSymbol(sp, g_span, sizeof(sp)));
        return sp[3] > sp[1] ? (double)(sp[2] - sp[0]) / (double)(sp[3] - sp[1]) * 1e3 : 0.0;
    };
    // DFMA again, its clock taken from inside the kernel: lanes per clock per SM
    double dfma2_ms = time_ms([&] { dfma_kernel<<<blocks, threads>>>(dout, iters, 1.0000001, 1e-7); }, 5);
    double dfma_mhz = span_mhz();
    double dfma_flops = 2.0 * CHAINS * (double)iters * n;
    double dfma2_tf = dfma_flops / (dfma2_ms * 1e-3) / 1e12;
    double dfma_lanes_per_clk = dfma_flops / 2.0 / (dfma2_ms * 1e-3) / (dfma_mhz * 1e6) / sms;

    // DFMA and DMMA alone and together (16 DFMA chains a thread, 4 DMMA chains a warp)
    const int mit = iters / 2;
    double f_d = 2.0 * 16 * (double)mit * n;                 // DFMA flops of a launch
    double f_m = 2.0 * 8 * 8 * 4 * 4.0 * (double)mit * warps; // DMMA flops of a launch
    double t_d = time_ms([&] { fp64_mix_kernel<16, 0, false><<<blocks, threads>>>(dout, mit, 1.0000001, 1e-7); }, 5);
    double mhz_d = span_mhz();
    double t_m = time_ms([&] { fp64_mix_kernel<0, 4, false><<<blocks, threads>>>(dout, mit, 1.0000001, 1e-7); }, 5);
    double mhz_m = span_mhz();
    double t_dm = time_ms([&] { fp64_mix_kernel<16, 4, false><<<blocks, threads>>>(dout, mit, 1.0000001, 1e-7); }, 5);
    double mhz_dm = span_mhz();
    double t_sp = time_ms([&] { fp64_mix_kernel<16, 4, true><<<blocks, threads>>>(dout, mit, 1.0000001, 1e-7); }, 5);
    double mhz_sp = span_mhz();

    clock_kernel<<<sms, 32>>>(cout, 1 << 22, 1.0000001);
    CK(cudaDeviceSynchronize());
    unsigned long long hc[2];
    CK(cudaMemcpy(hc, cout, sizeof(hc), cudaMemcpyDeviceToHost));
    double sm_mhz = hc[1] ? (double)hc[0] / (double)hc[1] * 1e3 : 0.0;

    printf("{\"sms\": %d, \"l2_bytes\": %d, \"smem_per_block_optin\": %zu, "
           "\"regs_per_sm\": %d, \"clock_attr_mhz\": %.0f, \"sm_mhz_during_probe\": %.0f, "
           "\"dfma_tflops\": %.4f, \"ffma_tflops\": %.3f, \"dmma_m8n8k4_tflops\": %.4f, "
           "\"dmma_m16n8k4_tflops\": %.4f, \"dmma_m16n8k16_tflops\": %.4f, "
           "\"iters\": %d, ",
           sms, prop.l2CacheSize, prop.sharedMemPerBlockOptin, prop.regsPerMultiprocessor,
           clk_khz / 1e3, sm_mhz, dfma_tf, ffma_tf, d884_tf, d1684_tf, d16816_tf, iters);
    printf("\"dfma_in_kernel\": {\"tflops\": %.4f, \"sm_mhz\": %.0f, "
           "\"dfma_lanes_per_clk_per_sm\": %.3f, \"tflops_at_max_clock\": %.4f}, ",
           dfma2_tf, dfma_mhz, dfma_lanes_per_clk,
           dfma_lanes_per_clk * 2.0 * sms * clk_khz * 1e3 / 1e12);
    // "add": the time of both together over the sum of the times alone (1 = one shared pipe,
    // max/sum = independent pipes)
    printf("\"fp64_mix\": {\"dfma_ms\": %.3f, \"dmma_ms\": %.3f, \"both_ms\": %.3f, "
           "\"split_warps_ms\": %.3f, \"dfma_tflops\": %.4f, \"dmma_tflops\": %.4f, "
           "\"both_tflops\": %.4f, \"split_warps_tflops\": %.4f, "
           "\"both_over_sum\": %.3f, \"independent_would_be\": %.3f, "
           "\"sm_mhz\": [%.0f, %.0f, %.0f, %.0f]}}\n",
           t_d, t_m, t_dm, t_sp, f_d / (t_d * 1e-3) / 1e12, f_m / (t_m * 1e-3) / 1e12,
           (f_d + f_m) / (t_dm * 1e-3) / 1e12, (f_d + f_m) / 2.0 / (t_sp * 1e-3) / 1e12,
           t_dm / (t_d + t_m), (t_d > t_m ? t_d : t_m) / (t_d + t_m), mhz_d, mhz_m, mhz_dm,
           mhz_sp);
    cudaFree(dout);
    cudaFree(cout);
    return 0;
}
