// Throughput of the arithmetic primitives the pair kernel is built from, on
// the GPU it runs on: operations per SM per clock.
//
// Each thread advances 8 independent chains for ITERS steps; each step
// applies the primitive once and feeds its result back, so nothing folds
// away.  The grid is SMs x 8 blocks x 256 threads.  The SM clock during a
// run is measured in the kernel (clock64 against globaltimer on one thread
// per block).  Build and run with `python -m paper_2004_04071_gb300.probe_primitives`.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#include "csrc/mlkd_device.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 2048;
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;

struct Clock {
    unsigned long long cycles, ns;
};

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// OP: 0 fmaf, 1 expf, 2 __expf, 3 expm1f, 4 logf, 5 __logf, 6 sincospif,
// 7 sqrtf, 8 rsqrtf, 9 x / y, 10 f32 -> u32 -> f32, 11 f32 -> i32,
// 12 umulhi + mul (one Philox multiply), 13 floorf, 14 double fma,
// 15 log_unit24, 16 sincos_2pi_unit24, 17 the integer step feeding 15/16 alone
template <int OP>
__global__ void __launch_bounds__(kThreads) probe(float *out, Clock *clk, float seed)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long c0 = 0, t0 = 0;
    if (threadIdx.x == 0) {
        c0 = clock64();
        t0 = globaltimer();
    }
    float x[kChains];
    uint32_t w[kChains];
    double d[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
        x[j] = 0.75f + 0.01f * (float)j + seed * (float)(tid & 7);
        w[j] = 2654435761u * (uint32_t)(tid * kChains + j + 1);
        d[j] = (double)x[j];
    }
#pragma unroll 1
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) {
            if (OP == 0) x[j] = fmaf(x[j], 0.999f, 0.001f);
            if (OP == 1) x[j] = expf(x[j]) * 0.3f;
            if (OP == 2) x[j] = __expf(x[j]) * 0.3f;
            if (OP == 3) x[j] = expm1f(x[j]) * 0.2f + 0.3f;
            if (OP == 4) x[j] = logf(x[j]) + 1.5f;
            if (OP == 5) x[j] = __logf(x[j]) + 1.5f;
            if (OP == 6) {
                float s, c;
                sincospif(x[j], &s, &c);
                x[j] = s + c + 1.5f;
            }
            if (OP == 7) x[j] = sqrtf(x[j]) + 0.5f;
            if (OP == 8) x[j] = rsqrtf(x[j]) + 0.5f;
            if (OP == 9) x[j] = 1.0f / x[j] + 0.5f;
            if (OP == 10) x[j] = (float)(uint32_t)(x[j] * 1048576.0f) * 9.5367431640625e-07f + 0.25f;
            if (OP == 11) x[j] = __int_as_float((int)x[j] ^ 0x3f400000);
            if (OP == 12) w[j] = __umulhi(w[j], 0xD2511F53u) ^ (w[j] * 0xCD9E8D57u) ^ 0x9E3779B9u;
            if (OP == 13) x[j] = floorf(x[j] * 7.3f) * 0.137f + 0.5f;
            if (OP == 14) d[j] = fma(d[j], 0.999, 0.001);
            if (OP == 15) w[j] = w[j] * 1664525u + 1013904223u + __float_as_uint(mlkd::log_unit24(w[j]));
            if (OP == 16) {
                float s, c;
                mlkd::sincos_2pi_unit24(w[j], &s, &c);
                w[j] = w[j] * 1664525u + 1013904223u + __float_as_uint(s + c);
            }
            if (OP == 17) w[j] = w[j] * 1664525u + 1013904223u + (w[j] >> 7);
        }
    }
    float acc = 0.0f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) acc += x[j] + (float)w[j] + (float)d[j];
    out[tid] = acc;
    if (threadIdx.x == 0) {
        clk[blockIdx.x].cycles = clock64() - c0;
        clk[blockIdx.x].ns = globaltimer() - t0;
    }
}

template <int OP>
void run(const char *name, int sms, float *out, Clock *clk, Clock *hclk)
{
    const int blocks = sms * kBlocksPerSM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    probe<OP><<<blocks, kThreads>>>(out, clk, 1e-3f);        // warm-up
    cudaEventRecord(e0);
    probe<OP><<<blocks, kThreads>>>(out, clk, 2e-3f);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaMemcpy(hclk, clk, sizeof(Clock) * blocks, cudaMemcpyDeviceToHost);
    double mhz = 0.0;
    for (int b = 0; b < blocks; ++b) mhz += (double)hclk[b].cycles / (double)hclk[b].ns * 1e3;
    mhz /= blocks;
    const double ops = (double)blocks * kThreads * kChains * kIters;
    const double per_clk_sm = ops / (ms * 1e-3) / (mhz * 1e6) / sms;
    printf("%-28s %9.3f ms  %7.0f MHz  %8.2f ops/clk/SM\n", name, ms, mhz, per_clk_sm);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

}  // namespace

int main()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * kBlocksPerSM;
    float *out = nullptr;
    Clock *clk = nullptr;
    if (cudaMalloc(&out, sizeof(float) * (size_t)blocks * kThreads) != cudaSuccess ||
        cudaMalloc(&clk, sizeof(Clock) * (size_t)blocks) != cudaSuccess) {
        printf("allocation failed\n");
        return 1;
    }
    Clock *hclk = new Clock[blocks];
    printf("%d SMs, %d blocks of %d threads, %d chains x %d steps per thread\n", sms, blocks,
           kThreads, kChains, kIters);
    run<0>("fmaf", sms, out, clk, hclk);
    run<1>("expf", sms, out, clk, hclk);
    run<2>("__expf", sms, out, clk, hclk);
    run<3>("expm1f", sms, out, clk, hclk);
    run<4>("logf", sms, out, clk, hclk);
    run<5>("__logf", sms, out, clk, hclk);
    run<6>("sincospif", sms, out, clk, hclk);
    run<7>("sqrtf", sms, out, clk, hclk);
    run<8>("rsqrtf", sms, out, clk, hclk);
    run<9>("1/x (IEEE division)", sms, out, clk, hclk);
    run<10>("f32 -> u32 -> f32", sms, out, clk, hclk);
    run<11>("f32 -> i32", sms, out, clk, hclk);
    run<12>("umulhi + mul (Philox)", sms, out, clk, hclk);
    run<13>("floorf", sms, out, clk, hclk);
    run<14>("double fma", sms, out, clk, hclk);
    run<15>("log_unit24 + LCG step", sms, out, clk, hclk);
    run<16>("sincos_2pi_unit24 + LCG", sms, out, clk, hclk);
    run<17>("LCG step alone", sms, out, clk, hclk);
    const cudaError_t e = cudaDeviceSynchronize();
    printf("status: %s\n", cudaGetErrorString(e));
    delete[] hclk;
    cudaFree(out);
    cudaFree(clk);
    return e == cudaSuccess ? 0 : 1;
}
