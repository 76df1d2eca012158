// FP32 FMA-throughput microbenchmark: the measured peak of the CUDA-core FP32
// pipe that the FP32 correlation pass is reported against (the ALU roofline).
// Every thread runs 16 independent FMA chains (enough in flight to cover the
// pipe's latency at full occupancy); the launch fills every SM with 8 CTAs of
// 256 threads.  A second kernel runs the chains as packed pairs (fma.rn.f32x2,
// two FMAs per instruction), which the paired plane loop of the pass uses: the
// peak is the faster of the two.  Measurement support, built as its own small
// library.
#include <cstdio>

#include <cuda_runtime.h>

namespace {

constexpr int kChains = 16;

__global__ void __launch_bounds__(256) fma_kernel(float *out, int iters, float x, float y)
{
    float a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = (float)threadIdx.x * 1e-3f + (float)j;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = fmaf(a[j], x, y);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == -1.f) out[blockIdx.x] = s;  // keeps the chains live; never true for these inputs
}

// The same chains as packed pairs: fma.rn.f32x2, two FMAs per instruction.
__global__ void __launch_bounds__(256) fma2_kernel(float *out, int iters, float x, float y)
{
    unsigned long long a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
        const float lo = (float)threadIdx.x * 1e-3f + (float)j, hi = lo + 0.5f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(a[j]) : "f"(lo), "f"(hi));
    }
    unsigned long long x2, y2;
    asm("mov.b64 %0, {%1, %1};" : "=l"(x2) : "f"(x));
    asm("mov.b64 %0, {%1, %1};" : "=l"(y2) : "f"(y));
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[j]) : "l"(x2), "l"(y2));
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j)
        s += __uint_as_float((unsigned)a[j]) + __uint_as_float((unsigned)(a[j] >> 32));
    if (s == -1.f) out[blockIdx.x] = s;  // keeps the chains live; never true for these inputs
}

}  // namespace

// Runs the kernel `reps` times on `stream` (after one warm-up launch) and
// returns the shortest launch in *best_ms and the FP32 flops of one launch in
// *flops (2 per FMA).  Returns 0, or a CUDA error code.
extern "C" int fma_peak_run2(int blocks_per_sm, int iters, int reps, int packed, float *best_ms, double *flops,
                             void *stream)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    const int blocks = sms * blocks_per_sm;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaMalloc(&out, sizeof(float) * blocks)) != cudaSuccess) return (int)e;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    auto launch = [&] {
        if (packed) fma2_kernel<<<blocks, 256, 0, st>>>(out, iters, 0.999999f, 1e-6f);
        else fma_kernel<<<blocks, 256, 0, st>>>(out, iters, 0.999999f, 1e-6f);
    };
    launch();
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        cudaEventRecord(e0, st);
        launch();
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best) best = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    *best_ms = best;
    *flops = 2.0 * kChains * (double)iters * 256.0 * (double)blocks * (packed ? 2.0 : 1.0);
    return (int)e;
}

// Scalar FMA chains (fma_peak_run2 with packed = 0).
extern "C" int fma_peak_run(int blocks_per_sm, int iters, int reps, float *best_ms, double *flops, void *stream)
{
    return fma_peak_run2(blocks_per_sm, iters, reps, 0, best_ms, flops, stream);
}
