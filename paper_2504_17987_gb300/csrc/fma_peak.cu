// FP32 FMA-throughput microbenchmark: the measured peak of the CUDA-core FP32
// pipe that the FP32 correlation pass is reported against (the ALU roofline).
// Every thread runs 16 independent FMA chains (enough in flight to cover the
// pipe's latency at full occupancy); the launch fills every SM with 8 CTAs of
// 256 threads.  Measurement support, built as its own small library.
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

}  // namespace

// Runs the kernel `reps` times on `stream` (after one warm-up launch) and
// returns the shortest launch in *best_ms and the FP32 flops of one launch in
// *flops (2 per FMA).  Returns 0, or a CUDA error code.
extern "C" int fma_peak_run(int blocks_per_sm, int iters, int reps, float *best_ms, double *flops, void *stream)
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
    fma_kernel<<<blocks, 256, 0, st>>>(out, iters, 0.999999f, 1e-6f);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        cudaEventRecord(e0, st);
        fma_kernel<<<blocks, 256, 0, st>>>(out, iters, 0.999999f, 1e-6f);
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
    *flops = 2.0 * kChains * (double)iters * 256.0 * (double)blocks;
    return (int)e;
}
