// tcgen05.mma issue-rate microbenchmark (measurement support): one CTA, one
// thread issues `count` MMAs of kind::f16 (BF16 operands, FP32 accumulate,
// K = 16) with the given M and N from K-major shared-memory operands without
// swizzle, into `nacc` accumulators in turn, then commits; the clock from the
// first issue to the commit's completion gives cycles per MMA.  Operands are
// all 1.0 (their values do not matter for timing).  Limits checked on the host:
// M 64 or 128, N a multiple of 16 from 16 to 256, nacc N <= 512 (the TMEM
// columns allocated), so every address an MMA forms stays in the 64 KB of
// shared memory (A at 0 reaches < 5 KB, B at 32 KB < 9 KB) and in TMEM.
#include <cstdint>

#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ uint32_t s_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t mdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__global__ void __launch_bounds__(128, 1) rate_kernel(int M, int N, int count, int nacc, long long *out)
{
    extern __shared__ __align__(1024) unsigned char smem[];  // 64 KB: [0, 32 KB) A, [32 KB, 64 KB) B
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 65536 - 16);
    uint32_t *slot = reinterpret_cast<uint32_t *>(smem + 65536 - 8);
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < (65536 - 16) / 4; i += blockDim.x) reinterpret_cast<uint32_t *>(smem)[i] = 0x3f803f80u;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(slot)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) asm volatile("mbarrier.init.shared.b64 [%0], %1;" ::"r"(s_addr(bar)), "r"(1));
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *slot;
    if (tid == 0) {
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
                               ((uint32_t)(M >> 4) << 24);
        const uint32_t base = s_addr(smem);
        const uint64_t da = mdesc(base, 2048, 128), db = mdesc(base + 32768, 4096, 128);
        const long long t0 = clock64();
        for (int j = 0; j < count; ++j) {
            const uint32_t d = tmem + (uint32_t)((j % nacc) * N);
            const uint32_t acc = j >= nacc ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::
                    "r"(d),
                "l"(da), "l"(db), "r"(idesc), "r"(acc)
                : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_addr(bar))
                     : "memory");
        uint32_t ok = 0;
        for (int it = 0; it < (1 << 24) && !ok; ++it)
            asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
                         : "=r"(ok)
                         : "r"(s_addr(bar)), "r"(0), "r"(256)
                         : "memory");
        out[0] = clock64() - t0;
        out[1] = ok;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

}  // namespace

// Cycles per MMA for the shape (M, N) over `count` MMAs into `nacc`
// accumulators (second launch of two); -1: arguments out of the checked
// limits; a positive CUDA error code on failure.
extern "C" double tc_rate_cycles(int M, int N, int count, int nacc)
{
    if ((M != 64 && M != 128) || N < 16 || N > 256 || N % 16 || nacc < 1 || nacc * N > 512 || count < 1)
        return -1.0;
    long long *d = nullptr, h[2] = {0, 0};
    if (cudaMalloc(&d, sizeof(h)) != cudaSuccess) return 2.0e9;
    cudaError_t e = cudaFuncSetAttribute(rate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536);
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        rate_kernel<<<1, 128, 65536>>>(M, N, count, nacc, d);
        e = cudaDeviceSynchronize();
    }
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return 1.0e9 + (double)e;
    if (!h[1]) return 3.0e9;
    return (double)h[0] / (double)count;
}
