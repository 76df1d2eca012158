// tcgen05.mma issue-rate microbenchmark (measurement support): in each CTA
// lane 0 of each of `issuers` warps issues `count` MMAs of kind::f16 (BF16
// operands, FP32 accumulate, K = 16) with the given M and N from K-major
// shared-memory operands without swizzle, into its own `nacc` accumulators in
// turn, then commits to its own barrier; the clock from the first issue to the
// last commit's completion gives cycles per MMA.  With several
// CTAs per SM, each CTA records its SM and its start and end clocks (the SM's
// own counter), so that the MMAs one SM completed per cycle can be counted
// whatever the placement.  Operands are all 1.0 (their values do not matter
// for timing).  Limits checked on the host: M 64 or 128, N a multiple of 16
// from 16 to 256, nacc N <= the TMEM columns a CTA allocates (a power of two
// from 32 to 512; at most 128 when several CTAs share an SM, which 64 KB of
// shared memory per CTA caps at three; issuers nacc N in all), so every address an MMA forms stays in
// the 64 KB of shared memory (A at 0 reaches < 5 KB, B at 32 KB < 9 KB) and in
// the CTA's TMEM.  A CTA that finds no free TMEM columns waits in the
// allocation until another CTA on its SM has freed them.
#include <algorithm>
#include <array>
#include <cstdint>
#include <map>
#include <vector>

#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ uint32_t s_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t mdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__global__ void __launch_bounds__(128) rate_kernel(int M, int N, int count, int nacc, int issuers, uint32_t cols,
                                                   long long *out)
{
    // 64 KB: [0, 32 KB) A, [32 KB, 64 KB - 128) B; then 4 barriers, 8 clock stamps, the TMEM address
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 65536 - 128);
    long long *stamp = reinterpret_cast<long long *>(smem + 65536 - 96);
    uint32_t *slot = reinterpret_cast<uint32_t *>(smem + 65536 - 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < (65536 - 128) / 4; i += blockDim.x) reinterpret_cast<uint32_t *>(smem)[i] = 0x3f803f80u;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(slot)), "r"(cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid < 4) asm volatile("mbarrier.init.shared.b64 [%0], %1;" ::"r"(s_addr(bar + tid)), "r"(1));
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *slot;
    // issuer warps: lane 0 of warps 0 .. issuers - 1, each into its own accumulators
    if (warp < issuers && lane == 0) {
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
                               ((uint32_t)(M >> 4) << 24);
        const uint32_t base = s_addr(smem);
        const uint64_t da = mdesc(base, 2048, 128), db = mdesc(base + 32768, 4096, 128);
        const uint32_t d0 = tmem + (uint32_t)(warp * nacc * N);
        const long long t0 = clock64();
        for (int j = 0; j < count; ++j) {
            const uint32_t d = d0 + (uint32_t)((j % nacc) * N);
            const uint32_t acc = j >= nacc ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::
                    "r"(d),
                "l"(da), "l"(db), "r"(idesc), "r"(acc)
                : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         s_addr(bar + warp))
                     : "memory");
        uint32_t ok = 0;
        for (int it = 0; it < (1 << 24) && !ok; ++it)
            asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
                         : "=r"(ok)
                         : "r"(s_addr(bar + warp)), "r"(0), "r"(256)
                         : "memory");
        stamp[2 * warp] = t0;
        stamp[2 * warp + 1] = ok ? clock64() : -1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
        long long t0 = stamp[0], t1 = stamp[1];
        bool ok = t1 >= 0;
        for (int k = 1; k < issuers; ++k) {
            t0 = min(t0, stamp[2 * k]);
            t1 = max(t1, stamp[2 * k + 1]);
            ok = ok && stamp[2 * k + 1] >= 0;
        }
        uint32_t smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        long long *o = out + 4 * blockIdx.x;
        o[0] = t0;
        o[1] = t1;
        o[2] = (long long)smid;
        o[3] = ok ? 1 : 0;
    }
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
}

}  // namespace

// Cycles per MMA for the shape (M, N) over `count` MMAs per issuer into `nacc`
// accumulators each, second launch of two, with `ctas` CTAs of `issuers`
// issuing warps and `cols` TMEM columns: the median over the SMs that ran CTAs
// of (cycles from the SM's first issue to its last completion) / (MMAs the
// SM's CTAs issued).  *per_cta (optional): the
// median over CTAs of their own cycles per MMA.  -1: arguments out of the
// checked limits; 1e9 + a CUDA error code on failure; 3e9: a commit's wait
// gave up.
extern "C" double tc_rate_sm(int M, int N, int count, int nacc, int issuers, int ctas, int cols, double *per_cta)
{
    const bool pow2 = cols >= 32 && cols <= 512 && (cols & (cols - 1)) == 0;
    if ((M != 64 && M != 128) || N < 16 || N > 256 || N % 16 || nacc < 1 || issuers < 1 || issuers > 4 || !pow2 ||
        issuers * nacc * N > cols || count < 1 || ctas < 1 || ctas > 4096 || (ctas > 1 && cols > 128))
        return -1.0;
    const size_t nb = sizeof(long long) * 4 * (size_t)ctas;
    long long *d = nullptr;
    if (cudaMalloc(&d, nb) != cudaSuccess) return 2.0e9;
    cudaError_t e = cudaFuncSetAttribute(rate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536);
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        rate_kernel<<<ctas, 128, 65536>>>(M, N, count, nacc, issuers, (uint32_t)cols, d);
        e = cudaDeviceSynchronize();
    }
    std::vector<long long> h(4 * (size_t)ctas, 0);
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), d, nb, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return 1.0e9 + (double)e;
    std::map<long long, std::array<long long, 3>> sm;  // smid -> first start, last end, CTAs
    std::vector<double> cta;
    for (int b = 0; b < ctas; ++b) {
        const long long *o = &h[4 * (size_t)b];
        if (!o[3]) return 3.0e9;
        cta.push_back((double)(o[1] - o[0]) / ((double)count * issuers));
        auto it = sm.find(o[2]);
        if (it == sm.end()) sm[o[2]] = {o[0], o[1], 1};
        else {
            it->second[0] = std::min(it->second[0], o[0]);
            it->second[1] = std::max(it->second[1], o[1]);
            it->second[2] += 1;
        }
    }
    std::vector<double> per_sm;
    for (const auto &kv : sm)
        per_sm.push_back((double)(kv.second[1] - kv.second[0]) / ((double)count * issuers * kv.second[2]));
    std::sort(per_sm.begin(), per_sm.end());
    std::sort(cta.begin(), cta.end());
    if (per_cta) *per_cta = cta[cta.size() / 2];
    return per_sm[per_sm.size() / 2];
}

// One CTA on one SM: cycles per MMA (see tc_rate_sm).
extern "C" double tc_rate_cycles(int M, int N, int count, int nacc)
{
    return tc_rate_sm(M, N, count, nacc, 1, 1, 512, nullptr);
}
