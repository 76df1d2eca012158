// BF16 tensor-core (mma.sync m16n8k16, k8 for 8 px blocks, FP32 accumulate)
// instantiations of the fused correlation pass.
#include "pass_impl.cuh"

namespace rpiv {

template <int RC, int GC = 0>
static cudaError_t go_bf16(const PassArgs &a, dim3 grid, int smem, cudaStream_t st)
{
    pass_kernel<RC, PREC_BF16, GC><<<grid, PASS_THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

// 50 % overlap with 8-, 16- and 32-px blocks at r = 4: specialised shapes
static cudaError_t go_bf16_r4(const PassArgs &a, dim3 grid, int smem, cudaStream_t st)
{
    const int G = a.plan.G;
    if (a.w == 2 * G && a.s == G) {
        if (G == 8) return go_bf16<4, 8>(a, grid, smem, st);
        if (G == 16) return go_bf16<4, 16>(a, grid, smem, st);
        if (G == 32) return go_bf16<4, 32>(a, grid, smem, st);
    }
    return go_bf16<4>(a, grid, smem, st);
}

bool pass_supported_bf16(int R) { return R == 1 || R == 2 || R == 4 || R == 6 || R == 8; }

cudaError_t launch_pass_bf16(const PassArgs &a, dim3 grid, int smem, cudaStream_t st)
{
    switch (a.R) {
    case 1: return go_bf16<1>(a, grid, smem, st);
    case 2: return go_bf16<2>(a, grid, smem, st);
    case 4: return go_bf16_r4(a, grid, smem, st);
    case 6: return go_bf16<6>(a, grid, smem, st);
    case 8: return go_bf16<8>(a, grid, smem, st);
    default: return cudaErrorInvalidValue;
    }
}

// Opt every instantiation in to the full shared-memory carve-out (done once,
// outside any stream capture).
void prepare_pass_bf16()
{
    auto set_smem = [](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    };
    set_smem(pass_kernel<1, PREC_BF16, 0>);
    set_smem(pass_kernel<2, PREC_BF16, 0>);
    set_smem(pass_kernel<4, PREC_BF16, 0>);
    set_smem(pass_kernel<6, PREC_BF16, 0>);
    set_smem(pass_kernel<8, PREC_BF16, 0>);
    set_smem(pass_kernel<4, PREC_BF16, 8>);
    set_smem(pass_kernel<4, PREC_BF16, 16>);
    set_smem(pass_kernel<4, PREC_BF16, 32>);
    cudaGetLastError();
}

}  // namespace rpiv
