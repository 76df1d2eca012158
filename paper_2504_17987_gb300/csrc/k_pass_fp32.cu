// FP32 CUDA-core instantiations of the fused correlation pass.
#include "pass_impl.cuh"

namespace rpiv {

template <int RC, int GC = 0>
static cudaError_t go_fp32(const PassArgs &a, dim3 grid, int smem, cudaStream_t st)
{
    pass_kernel<RC, PREC_FP32, GC><<<grid, PASS_THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

// Specialised shapes: 50 % overlap with blocks of 8, 16 or 32 pixels (16, 32
// and 64 px windows) at the radii of the benchmark schedules (1 and 4).
template <int RC, int GC>
static cudaError_t go_strip(const PassArgs &a, dim3 grid, int smem, cudaStream_t st)
{
    strip_kernel<RC, GC><<<grid, PASS_THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

template <int RC>
static cudaError_t go_shaped(const PassArgs &a, dim3 grid, int smem, cudaStream_t st)
{
    const int G = a.plan.G;
    if (a.plan.strip_rows > 0) {
        // strips are planned only for these shapes
        if (G == 16) return go_strip<RC, 16>(a, grid, smem, st);
        if (G == 32) return go_strip<RC, 32>(a, grid, smem, st);
        return cudaErrorInvalidValue;
    }
    if (a.w == 2 * G && a.s == G) {
        if (G == 8) return go_fp32<RC, 8>(a, grid, smem, st);
        if (G == 16) return go_fp32<RC, 16>(a, grid, smem, st);
        if (G == 32) return go_fp32<RC, 32>(a, grid, smem, st);
    }
    return go_fp32<RC>(a, grid, smem, st);
}

// Radii with a register-blocked fast path (the block size must be a multiple
// of 4 for its aligned loads); everything else runs the runtime-radius kernel.
cudaError_t launch_pass_fp32(const PassArgs &a, dim3 grid, int smem, cudaStream_t st)
{
    if (a.plan.G % 4 == 0) {
        switch (a.R) {
        case 0: return go_fp32<0>(a, grid, smem, st);
        case 1: return go_shaped<1>(a, grid, smem, st);
        case 2: return go_fp32<2>(a, grid, smem, st);
        case 3: return go_fp32<3>(a, grid, smem, st);
        case 4: return go_shaped<4>(a, grid, smem, st);
        case 6: return go_fp32<6>(a, grid, smem, st);
        case 8: return go_fp32<8>(a, grid, smem, st);
        default: break;
        }
    }
    return go_fp32<-1>(a, grid, smem, st);
}

// Opt every instantiation in to the full shared-memory carve-out (done once,
// outside any stream capture).
void prepare_pass_fp32()
{
    auto set_smem = [](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    };
    set_smem(pass_kernel<0, PREC_FP32, 0>);
    set_smem(pass_kernel<1, PREC_FP32, 0>);
    set_smem(pass_kernel<2, PREC_FP32, 0>);
    set_smem(pass_kernel<3, PREC_FP32, 0>);
    set_smem(pass_kernel<4, PREC_FP32, 0>);
    set_smem(pass_kernel<6, PREC_FP32, 0>);
    set_smem(pass_kernel<8, PREC_FP32, 0>);
    set_smem(pass_kernel<-1, PREC_FP32, 0>);
    set_smem(pass_kernel<1, PREC_FP32, 8>);
    set_smem(pass_kernel<1, PREC_FP32, 16>);
    set_smem(pass_kernel<1, PREC_FP32, 32>);
    set_smem(pass_kernel<4, PREC_FP32, 8>);
    set_smem(pass_kernel<4, PREC_FP32, 16>);
    set_smem(pass_kernel<4, PREC_FP32, 32>);
    set_smem(strip_kernel<1, 16>);
    set_smem(strip_kernel<1, 32>);
    set_smem(strip_kernel<4, 16>);
    set_smem(strip_kernel<4, 32>);
    cudaGetLastError();
}

}  // namespace rpiv
