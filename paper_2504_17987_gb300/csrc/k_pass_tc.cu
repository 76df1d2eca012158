// 16-bit tensor-core instantiations of the fused correlation pass, BF16 and
// FP16 from one template: the tcgen05 kernel (tc_pass.cuh) for 50 % overlap
// with 8-, 16- and 32-px steps at r = 4, and the mma.sync kernel (m16n8k16,
// k8 for 8 px blocks, FP32 accumulate) for every other supported shape.
#include "tc_pass.cuh"

namespace rpiv {

template <int PREC, int RC, int GC = 0>
static cudaError_t go_mma(const PassArgs &a, dim3 grid, int smem, cudaStream_t st)
{
    pass_kernel<RC, PREC, GC><<<grid, PASS_THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

template <int PREC, int GC>
static cudaError_t go_tcgen05(const PassArgs &a, dim3 grid, int smem, cudaStream_t st)
{
    tc_pass_kernel<PREC, GC><<<grid, PASS_THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

// 50 % overlap with 8-, 16- and 32-px blocks at r = 4: the tcgen05 kernel when
// the plan is laid out for it, else the specialised mma.sync shapes
template <int PREC>
static cudaError_t go_r4(const PassArgs &a, dim3 grid, int smem, cudaStream_t st)
{
    const int G = a.plan.G;
    if (a.plan.tc) {
        if (a.w != 2 * G || a.s != G) return cudaErrorInvalidValue;
        if (G == 8) return go_tcgen05<PREC, 8>(a, grid, smem, st);
        if (G == 16) return go_tcgen05<PREC, 16>(a, grid, smem, st);
        if (G == 32) return go_tcgen05<PREC, 32>(a, grid, smem, st);
        return cudaErrorInvalidValue;
    }
    if (a.w == 2 * G && a.s == G) {
        if (G == 8) return go_mma<PREC, 4, 8>(a, grid, smem, st);
        if (G == 16) return go_mma<PREC, 4, 16>(a, grid, smem, st);
        if (G == 32) return go_mma<PREC, 4, 32>(a, grid, smem, st);
    }
    return go_mma<PREC, 4>(a, grid, smem, st);
}

template <int PREC>
static cudaError_t launch_16bit(const PassArgs &a, dim3 grid, int smem, cudaStream_t st)
{
    switch (a.R) {
    case 1: return go_mma<PREC, 1>(a, grid, smem, st);
    case 2: return go_mma<PREC, 2>(a, grid, smem, st);
    case 4: return go_r4<PREC>(a, grid, smem, st);
    case 6: return go_mma<PREC, 6>(a, grid, smem, st);
    case 8: return go_mma<PREC, 8>(a, grid, smem, st);
    default: return cudaErrorInvalidValue;
    }
}

bool pass_supported_bf16(int R) { return R == 1 || R == 2 || R == 4 || R == 6 || R == 8; }
bool pass_supported_fp16(int R) { return pass_supported_bf16(R); }

cudaError_t launch_pass_bf16(const PassArgs &a, dim3 grid, int smem, cudaStream_t st)
{
    return launch_16bit<PREC_BF16>(a, grid, smem, st);
}

cudaError_t launch_pass_fp16(const PassArgs &a, dim3 grid, int smem, cudaStream_t st)
{
    return launch_16bit<PREC_FP16>(a, grid, smem, st);
}

// Opt every instantiation in to the full shared-memory carve-out (done once,
// outside any stream capture).
template <int PREC>
static void prepare_16bit()
{
    auto set_smem = [](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    };
    set_smem(pass_kernel<1, PREC, 0>);
    set_smem(pass_kernel<2, PREC, 0>);
    set_smem(pass_kernel<4, PREC, 0>);
    set_smem(pass_kernel<6, PREC, 0>);
    set_smem(pass_kernel<8, PREC, 0>);
    set_smem(pass_kernel<4, PREC, 8>);
    set_smem(pass_kernel<4, PREC, 16>);
    set_smem(pass_kernel<4, PREC, 32>);
    set_smem(tc_pass_kernel<PREC, 8>);
    set_smem(tc_pass_kernel<PREC, 16>);
    set_smem(tc_pass_kernel<PREC, 32>);
    cudaGetLastError();
}

void prepare_pass_bf16() { prepare_16bit<PREC_BF16>(); }
void prepare_pass_fp16() { prepare_16bit<PREC_FP16>(); }

}  // namespace rpiv
