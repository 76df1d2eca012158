// FP32 CUDA-core instantiations of the fused correlation pass, and the
// tensor maps every pass kernel loads its regions through.
#include <cudaTypedefs.h>

#include "pass_impl.cuh"

namespace rpiv {

namespace {

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (no link against the driver library); null where it is unavailable
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// A float frame of the margin layout per pair: columns (pitch), rows, pairs.
bool encode_frames(CUtensorMap *m, const char *base, long long pitch, long long rows, int pairs,
                   long long pair_stride, int box_w, int box_h)
{
    const PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
    if (!fn || !base || pitch <= 0 || rows <= 0 || pairs < 1) return false;
    const long long row_bytes = pitch * 4;
    if (pairs == 1) pair_stride = row_bytes * rows;
    if (((uintptr_t)base & 15) || (row_bytes & 15) || pair_stride <= 0 || (pair_stride & 15)) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)pitch, (cuuint64_t)rows, (cuuint64_t)pairs};
    const cuuint64_t strides[2] = {(cuuint64_t)row_bytes, (cuuint64_t)pair_stride};
    const cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<char *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// The regions of a tile are a_pitch x ah floats of frame A (or the warped A')
// and b_pitch x BR floats of B', at column offsets that are multiples of 4
// (steps that are multiples of 4): one box each per load instead of one bulk
// copy per row.  Boxes reach a few columns past a region (the row pitch of
// the shared-memory copy) and, at the last tiles, past the frame, which the
// copy fills with zeros; the kernels read only the region.
void attach_region_maps(PassArgs &a, int n_pairs)
{
    a.tma = 0;
    const PassPlan &P = a.plan;
    if (!P.tma_ok || n_pairs < 1 || a.s % 4 != 0) return;
    const PtrRef &ar = a.adef.base ? a.adef : a.afl;
    const PtrRef &br = a.bdef;
    if (!ar.base || !br.base || ar.indirect || br.indirect) return;
    if (n_pairs > 1 && (ar.stride <= 0 || br.stride <= 0)) return;
    const long long rows = (long long)a.H + 2LL * a.def_margin;
    if (!encode_frames(&a.tm_a, ar.base, a.def_pitch, rows, n_pairs, ar.stride, P.a_pitch, P.box_ah)) return;
    if (!encode_frames(&a.tm_b, br.base, a.def_pitch, rows, n_pairs, br.stride, P.b_pitch, P.box_br)) return;
    a.tma = 1;
}

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
