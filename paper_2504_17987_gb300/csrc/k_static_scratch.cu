// One correlation pass for callers that cannot allocate device memory.
//
// Some callers of this library cannot call cudaMalloc when they run a pass:
// a real-time camera loop whose frame deadline cannot absorb the allocator (it
// may synchronise the device and take an unbounded time), or code embedded in
// a host application that has handed all device memory to its own pool and
// forbids further allocations.  rpiv_stage_correlate asks such callers for a
// scratch buffer; this variant needs none.  Its scratch (the warped frame, and
// the warped first frame for the central warp) lives in the file-scope array
// below, which every GPU that loads the library holds until the process
// exits.  Nothing in it has to start at zero: the deformation kernel writes
// every element the correlation kernel later reads.
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "rpiv.h"
#include "rpiv_internal.h"

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {};

int grid_count(int extent, int w, int s) { return (extent < w || w < 1 || s < 1) ? 0 : (extent - w) / s + 1; }

rpiv_status bad(rpiv_status st, const char *msg)
{
    rpiv::set_last_error(msg);
    return st;
}

// Device address of the array on the current device, looked up once per
// device (the host-side name of a __device__ variable is not its address).
rpiv_status scratch_address(void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return bad(RPIV_ERR_NO_DEVICE, "no current CUDA device");
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || p == nullptr) {
            char msg[160];
            std::snprintf(msg, sizeof(msg), "cudaGetSymbolAddress of the static scratch failed: %s",
                          cudaGetErrorString(e));
            return bad(RPIV_ERR_CUDA, msg);
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return RPIV_OK;
}

}  // namespace

extern "C" rpiv_status rpiv_stage_correlate_noalloc(const void *img_a, const void *img_b, size_t pitch_bytes, int fmt,
                                                    int width, int height, int window, int step, int radius,
                                                    rpiv_precision precision, rpiv_deform deform_mode,
                                                    const float *pred_u, const float *pred_v, float *u, float *v,
                                                    int32_t *info, void *cuda_stream)
{
    using namespace rpiv;
    if (!img_a || !img_b || !u || !v || !info) return bad(RPIV_ERR_INVALID_ARG, "null argument");
    if ((pred_u == nullptr) != (pred_v == nullptr)) return bad(RPIV_ERR_INVALID_ARG, "pred_u and pred_v: both or neither");
    if (fmt != 0 && fmt != RPIV_U8 && fmt != RPIV_U16) return bad(RPIV_ERR_INVALID_ARG, "fmt");
    if (window < 2 || step < 1 || radius < 0 || radius > RPIV_MAX_RADIUS)
        return bad(RPIV_ERR_INVALID_ARG, "window, step or radius out of range");
    if (width < window + 2 * (radius + 1) || height < window + 2 * (radius + 1))
        return bad(RPIV_ERR_INVALID_ARG, "image smaller than window + 2 (radius + 1)");
    const int bpp = fmt == RPIV_U8 ? 1 : (fmt == RPIV_U16 ? 2 : 4);
    if (pitch_bytes < (size_t)width * bpp || pitch_bytes % bpp) return bad(RPIV_ERR_INVALID_ARG, "pitch_bytes");
    if (precision != RPIV_FP32 && precision != RPIV_BF16 && precision != RPIV_FP16)
        return bad(RPIV_ERR_INVALID_ARG, "precision");
    if (deform_mode != RPIV_DEFORM_B && deform_mode != RPIV_DEFORM_CENTRAL)
        return bad(RPIV_ERR_INVALID_ARG, "deform_mode");
    size_t need = 0;
    rpiv_status st0 = rpiv_stage_correlate_scratch_bytes(width, height, radius, deform_mode, &need);
    if (st0 != RPIV_OK) return st0;
    if (need > kStaticScratchBytes) {
        char msg[200];
        std::snprintf(msg, sizeof(msg),
                      "image needs %zu bytes of scratch; the static scratch holds %zu (use rpiv_stage_correlate)", need,
                      kStaticScratchBytes);
        return bad(RPIV_ERR_INVALID_ARG, msg);
    }
    const int nx = grid_count(width, window, step), ny = grid_count(height, window, step);
    if (!deform_nodes_fit(window, step, nx, ny)) return bad(RPIV_ERR_UNSUPPORTED, "step too small (minimum 3)");
    PassArgs a;
    std::memset(&a, 0, sizeof(a));
    a.prec = radius == 0 ? PREC_FP32 : (precision == RPIV_FP32 ? PREC_FP32 : (precision == RPIV_BF16 ? PREC_BF16 : PREC_FP16));
    if (!pass_plan(window, step, radius, nx, ny, a.prec, &a.plan))
        return bad(RPIV_ERR_UNSUPPORTED, "no kernel for this radius/precision/block size");
    void *scratch = nullptr;
    rpiv_status st1 = scratch_address(&scratch);
    if (st1 != RPIV_OK) return st1;
    // same geometry as rpiv_stage_correlate: frames grown by radius + 1, rows of 32-float multiples
    const int M = radius + 1;
    const long long dpitch = (long long)(((size_t)width + 2 * M + 31) / 32 * 32);
    const size_t one = (size_t)dpitch * (height + 2 * M) * 4;
    char *bdef = static_cast<char *>(scratch);
    char *adef = deform_mode == RPIV_DEFORM_CENTRAL ? bdef + (one + 255) / 256 * 256 : nullptr;
    const int pfmt = fmt == RPIV_U8 ? PIX_U8 : (fmt == RPIV_U16 ? PIX_U16 : PIX_F32);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    prepare_pass_kernels();
    for (int which = adef ? 0 : 1; which < 2; ++which) {
        DeformArgs da;
        std::memset(&da, 0, sizeof(da));
        da.img = ptr_direct(which ? img_b : img_a, 0);
        da.fmt = pfmt;
        da.pitch = (long long)pitch_bytes;
        da.W = width;
        da.H = height;
        da.pred_u = ptr_direct(pred_u, 0);
        da.pred_v = ptr_direct(pred_v, 0);
        da.w = window;
        da.s = step;
        da.nx = nx;
        da.ny = ny;
        da.scale = adef ? (which ? 0.5f : -0.5f) : 1.0f;
        da.M = M;
        da.out = ptr_direct(which ? bdef : adef, 0);
        da.out_pitch = dpitch;
        cudaError_t e = launch_deform(da, 1, st);
        if (e != cudaSuccess) return bad(RPIV_ERR_CUDA, cudaGetErrorString(e));
    }
    a.W = width;
    a.H = height;
    a.fmt = pfmt;
    a.pitch = (long long)pitch_bytes;
    a.img_a = ptr_direct(img_a, 0);
    a.img_b = ptr_direct(img_b, 0);
    a.bdef = ptr_direct(bdef, 0);
    a.adef = ptr_direct(adef, 0);
    a.def_pitch = dpitch;
    a.def_margin = M;
    a.w = window;
    a.s = step;
    a.R = radius;
    a.nx = nx;
    a.ny = ny;
    a.deform = adef ? 1 : 0;
    a.pred_u = ptr_direct(pred_u, 0);
    a.pred_v = ptr_direct(pred_v, 0);
    a.out_u = ptr_direct(u, 0);
    a.out_v = ptr_direct(v, 0);
    a.out_info = ptr_direct(info, 0);
    cudaError_t e = launch_pass(a, 1, st);
    if (e != cudaSuccess) return bad(RPIV_ERR_CUDA, cudaGetErrorString(e));
    return RPIV_OK;
}
