// One correlation pass for callers that cannot allocate device memory.
//
// Some callers of this library cannot call cudaMalloc when they run a pass:
// a real-time camera loop whose frame deadline cannot absorb the allocator (it
// may synchronise the device and take an unbounded time), or code embedded in
// a host application that has handed all device memory to its own pool and
// forbids further allocations.  rpiv_stage_correlate asks such callers for a
// scratch buffer; this variant needs none.  Its scratch (frame A as float, or
// the warped first frame for the central warp, and the warped second frame)
// lives in the file-scope array below, which every GPU that loads the library
// holds until the process exits.  Nothing in it has to start at zero: the
// ingest and deformation kernels write every element the correlation kernel
// later uses.
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include <cuda_runtime.h>

#include "rpiv.h"
#include "rpiv_internal.h"

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

rpiv_status bad(rpiv_status st, const char *msg)
{
    rpiv::set_last_error(msg);
    return st;
}

// Device address of the array on the current device.  The host-side name of
// a __device__ variable is not its address, so it is looked up; the lookup is
// made on every call (it allocates nothing once the library's module is
// loaded on the device, which the first call does), so that an address can
// never outlive the context it belongs to.
rpiv_status scratch_address(void **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        char msg[160];
        std::snprintf(msg, sizeof(msg), "cudaGetSymbolAddress of the static scratch failed: %s",
                      cudaGetErrorString(e));
        return bad(e == cudaErrorNoDevice ? RPIV_ERR_NO_DEVICE : RPIV_ERR_CUDA, msg);
    }
    *out = p;
    return RPIV_OK;
}

// RPIV_POISON_SCRATCH=1 (testing aid): the part of the array a call uses is
// filled with 0xFF bytes (NaN as float) on the caller's stream first, so that
// a read of an element the call did not write surfaces instead of finding a
// finite value left by an earlier call.  A memset, not an allocation.
bool poison_scratch()
{
    const char *e = std::getenv("RPIV_POISON_SCRATCH");
    return e && std::strcmp(e, "1") == 0;
}

}  // namespace

extern "C" rpiv_status rpiv_stage_correlate_noalloc(const void *img_a, const void *img_b, size_t pitch_bytes, int fmt,
                                                    int width, int height, int window, int step, int radius,
                                                    rpiv_precision precision, rpiv_deform deform_mode,
                                                    const float *pred_u, const float *pred_v, float *u, float *v,
                                                    int32_t *info, void *cuda_stream)
{
    if (width < 1 || height < 1 || width > 65536 || height > 65536 || radius < 0 || radius > RPIV_MAX_RADIUS)
        return bad(RPIV_ERR_INVALID_ARG, "image size or radius out of range");
    // the same frames rpiv_stage_correlate takes from its caller's scratch
    const size_t need = rpiv::single_pass_scratch_bytes(width, height, radius);
    if (need > kStaticScratchBytes) {
        char msg[200];
        std::snprintf(msg, sizeof(msg),
                      "image needs %zu bytes of scratch; the static scratch holds %zu (use rpiv_stage_correlate)", need,
                      kStaticScratchBytes);
        return bad(RPIV_ERR_INVALID_ARG, msg);
    }
    void *scratch = nullptr;
    rpiv_status st1 = scratch_address(&scratch);
    if (st1 != RPIV_OK) return st1;
    if (poison_scratch()) {
        const cudaError_t e = cudaMemsetAsync(scratch, 0xFF, need, static_cast<cudaStream_t>(cuda_stream));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return bad(RPIV_ERR_CUDA, "static scratch fill failed");
        }
    }
    return (rpiv_status)rpiv::single_pass(img_a, img_b, pitch_bytes, fmt, width, height, window, step, radius,
                                          (int)precision, (int)deform_mode, pred_u, pred_v, u, v, info, scratch,
                                          static_cast<cudaStream_t>(cuda_stream));
}
