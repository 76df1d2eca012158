// Host probe of the correlation-pass planner (pass_plan.cpp), built by
// tests/test_plan_host.py with the host compiler: the launch and prepare
// entry points it refers to are stubs, so no device is involved.  Reads
// "w s R nx ny prec" lines on stdin and prints one line per case:
//   ok TX TY tiles_x tiles_y smem RGx lv lh nv nh | sTX srows stiles_x stiles_y ssmem slv slh snv snh
#include <cstdio>

#include "rpiv_internal.h"

namespace rpiv {
cudaError_t launch_pass_bf16(const PassArgs &, dim3, int, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_pass_fp16(const PassArgs &, dim3, int, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_pass_fp32(const PassArgs &, dim3, int, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t prepare_pass_bf16() { return cudaErrorNotSupported; }
cudaError_t prepare_pass_fp16() { return cudaErrorNotSupported; }
cudaError_t prepare_pass_fp32() { return cudaErrorNotSupported; }
bool pass_supported_bf16(int R) { return R >= 0 && R <= 16; }
bool pass_supported_fp16(int R) { return R >= 0 && R <= 16; }
}  // namespace rpiv

extern "C" cudaError_t cudaGetDevice(int *d)
{
    *d = 0;
    return cudaSuccess;
}

int main()
{
    int w, s, R, nx, ny, prec;
    while (std::scanf("%d %d %d %d %d %d", &w, &s, &R, &nx, &ny, &prec) == 6) {
        rpiv::PassPlan p{}, st{};
        const bool ok = rpiv::pass_plan(w, s, R, nx, ny, prec, &p, &st);
        std::printf("%d %d %d %d %d %d %d %d %d %d %d | %d %d %d %d %d %d %d %d %d\n", ok ? 1 : 0, p.TX, p.TY,
                    p.tiles_x, p.tiles_y, p.smem_bytes, p.RGx, p.box_lv, p.box_lh, p.box_nv, p.box_nh, st.TX,
                    st.strip_rows, st.tiles_x, st.tiles_y, st.smem_bytes, st.box_lv, st.box_lh, st.box_nv,
                    st.box_nh);
    }
    return 0;
}
