// Host probe of the correlation-pass planner (pass_plan.cpp), built by
// tests/test_plan_host.py with the host compiler: the launch and prepare
// entry points it refers to are stubs, so no device is involved.  Reads
// "w s R nx ny prec" lines on stdin and prints one line per case:
//   ok TX TY tiles_x tiles_y smem RGx lv lh nv nh | sTX srows stiles_x stiles_y ssmem slv slh snv snh
//   | tc off_p off_red off_gst off_h off_slab slab_rows slab_lbo off_cp cp_bytes cp_lbo nbuf off_ebuf tmem_cols
//     off_c5 off_dpart cp_group off_refit
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
void attach_region_maps(PassArgs &a, int) { a.tma = 0; }
}  // namespace rpiv

extern "C" cudaError_t cudaGetDevice(int *d)
{
    *d = 0;
    return cudaSuccess;
}

extern "C" cudaError_t cudaDeviceGetAttribute(int *v, cudaDeviceAttr, int)
{
    *v = 152;
    return cudaSuccess;
}

int main()
{
    int w, s, R, nx, ny, prec;
    while (std::scanf("%d %d %d %d %d %d", &w, &s, &R, &nx, &ny, &prec) == 6) {
        rpiv::PassPlan p{}, st{};
        const bool ok = rpiv::pass_plan(w, s, R, nx, ny, prec, &p, &st);
        std::printf("%d %d %d %d %d %d %d %d %d %d %d | %d %d %d %d %d %d %d %d %d", ok ? 1 : 0, p.TX, p.TY,
                    p.tiles_x, p.tiles_y, p.smem_bytes, p.RGx, p.box_lv, p.box_lh, p.box_nv, p.box_nh, st.TX,
                    st.strip_rows, st.tiles_x, st.tiles_y, st.smem_bytes, st.box_lv, st.box_lh, st.box_nv,
                    st.box_nh);
        std::printf(" | %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d\n", p.tc, p.off_p, p.off_red,
                    p.off_gst, p.off_h, p.off_slab, p.slab_rows, p.slab_lbo, p.off_cp, p.cp_bytes, p.cp_lbo,
                    p.tc_nbuf, p.off_ebuf, p.tmem_cols, p.off_c5, p.off_dpart, p.cp_group, p.off_refit);
    }
    return 0;
}
