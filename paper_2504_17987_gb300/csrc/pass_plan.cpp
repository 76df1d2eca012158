// Host-side tiling and shared-memory layout of the fused correlation pass,
// and dispatch to the per-precision kernel instantiations.
#include <algorithm>
#include <cstring>

#include "rpiv_internal.h"

namespace rpiv {

cudaError_t launch_pass_fp32(const PassArgs &a, dim3 grid, int smem, cudaStream_t st);
cudaError_t launch_pass_bf16(const PassArgs &a, dim3 grid, int smem, cudaStream_t st);
cudaError_t launch_pass_fp16(const PassArgs &a, dim3 grid, int smem, cudaStream_t st);
bool pass_supported_bf16(int R);
bool pass_supported_fp16(int R);
void prepare_pass_fp32();
void prepare_pass_bf16();
void prepare_pass_fp16();

void prepare_pass_kernels()
{
    static int prepared_device = -1;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    if (dev == prepared_device) return;
    prepare_pass_fp32();
    prepare_pass_bf16();
    prepare_pass_fp16();
    prepared_device = dev;
}

namespace {

constexpr int kThreads = 256;
constexpr int kSmemBudget = 110 * 1024;  // two CTAs per SM
constexpr int kSmemMax = 227 * 1024;

int gcd(int a, int b)
{
    while (b) {
        int t = a % b;
        a = b;
        b = t;
    }
    return a;
}

int up(int x, int m) { return (x + m - 1) / m * m; }

struct Layout {
    int bytes;
    PassPlan p;
};

Layout layout_for(int TX, int TY, int w, int s, int R, int G, int prec)
{
    PassPlan p;
    std::memset(&p, 0, sizeof(p));
    const int ND = 2 * R + 1, NP = ND * ND;
    const int aw = (TX - 1) * s + w, ah = (TY - 1) * s + w;
    const int BC = aw + 2 * (R + 1), BR = ah + 2 * (R + 1);
    const int hw = BC - w + 1, vh = BR - w + 1;
    const int nb = (aw / G) * (ah / G);
    p.TX = TX;
    p.TY = TY;
    p.G = G;
    p.threads = kThreads;
    p.padl = up(R + 1, 4);
    p.a_pitch = up(aw, 4);
    p.b_pitch = up(p.padl + aw + R + 1 + 8, 4);
    p.h_pitch = up(hw, 4);
    if (p.h_pitch % 32 == 0) p.h_pitch += 4;
    if (prec == PREC_FP32) {
        // partial planes per block: enough (block, sy, row-group) items to fill the CTA
        int RG = 1;
        while (RG < G && nb * ND * RG < kThreads) {
            int nx = RG + 1;
            while (nx < G && G % nx) ++nx;
            RG = nx;
        }
        p.RGx = RG;
    } else {
        p.RGx = (G + 7) / 8;
    }
    int off = 0;
    auto take = [&](int bytes) {
        int o = off;
        off = up(off + bytes, 16);
        return o;
    };
    p.node_cap = ((BC + s - 1) / s + 3) * ((BR + s - 1) / s + 3);
    p.off_nodes = take(2 * p.node_cap * 4);
    p.off_tabs = take(2 * (BC + BR) * 4);
    p.off_a = take(ah * p.a_pitch * 4);
    p.off_b = take(BR * p.b_pitch * 4);
    p.off_v = take(2 * vh * p.h_pitch * 4);
    p.off_stats = take(2 * TX * TY * 4);
    p.off_red = take(40 * 4);
    // region shared by H (box-sum phase) and the block planes / TC copies
    const int h_bytes = 2 * BR * p.h_pitch * 4;
    const int p_bytes = up(nb * p.RGx * NP * 4, 16);
    int tc_bytes = 0;
    if (prec != PREC_FP32) {
        p.tca_pitch = up(aw + 8, 8);
        p.tcb_pitch = up(p.padl + aw + R + 1 + 16, 8);
        const int ta_rows = up(ah, 8) + 8;
        const int ta_bytes = up(ta_rows * p.tca_pitch * 2, 16);
        const int tb_bytes = up(2 * (BR + 32) * p.tcb_pitch * 2, 16);
        const int sxc = ND < 9 ? ND : 9;
        const int scr_bytes = (kThreads / 32) * sxc * ND * 8 * 4;
        tc_bytes = ta_bytes + tb_bytes + scr_bytes;
        p.off_h = off;
        p.off_p = off;
        p.off_tca = off + p_bytes;
        p.off_tcb = p.off_tca + ta_bytes;
        p.off_scr = p.off_tcb + tb_bytes;
    } else {
        p.off_h = off;
        p.off_p = off;
    }
    off = up(off + std::max(h_bytes, p_bytes + tc_bytes), 16);
    p.smem_bytes = off;
    p.max_windows = TX * TY;
    p.max_blocks = nb;
    Layout L;
    L.bytes = off;
    L.p = p;
    return L;
}

}  // namespace

bool pass_supported(int R, int prec)
{
    if (R < 0 || R > 16) return false;
    if (prec == PREC_FP32) return true;
    if (prec == PREC_BF16) return pass_supported_bf16(R);
    if (prec == PREC_FP16) return pass_supported_fp16(R);
    return false;
}

bool pass_plan(int w, int s, int R, int nx, int ny, int prec, PassPlan *plan)
{
    if (w < 2 || s < 1 || nx < 1 || ny < 1 || !pass_supported(R, prec)) return false;
    const int G = gcd(w, s);
    if (prec != PREC_FP32 && (G % 2) != 0) return false;  // paired 16-bit loads need even blocks
    for (int t = 8; t >= 1; --t) {
        const int TX = std::min(t, nx), TY = std::min(t, ny);
        Layout L = layout_for(TX, TY, w, s, R, G, prec);
        if (L.bytes <= kSmemBudget || (t == 1 && L.bytes <= kSmemMax)) {
            *plan = L.p;
            plan->tiles_x = (nx + TX - 1) / TX;
            plan->tiles_y = (ny + TY - 1) / TY;
            return true;
        }
    }
    return false;
}

cudaError_t launch_pass(const PassArgs &args, int n_pairs, cudaStream_t st)
{
    dim3 grid(args.plan.tiles_x, args.plan.tiles_y, n_pairs);
    const int smem = args.plan.smem_bytes;
    switch (args.prec) {
    case PREC_FP32: return launch_pass_fp32(args, grid, smem, st);
    case PREC_BF16: return launch_pass_bf16(args, grid, smem, st);
    case PREC_FP16: return launch_pass_fp16(args, grid, smem, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace rpiv
