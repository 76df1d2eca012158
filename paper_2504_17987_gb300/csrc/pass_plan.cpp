// Host-side tiling and shared-memory layout of the fused correlation pass,
// and dispatch to the per-precision kernel instantiations.
#include <algorithm>
#include <cstdlib>
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

int device_sm_count()
{
    constexpr int kMaxDev = 64;
    static int count[kMaxDev] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 152;
    if (!count[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 152;
        count[dev] = n;
    }
    return count[dev];
}

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
// RPIV_TILE_SMEM_KB caps the shared memory of a tile (tuning).
int smem_budget_override()
{
    static int kb = [] {
        const char *e = std::getenv("RPIV_TILE_SMEM_KB");
        const int v = e ? std::atoi(e) : 0;
        return (v >= 16 && v <= 227) ? v : 0;
    }();
    return kb;
}

constexpr int kSmemMax = 227 * 1024;

// (block, sy, row group) items the FP32 plane loop aims for before it stops
// splitting blocks into row groups: half the CTA's threads (swept on GB300:
// 64..512, 128 best, again after row groups came to be summed by shuffles;
// more groups cost more shuffles).
// RPIV_PLANE_ITEMS overrides it (tuning).
int plane_items()
{
    static int n = [] {
        const char *e = std::getenv("RPIV_PLANE_ITEMS");
        const int v = e ? std::atoi(e) : 0;
        return (v >= 1 && v <= 4096) ? v : kThreads / 2;
    }();
    return n;
}

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

// strip: a one-row tile whose CTA walks window rows; its block planes live in
// a two-row ring outside the reused region, since they outlive a step
// Outputs per running sum of a box-sum pass, for n outputs along a run and
// `across` runs side by side: 8, unless a longer run (up to 16) brings all
// runs into one round of the CTA's threads and still keeps 7/8 of them busy.
// Each run starts with a full w-term sum, and a longer run of add/subtract
// updates drifts further.  Measured per 64-pair 1 MP launch: 16 px tiles
// (410 -> 246 column runs, 315 -> 245 row runs) 1.200 -> 1.158 ms; runs
// that left threads idle were slower (strips of 32 px windows, 308 -> 154
// column runs, 0.993 -> 1.033 ms).
int box_run(int n, int across)
{
    const int runs = kThreads / across;
    if (runs < 1) return 8;
    const int L = (n + runs - 1) / runs;
    if (L <= 8 || L > 16) return 8;
    const int items = across * ((n + L - 1) / L);
    return 8 * items >= 7 * kThreads ? L : 8;
}

Layout layout_for(int TX, int TY, int w, int s, int R, int G, int prec, bool strip = false)
{
    PassPlan p;
    std::memset(&p, 0, sizeof(p));
    const int ND = 2 * R + 1, NP = ND * ND;
    const int aw = (TX - 1) * s + w, ah = (TY - 1) * s + w;
    const int BC = aw + 2 * (R + 1), BR = ah + 2 * (R + 1);
    const int vh = BR - w + 1;
    const int nb = (aw / G) * (ah / G);
    const int nwin = TX * TY;
    p.TX = TX;
    p.TY = TY;
    p.G = G;
    p.threads = kThreads;
    p.padl = up(R + 1, 4);
    // pitches chosen so the dominant access patterns are bank-conflict free:
    // 128-bit loads down consecutive rows need pitch/4 odd; the scalar sliding
    // sums along rows need an odd pitch; paired 16-bit loads of 8 rows x 4
    // words need pitch/2 = 4 (mod 8)
    auto odd4 = [](int x) { x = up(x, 4); return ((x / 4) % 2) ? x : x + 4; };
    auto odd8 = [](int x) { x = up(x, 8); return ((x / 8) % 2) ? x : x + 8; };
    p.a_pitch = odd4(aw);
    p.b_pitch = odd4(p.padl + aw + R + 4);
    p.h_pitch = BC | 1;
    p.v_pitch = (BC - w + 1) | 1;
    p.box_lv = box_run(vh, BC);
    p.box_lh = box_run(BC - w + 1, vh);
    p.box_nv = (vh + p.box_lv - 1) / p.box_lv;
    p.box_nh = (BC - w + 1 + p.box_lh - 1) / p.box_lh;
    if (prec == PREC_FP32) {
        // row groups per block: enough (block, sy, row-group) items to fill the
        // CTA; a power of two dividing G, so that a group's partial planes sit
        // in aligned lanes of one warp and are summed by shuffles.  A strip step
        // computes one block row.
        const int nb_step = strip ? aw / G : nb;
        int RG = 1;
        while (2 * RG <= 32 && G % (2 * RG) == 0 && nb_step * ND * RG < plane_items()) RG *= 2;
        p.RGx = RG;
    } else {
        // warp per (block, row group): enough groups for the CTA's warps; a
        // power of two dividing G, groups of at least two rows
        int RG = 1;
        while (nb * RG < kThreads / 32 && G % (2 * RG) == 0 && G / (2 * RG) >= 2) RG *= 2;
        p.RGx = RG;
    }
    int off = 0;
    auto take = [&](int bytes) {
        int o = off;
        off = up(off + bytes, 16);
        return o;
    };
    // the regions start on 128-byte boundaries (tensor-map destinations)
    p.off_a = take(ah * p.a_pitch * 4);
    off = up(off, 128);
    p.off_b = take(BR * p.b_pitch * 4);
    p.box_ah = ah;
    p.box_br = BR;
    p.tma_ok = (s % 4 == 0 && p.a_pitch <= 256 && p.b_pitch <= 256 && ah <= 256 && BR <= 256) ? 1 : 0;
    p.off_v = take(2 * vh * p.v_pitch * 4);
    p.off_stats = take(2 * nwin * 4);
    p.off_red = take(16);      // the region loads' mbarrier
    p.off_gst = take(nb * 8);  // per-block (sum, centred sum of squares) of A
    if (strip) p.off_p = take(2 * (aw / G) * NP * 4);
    // region reused over the phases:
    //   FP32: C (column box sums) -> P (block planes) + per-window stencil buffers
    //   TC:   C -> 16-bit copies TA, TB + P -> per-window buffers (over TA, TB) + P
    const int c_bytes = 2 * vh * p.h_pitch * 4;
    // FP32: one plane per block; TC: the row groups' partial planes, summed in place
    p.pstride = (prec == PREC_FP32 ? 1 : p.RGx) * NP;
    const int p_bytes = up(nb * p.pstride * 4, 16);
    // direct stencil partials: (window, row group) items, at most max(nwin, warps)
    const int win_bytes = up(nwin * 5 * 4, 16) + up(nwin * 4, 16) * 2 + up(std::max(nwin, kThreads / 32) * 5 * 4, 16);
    p.off_h = off;
    int region = 0, win_off = 0;
    if (prec == PREC_FP32 && strip) {
        win_off = off;
        region = std::max(c_bytes, win_bytes);
    } else if (prec == PREC_FP32) {
        p.off_p = off;
        win_off = off + p_bytes;
        region = std::max(c_bytes, p_bytes + win_bytes);
    } else {
        // Toeplitz fragments of unused shifts reach 16 MT (+ 8 for uneven
        // blocks) columns past the last window column: those columns hold zeros
        const int MT = (ND + 15) / 16;
        p.tb_rows = BR;
        p.tb_cols = up(p.padl - R + aw + 16 * MT + 8, 2);
        p.tca_pitch = odd8(aw);
        p.tcb_pitch = odd8(p.tb_cols);
        // A in slabs per (block row, row group), 2R zero rows between them and
        // around, after the leading rows that keep unused fragments in range
        const int NT = (ND + 7) / 8, rows = G / p.RGx;
        const int front = std::max(0, 8 * NT - 1 - 2 * R);
        const int ta_rows = front + 2 * R + (ah / G) * p.RGx * (rows + 2 * R);
        const int ta_bytes = up(ta_rows * p.tca_pitch * 2, 16);
        const int tb_bytes = up(2 * p.tb_rows * p.tcb_pitch * 2, 16);
        p.off_tca = off;
        p.off_tcb = off + ta_bytes;
        p.off_p = off + ta_bytes + tb_bytes;
        if (win_bytes <= ta_bytes + tb_bytes) {
            win_off = off;
            region = std::max(c_bytes, ta_bytes + tb_bytes + p_bytes);
        } else {
            win_off = p.off_p + p_bytes;
            region = std::max(c_bytes, ta_bytes + tb_bytes + p_bytes + win_bytes);
        }
    }
    p.off_c5 = win_off;
    p.off_peaks = p.off_c5 + up(nwin * 5 * 4, 16);
    p.off_need = p.off_peaks + up(nwin * 4, 16);
    p.off_dpart = p.off_need + up(nwin * 4, 16);
    off = up(off + region, 16);
    p.smem_bytes = off;
    p.max_windows = nwin;
    p.max_blocks = nb;
    Layout L;
    L.bytes = off;
    L.p = p;
    return L;
}

// Tensor-core (tcgen05) tiles: 50 % overlap (w = 2s, s a multiple of 8) at
// r = 4.  The FP32 regions, box sums and statistics are laid out as for the
// FP32 kernel; then the phase's barriers, one NP-float plane per window and
// the FP32 refit planes (|s| <= 2) per block, kept for the whole tile; the
// dead column box sums hold two A slabs, the ring of copy slots and the
// epilogue buffer, and later the per-window stencil buffers.  A slot holds one
// 8-column chunk past the tile's columns; an MMA reads up to 2048 - 512 bytes
// past its slot's last chunk (shift slots it does not need), so the ring ends
// with 1 KB of slack.
constexpr int kTcRows = 4;
constexpr int kTcEbufBytes = 3 * 32 * 20 * 4;
constexpr int kTcRn = 2;

bool tc_shape(int w, int s, int R) { return R == 4 && w == 2 * s && (s == 8 || s == 16 || s == 32); }

Layout layout_for_tc(int TX, int TY, int w, int s, int R, int ns)
{
    Layout L = layout_for(TX, TY, w, s, R, s, PREC_FP32);
    PassPlan &p = L.p;
    const int ND = 2 * R + 1, NP = ND * ND, NDN = 2 * kTcRn + 1;
    const int aw = (TX - 1) * s + w, ah = (TY - 1) * s + w;
    const int BR = ah + 2 * (R + 1), vh = BR - w + 1;
    const int nwin = TX * TY, nch = aw / 8, nb = (aw / s) * (ah / s);
    // row groups of the refit planes: enough (block, sy, group) items for the CTA
    int RG = 1;
    while (2 * RG <= 32 && s % (2 * RG) == 0 && nb * NDN * RG < kThreads) RG *= 2;
    p.RGx = RG;
    p.pstride = NP;
    p.tc = 1;
    p.slab_rows = w + 2 * R + 16 - kTcRows;
    p.slab_lbo = p.slab_rows * 16;
    p.cp_lbo = 8 * kTcRows * 16;
    p.cp_group = (nch + 1) * p.cp_lbo;
    p.tc_nbuf = ns;
    p.cp_bytes = ns * p.cp_group + 1024;
    int cols = 32;
    while (cols < 32 * TX) cols *= 2;
    p.tmem_cols = cols;
    // rebuild the offsets past the box sums
    int off = p.off_v + up(2 * vh * p.v_pitch * 4, 16);
    auto take = [&](int bytes) {
        int o = off;
        off = up(off + bytes, 16);
        return o;
    };
    p.off_stats = take(2 * nwin * 4);
    // the regions' barrier, the phase's 2 ns + 6, then the TMEM address, the tile offset, the abort flag
    p.off_red = take(8 * (1 + 2 * ns + 6) + 16);
    p.off_gst = take(nb * 8);
    p.off_p = take(nwin * NP * 4);
    p.off_refit = take(nb * NDN * NDN * 4);
    p.off_h = off;
    const int c_bytes = 2 * vh * p.h_pitch * 4;
    p.off_slab = off;
    p.off_cp = up(p.off_slab + 2 * nch * p.slab_lbo, 16);
    p.off_ebuf = up(p.off_cp + p.cp_bytes, 16);
    const int tc_end = p.off_ebuf + kTcEbufBytes;
    const int win_bytes = up(nwin * 5 * 4, 16) + up(nwin * 4, 16) * 2 + up(std::max(nwin, kThreads / 32) * 5 * 4, 16);
    p.off_c5 = off;
    p.off_peaks = p.off_c5 + up(nwin * 5 * 4, 16);
    p.off_need = p.off_peaks + up(nwin * 4, 16);
    p.off_dpart = p.off_need + up(nwin * 4, 16);
    off = std::max({off + c_bytes, tc_end, off + win_bytes});
    p.smem_bytes = up(off, 16);
    p.max_windows = nwin;
    p.max_blocks = nb;
    L.bytes = p.smem_bytes;
    return L;
}

}  // namespace

// RPIV_TC_PLANES=1 runs the tcgen05 kernel for the shapes it covers (tests
// run both kernels); read at each plan.  The mma.sync kernel is the default:
// measured on GB300 at 1 MP it is faster (6.3k against 4.1k pairs/s).  One
// thread's tcgen05.mma of K = 16 complete about 150 cycles apart whatever N
// is; the banded correlation fills at most 16 N columns of an MMA usefully,
// and the kernel has one issuing thread per CTA.
bool tc_planes_enabled()
{
    const char *e = std::getenv("RPIV_TC_PLANES");
    return e && std::strcmp(e, "1") == 0;
}

bool pass_supported(int R, int prec)
{
    if (R < 0 || R > 16) return false;
    if (prec == PREC_FP32) return true;
    if (prec == PREC_BF16) return pass_supported_bf16(R);
    if (prec == PREC_FP16) return pass_supported_fp16(R);
    return false;
}

// CTAs per SM a tile must leave room for.  Swept on GB300 (targets 2..6):
// FP32 windows of 48 px and more run best at three CTAs, whose larger tiles
// let neighbouring windows share their blocks (64 px: 0.78 -> 0.59 ms at
// 16 MP), 24..40 px at four; below 24 px three at r >= 4 (16 px, r = 4:
// 1.235 -> 1.192 ms per 64 MP launch) and five at small radii (16 px, r = 1:
// 0.80 -> 0.69 ms); the tensor-core kernel, with its 16-bit copies, at three.
// RPIV_MIN_CTAS overrides it (tuning).
int min_ctas(int w, int R, int prec)
{
    static int n = [] {
        const char *e = std::getenv("RPIV_MIN_CTAS");
        const int v = e ? std::atoi(e) : 0;
        return (v >= 1 && v <= 8) ? v : 0;
    }();
    if (n) return n;
    if (prec != PREC_FP32) return 3;
    if (w >= 48) return 3;
    if (w >= 24) return 4;
    return R >= 4 ? 3 : 5;
}

// Tiles: among shapes of up to 8 x 8 windows (not necessarily square) that
// leave room for min_ctas() CTAs per SM, counting shared memory (228 KB per
// SM, 1 KB reserved per CTA), threads and registers, the one with the most
// windows; ties go to fewer blocks per window, then to the squarer tile.  If
// none fits, the shape with the most CTAs per SM.
bool plan_search(int w, int s, int R, int G, int nx, int ny, int prec, PassPlan *plan)
{
    // registers per thread as the kernels are built: the FP32 kernel is bounded
    // to five CTAs per SM up to r = 4 (48 registers), three beyond, for the
    // kernel specialised to 64 px windows at 50 % overlap and for 16 px windows
    // at r = 4; the tensor-core kernel to three
    const bool wide = (w == 64 && s == 32 && (R == 1 || R == 4)) || (w == 16 && s == 8 && R == 4);
    const int regs = (prec == PREC_FP32 && R <= 4 && !wide) ? 48 : 80;
    const int by_regs = 65536 / (regs * kThreads), by_threads = 2048 / kThreads;
    const int override_kb = smem_budget_override();
    const int target = min_ctas(w, R, prec);
    double best = -1e30;
    Layout pick{};
    int pick_tx = 0, pick_ty = 0;
    for (int ty = 1; ty <= std::min(8, ny); ++ty)
        for (int tx = 1; tx <= std::min(8, nx); ++tx) {
            Layout L = layout_for(tx, ty, w, s, R, G, prec);
            if (L.bytes > kSmemMax) continue;
            if (override_kb && L.bytes > override_kb * 1024 && !(tx == 1 && ty == 1)) continue;
            const int ctas = std::min({228 * 1024 / (L.bytes + 1024), by_regs, by_threads});
            if (ctas < 1) continue;
            const int aw = (tx - 1) * s + w, ah = (ty - 1) * s + w;
            const double blocks_per_win = (double)(aw / G) * (ah / G) / (tx * ty);
            const double score = std::min(ctas, target) * 1e8 + (double)tx * ty * 1e5 - blocks_per_win * 1e2 -
                                 std::abs(tx - ty);
            if (score > best) {
                best = score;
                pick = L;
                pick_tx = tx;
                pick_ty = ty;
            }
        }
    if (pick_tx == 0) return false;
    *plan = pick.p;
    plan->tiles_x = (nx + pick_tx - 1) / pick_tx;
    plan->tiles_y = (ny + pick_ty - 1) / pick_ty;
    return true;
}

namespace {

// Window rows a strip CTA walks (RPIV_STRIP_ROWS, tuning; 0 turns strips off).
// The first row of a segment computes both block rows, the others one.
int strip_rows_setting()
{
    static int n = [] {
        const char *e = std::getenv("RPIV_STRIP_ROWS");
        if (!e) return 8;
        const int v = std::atoi(e);
        return (v >= 0 && v <= 4096) ? v : 8;
    }();
    return n;
}

}  // namespace

// Strips for the FP32 kernels specialised to 50 % overlap with 16 or 32 px
// blocks (32 and 64 px windows) at r = 1 and 4: among one-row tiles of up to
// 8 windows that leave room for the kernel's CTAs per SM, the widest.
// Measured per 64-pair launch of the 1 MP workload: 64 px passes 1.346 ->
// 1.160 ms (three CTAs per SM), 32 px passes 1.083 -> 1.001 ms (four; at
// three they were no faster).  16 px strips were slower (1.215 -> 1.789 ms):
// with 8 px blocks the per-row box sums and barriers outweigh the planes saved.
bool plan_strip(int w, int s, int R, int G, int nx, int ny, int prec, PassPlan *plan)
{
    const int L = strip_rows_setting();
    if (prec != PREC_FP32 || L < 2 || ny < 2 || w != 2 * s || s != G || (G != 16 && G != 32) || (R != 1 && R != 4))
        return false;
    // the strip kernels are bounded to three CTAs per SM (80 registers), four for 16 px blocks
    const int target = G == 32 ? 3 : 4;
    const int regs = G == 32 ? 80 : 64;
    const int by_regs = 65536 / (regs * kThreads), by_threads = 2048 / kThreads;
    int pick_tx = 0;
    Layout pick{};
    for (int tx = 1; tx <= std::min(8, nx); ++tx) {
        Layout Lo = layout_for(tx, 1, w, s, R, G, prec, true);
        if (Lo.bytes > kSmemMax) continue;
        const int ctas = std::min({228 * 1024 / (Lo.bytes + 1024), by_regs, by_threads});
        if (ctas < target) continue;
        pick_tx = tx;
        pick = Lo;
    }
    if (pick_tx == 0) return false;
    *plan = pick.p;
    plan->strip_rows = std::min(L, ny);
    plan->tiles_x = (nx + pick_tx - 1) / pick_tx;
    plan->tiles_y = (ny + plan->strip_rows - 1) / plan->strip_rows;
    return true;
}

// Tensor-core tiles: among shapes of up to 8 x 8 windows with rings of 6 or 4
// copy slots, those that leave room for two CTAs per SM (shared memory, and
// 512 TMEM columns per SM: two rows of 16 columns per window): the most
// windows, then the longer ring, then the squarer tile.
bool plan_tc(int w, int s, int R, int nx, int ny, PassPlan *plan)
{
    double best = -1e30;
    Layout pick{};
    int pick_tx = 0, pick_ty = 0;
    for (int ty = 1; ty <= std::min(8, ny); ++ty)
        for (int tx = 1; tx <= std::min(8, nx); ++tx)
            for (int ns : {6, 4}) {
                Layout L = layout_for_tc(tx, ty, w, s, R, ns);
                if (L.bytes > kSmemMax) continue;
                const int ctas = std::min({228 * 1024 / (L.bytes + 1024), 2048 / kThreads, 512 / L.p.tmem_cols});
                if (ctas < 1) continue;
                const double score = std::min(ctas, 2) * 1e8 + (double)tx * ty * 1e5 + ns * 1e3 - std::abs(tx - ty);
                if (score > best) {
                    best = score;
                    pick = L;
                    pick_tx = tx;
                    pick_ty = ty;
                }
            }
    if (pick_tx == 0) return false;
    *plan = pick.p;
    plan->tiles_x = (nx + pick_tx - 1) / pick_tx;
    plan->tiles_y = (ny + pick_ty - 1) / pick_ty;
    return true;
}

bool pass_plan(int w, int s, int R, int nx, int ny, int prec, PassPlan *plan, PassPlan *strip)
{
    if (w < 2 || s < 1 || nx < 1 || ny < 1 || !pass_supported(R, prec)) return false;
    if (prec != PREC_FP32 && tc_shape(w, s, R) && tc_planes_enabled()) {
        if (strip) std::memset(strip, 0, sizeof(*strip));
        return plan_tc(w, s, R, nx, ny, plan);
    }
    const int G = gcd(w, s);
    if (prec != PREC_FP32 && (G % 2) != 0) return false;  // paired 16-bit loads need even blocks
    if (strip) {
        std::memset(strip, 0, sizeof(*strip));
        if (!plan_strip(w, s, R, G, nx, ny, prec, strip)) std::memset(strip, 0, sizeof(*strip));
    }
    return plan_search(w, s, R, G, nx, ny, prec, plan);
}

// A strip launch walks its segments serially inside each CTA, so it is taken
// only when its segments (8 window rows, or 4 or 2) give at least 1.5 CTAs per
// SM of the device.  Swept on the 1 MP workload, whose captured batch runs as
// two halves of 32 pairs on forked streams, and on single pairs: with four
// waves (1824 CTAs on 152 SMs) the pyramid passes of a half and every pass of
// a single pair took tiles; at 1.5 per SM they take 8- to 2-row strips,
// 18,968 -> 19,209 pairs/s and 0.188 -> 0.177 ms per single pair on the device.
// Fewer CTAs were slower: 100 gave a single pair 4-row strips for the 32 px
// pass (0.205 ms).  RPIV_STRIP_MIN_CTAS overrides the threshold (tuning, and
// the tests that run both forms); it is read at each launch.
long long strip_min_ctas()
{
    const char *e = std::getenv("RPIV_STRIP_MIN_CTAS");
    if (e) {
        const long long v = std::atoll(e);
        if (v >= 1) return v;
    }
    return 3LL * device_sm_count() / 2;
}

cudaError_t launch_pass(const PassArgs &args_in, int n_pairs, cudaStream_t st)
{
    const PassArgs *pa = &args_in;
    PassArgs strip_args;
    if (args_in.strip.strip_rows > 0) {
        // the planned segment length, or shorter segments (down to 2 window
        // rows) when those give the launch enough CTAs
        const int ny = args_in.ny;
        for (int L = args_in.strip.strip_rows; L >= 2; L /= 2) {
            const long long segs = (ny + L - 1) / L;
            if ((long long)args_in.strip.tiles_x * segs * n_pairs >= strip_min_ctas()) {
                strip_args = args_in;
                strip_args.plan = args_in.strip;
                strip_args.plan.strip_rows = L;
                strip_args.plan.tiles_y = (int)segs;
                pa = &strip_args;
                break;
            }
        }
    }
    PassArgs args = *pa;
    attach_region_maps(args, n_pairs);
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
