// C ABI of librpiv (declared in include/rpiv.h): configuration checks, the
// per-handle schedule of stages (pyramid levels, passes), device workspace,
// per-call pointer tables and the CUDA-graph cache.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "rpiv.h"
#include "rpiv_internal.h"

namespace {

// RPIV_POISON_SCRATCH=1: fill freshly allocated workspaces with 0xFF bytes
// (NaN as float) so that reads of unwritten values surface (testing aid)
bool poison_scratch()
{
    static const bool on = [] {
        const char *e = std::getenv("RPIV_POISON_SCRATCH");
        return e && std::strcmp(e, "1") == 0;
    }();
    return on;
}

}  // namespace

using namespace rpiv;

namespace rpiv {
void prepare_pass_kernels();
}

namespace {

thread_local std::string g_err;

rpiv_status fail(rpiv_status st, const std::string &msg)
{
    g_err = msg;
    return st;
}

}  // namespace

void rpiv::set_last_error(const char *msg) { g_err = msg ? msg : ""; }

namespace {

rpiv_status cuda_fail(cudaError_t e, const char *what)
{
    g_err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return RPIV_ERR_CUDA;
}

#define CK(call, what)                                     \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

size_t up(size_t x, size_t m) { return (x + m - 1) / m * m; }

int grid_n(int extent, int w, int s) { return (extent < w || w < 1 || s < 1) ? 0 : (extent - w) / s + 1; }

bool step_of(int w, float overlap, int *s)
{
    const double sd = (double)w * (1.0 - (double)overlap);
    const int si = (int)std::lround(sd);
    if (si < 1 || std::fabs(sd - si) > 1e-4) return false;
    *s = si;
    return true;
}

int prec_of(rpiv_precision p) { return p == RPIV_FP32 ? PREC_FP32 : (p == RPIV_BF16 ? PREC_BF16 : PREC_FP16); }

struct StageDef {
    bool level;  // pyramid level (float images in the workspace) or full-resolution pass
    int lvl;     // pyramid level index (0 for passes)
    int W, H;    // image size of this stage
    int w, s, R;
    int nx, ny;
    int prec;
    long long fpitch;  // floats per row of this stage's frames (margin layout)
    size_t off_pred, off_raw, off_info, off_out, off_mask;  // per-pair workspace offsets
    PassPlan plan, strip;
};

std::string check_config(const rpiv_config *c, std::vector<StageDef> *stages_out)
{
    if (!c) return "config is NULL";
    if (c->fmt != RPIV_U8 && c->fmt != RPIV_U16 && c->fmt != RPIV_F32) return "fmt must be RPIV_U8, RPIV_U16 or RPIV_F32";
    if (c->bit_depth != 8 && c->bit_depth != 12 && c->bit_depth != 16) return "bit_depth must be 8, 12 or 16";
    if (c->fmt == RPIV_U8 && c->bit_depth != 8) return "RPIV_U8 requires bit_depth 8";
    if (c->n_passes < 1 || c->n_passes > RPIV_MAX_PASSES) return "n_passes must be in [1, 4]";
    if (c->predictor_levels < 0 || c->predictor_levels > RPIV_MAX_LEVELS) return "predictor_levels must be in [0, 4]";
    if (c->max_batch < 1 || c->max_batch > RPIV_MAX_BATCH) return "max_batch must be in [1, 64]";
    if (c->host_frames != 0 && c->host_frames != 1) return "host_frames must be 0 or 1";
    if (c->precision != RPIV_FP32 && c->precision != RPIV_BF16 && c->precision != RPIV_FP16)
        return "unknown precision";
    if (c->deform_mode != RPIV_DEFORM_B && c->deform_mode != RPIV_DEFORM_CENTRAL) return "unknown deform_mode";
    if (!(c->uod_threshold > 0.f) || !(c->uod_eps >= 0.f) || !std::isfinite(c->uod_threshold) ||
        !std::isfinite(c->uod_eps))
        return "uod_threshold must be > 0 and uod_eps >= 0";
    if (c->width < 8 || c->height < 8 || c->width > 65536 || c->height > 65536) return "image size out of range";
    for (int p = 0; p < c->n_passes; ++p) {
        const int w = c->window[p];
        if (w < 8 || w > 128 || (w & 1)) return "window[" + std::to_string(p) + "] must be even and in [8, 128]";
        if (!(c->overlap[p] >= 0.f && c->overlap[p] < 1.f)) return "overlap must be in [0, 1)";
        int s;
        if (!step_of(w, c->overlap[p], &s)) return "window * (1 - overlap) must be a positive integer";
        const int R = c->search_radius[p];
        if (R < 0 || R > RPIV_MAX_RADIUS) return "search_radius must be in [0, 16]";
    }
    std::vector<StageDef> st;
    {
        int s0 = 1;
        step_of(c->window[0], c->overlap[0], &s0);
        int W = c->width, H = c->height;
        std::vector<StageDef> lv;
        for (int l = 1; l <= c->predictor_levels; ++l) {
            W /= 2;
            H /= 2;
            StageDef d{};
            d.level = true;
            d.lvl = l;
            d.W = W;
            d.H = H;
            d.w = c->window[0];
            d.s = s0;
            d.R = c->search_radius[0];
            lv.push_back(d);
        }
        for (int i = (int)lv.size() - 1; i >= 0; --i) st.push_back(lv[i]);  // coarsest first
    }
    for (int p = 0; p < c->n_passes; ++p) {
        StageDef d{};
        d.level = false;
        d.W = c->width;
        d.H = c->height;
        d.w = c->window[p];
        step_of(d.w, c->overlap[p], &d.s);
        d.R = c->search_radius[p];
        st.push_back(d);
    }
    for (auto &d : st) {
        if (d.W < d.w + 2 * (d.R + 1) || d.H < d.w + 2 * (d.R + 1))
            return std::string(d.level ? "pyramid level " + std::to_string(d.lvl) : std::string("image")) + " of " +
                   std::to_string(d.W) + "x" + std::to_string(d.H) + " is smaller than window + 2 (radius + 1)";
        d.nx = grid_n(d.W, d.w, d.s);
        d.ny = grid_n(d.H, d.w, d.s);
        if (!deform_nodes_fit(d.w, d.s, d.nx, d.ny))
            return "step " + std::to_string(d.s) + " is too small for the deformation kernel (minimum 3)";
        // a zero radius has a one-point plane: the FP32 kernel serves every precision
        d.prec = d.R == 0 ? PREC_FP32 : prec_of(c->precision);
        if (!pass_plan(d.w, d.s, d.R, d.nx, d.ny, d.prec, &d.plan, &d.strip))
            return "precision " + std::to_string((int)c->precision) + " is not built for radius " +
                   std::to_string(d.R) + " with window " + std::to_string(d.w) + " and step " + std::to_string(d.s);
    }
    if (stages_out) *stages_out = st;
    return "";
}

constexpr int kRing = 16;

}  // namespace

struct rpiv_handle {
    rpiv_config cfg{};
    int device = 0;
    std::vector<StageDef> stages;
    // per-pair offsets of the float frames (margin layout): [l][0] frame A at
    // level l (level 0: ingested from the caller's image each call), [l][1]
    // frame B at pyramid level l >= 1
    size_t frame_off[RPIV_MAX_LEVELS + 1][2] = {};
    size_t def_off[2] = {};  // per-pair offsets of the warped frames B' (and A')
    size_t in_off[2] = {};   // host_frames: per-pair offsets of the uploaded frames A and B
    long long in_pitch = 0;  // host_frames: bytes between their rows (a multiple of 16)
    int margin = 0;          // M of every frame
    size_t pair_stride = 0;
    int *err_dev = nullptr;  // error word of the kernels' bounded waits
    char *ws = nullptr;
    size_t ws_bytes = 0;
    PairIO *io_dev = nullptr;
    PairIO *ring = nullptr;  // pinned host, kRing slots of max_batch entries
    cudaEvent_t ring_ev[kRing] = {};
    bool ring_used[kRing] = {};
    int ring_pos = 0;
    cudaEvent_t done_ev = nullptr;
    bool done_recorded = false;
    cudaStream_t cap_stream = nullptr;
    // capture streams of the further parts of a split batch, fork and join events
    static constexpr int kParts = 4;
    cudaStream_t cap_part[kParts] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[kParts] = {};
    std::map<std::string, cudaGraphExec_t> graphs;
    char *adj_ws = nullptr;
    size_t adj_bytes = 0;
    float *ref_ws = nullptr;  // refinement: gu, gv, cu, cv (n floats each), score, max|g|
    size_t ref_n = 0;
    // stage tracing
    bool tracing = false;
    struct TraceEv {
        std::string name;
        cudaEvent_t t0, t1;
        rpiv_trace_record geom;
    };
    std::vector<TraceEv> trace_evs;
    std::vector<cudaEvent_t> ev_pool;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

cudaEvent_t pool_event(rpiv_handle *h)
{
    if (!h->ev_pool.empty()) {
        cudaEvent_t e = h->ev_pool.back();
        h->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Brackets one launch with events when tracing (never inside a capture).
struct TraceScope {
    rpiv_handle *h;
    cudaStream_t st;
    bool on;
    rpiv_handle::TraceEv ev;
    TraceScope(rpiv_handle *h_, cudaStream_t st_, const std::string &name, const rpiv_trace_record &g)
        : h(h_), st(st_), on(h_->tracing)
    {
        if (!on) return;
        ev.name = name;
        ev.geom = g;
        ev.t0 = pool_event(h);
        ev.t1 = pool_event(h);
        cudaEventRecord(ev.t0, st);
    }
    ~TraceScope()
    {
        if (!on) return;
        cudaEventRecord(ev.t1, st);
        h->trace_evs.push_back(ev);
    }
};

rpiv_trace_record geom_of(int W, int H, int w, int s, int R, int nx, int ny, int n)
{
    rpiv_trace_record g;
    std::memset(&g, 0, sizeof(g));
    g.width = W;
    g.height = H;
    g.window = w;
    g.step = s;
    g.radius = R;
    g.nx = nx;
    g.ny = ny;
    g.pairs = n;
    return g;
}

std::string stage_tag(const rpiv_handle *h, const StageDef &d)
{
    if (d.level) return "L" + std::to_string(d.lvl);
    const int p = (int)(&d - &h->stages[0]) - h->cfg.predictor_levels;
    return "p" + std::to_string(p);
}

// The full schedule for n pairs whose pointers are in h->io_dev.
// The launch sequence of pairs pair0 .. pair0 + n - 1 of the call.
rpiv_status enqueue_schedule(rpiv_handle *h, int n, size_t pitch, bool any_pred, bool any_nopred, cudaStream_t st,
                             int pair0 = 0)
{
    const rpiv_config &c = h->cfg;
    const int L = c.predictor_levels;
    const long long ps = (long long)h->pair_stride;
    const PairIO *io = h->io_dev + pair0;
    const long long ios = sizeof(PairIO);
    char *const wbase = h->ws + (size_t)pair0 * h->pair_stride;
    auto ws = [&](size_t off) { return ptr_direct(wbase + off, ps); };
    auto tab = [&](const void *field) { return ptr_table(field, ios); };
    const int user_fmt = c.fmt == RPIV_U8 ? PIX_U8 : (c.fmt == RPIV_U16 ? PIX_U16 : PIX_F32);
    const StageDef &p0 = h->stages[L];
    const bool run_pyr = L > 0 && any_nopred;
    const bool central = c.deform_mode == RPIV_DEFORM_CENTRAL;
    const int M = h->margin;
    // byte offset of pixel (0, 0) inside a frame of the margin layout
    auto interior = [&](long long fpitch) { return (size_t)((M * fpitch + M) * 4); };

    // A, B: the images the warp samples; afl: frame A of the margin layout
    // (read by the pass when the first frame is not warped)
    auto run_pass = [&](const StageDef &d, PtrRef A, PtrRef B, int fmt, long long pch, PtrRef afl,
                        bool pred) -> rpiv_status {
        const size_t n1 = (size_t)d.nx * d.ny;
        for (int which = central ? 0 : 1; which < 2; ++which) {
            DeformArgs da;
            std::memset(&da, 0, sizeof(da));
            da.img = which ? B : A;
            da.fmt = fmt;
            da.pitch = pch;
            da.W = d.W;
            da.H = d.H;
            da.pred_u = pred ? ws(d.off_pred) : ptr_direct(nullptr, 0);
            da.pred_v = pred ? ws(d.off_pred + 4 * n1) : ptr_direct(nullptr, 0);
            da.w = d.w;
            da.s = d.s;
            da.nx = d.nx;
            da.ny = d.ny;
            da.scale = central ? (which ? 0.5f : -0.5f) : 1.0f;
            da.M = M;
            da.out = ws(h->def_off[which]);
            da.out_pitch = d.fpitch;
            TraceScope ts(h, st, std::string(which ? "deform/" : "deformA/") + stage_tag(h, d),
                          geom_of(d.W, d.H, d.w, d.s, d.R, d.nx, d.ny, n));
            CK(launch_deform(da, n, st), "deformation launch");
        }
        PassArgs a;
        std::memset(&a, 0, sizeof(a));
        a.afl = central ? ptr_direct(nullptr, 0) : afl;
        a.bdef = ws(h->def_off[1]);
        a.adef = central ? ws(h->def_off[0]) : ptr_direct(nullptr, 0);
        a.def_pitch = d.fpitch;
        a.def_margin = M;
        a.err = h->err_dev;
        a.W = d.W;
        a.H = d.H;
        a.fmt = fmt;
        a.pitch = pch;
        a.img_a = A;
        a.img_b = B;
        a.w = d.w;
        a.s = d.s;
        a.R = d.R;
        a.nx = d.nx;
        a.ny = d.ny;
        a.deform = c.deform_mode == RPIV_DEFORM_CENTRAL ? 1 : 0;
        a.prec = d.prec;
        a.pred_u = pred ? ws(d.off_pred) : ptr_direct(nullptr, 0);
        a.pred_v = pred ? ws(d.off_pred + 4 * n1) : ptr_direct(nullptr, 0);
        a.out_u = ws(d.off_raw);
        a.out_v = ws(d.off_raw + 4 * n1);
        a.out_info = ws(d.off_info);
        a.plan = d.plan;
        a.strip = d.strip;
        TraceScope ts(h, st, "pass/" + stage_tag(h, d), geom_of(d.W, d.H, d.w, d.s, d.R, d.nx, d.ny, n));
        CK(launch_pass(a, n, st), "correlation pass launch");
        return RPIV_OK;
    };
    auto run_uod = [&](const StageDef &d, bool final_stage) -> rpiv_status {
        UodArgs u;
        const size_t n1 = (size_t)d.nx * d.ny;
        u.u = ws(d.off_raw);
        u.v = ws(d.off_raw + 4 * n1);
        u.info = ws(d.off_info);
        u.nx = d.nx;
        u.ny = d.ny;
        u.thr = c.uod_threshold;
        u.eps = c.uod_eps;
        u.replace = c.replace_outliers ? 1 : 0;
        if (final_stage) {
            u.u_out = tab(&io[0].u);
            u.v_out = tab(&io[0].v);
            u.mask = tab(&io[0].mask);
        } else {
            u.u_out = ws(d.off_out);
            u.v_out = ws(d.off_out + 4 * n1);
            u.mask = ws(d.off_mask);
        }
        TraceScope ts(h, st, "uod/" + stage_tag(h, d), geom_of(d.W, d.H, d.w, d.s, d.R, d.nx, d.ny, n));
        CK(launch_uod(u, n, st), "outlier test launch");
        return RPIV_OK;
    };
    auto run_interp = [&](const StageDef &src, PtrRef su, PtrRef sv, const StageDef &dst, int lv_up,
                          int zero_if_null) -> rpiv_status {
        InterpArgs ia;
        const size_t nd = (size_t)dst.nx * dst.ny;
        ia.su = su;
        ia.sv = sv;
        ia.snx = src.nx;
        ia.sny = src.ny;
        ia.sw = src.w;
        ia.ss = src.s;
        ia.du = ws(dst.off_pred);
        ia.dv = ws(dst.off_pred + 4 * nd);
        ia.dnx = dst.nx;
        ia.dny = dst.ny;
        ia.dw = dst.w;
        ia.ds = dst.s;
        ia.levels_up = lv_up;
        ia.zero_if_null = zero_if_null;
        TraceScope ts(h, st, "interp/" + stage_tag(h, dst),
                      geom_of(dst.W, dst.H, dst.w, dst.s, dst.R, dst.nx, dst.ny, n));
        CK(launch_interp(ia, n, st), "interpolation launch");
        return RPIV_OK;
    };
    rpiv_status rs;

    // the caller's frames: the pointer table entries, or (host frames) the
    // workspace copies the upload kernel makes of them first
    PtrRef img_a = tab(&io[0].a), img_b = tab(&io[0].b);
    long long img_pitch = (long long)pitch;
    if (c.host_frames) {
        UploadArgs ua;
        ua.src_a = img_a;
        ua.src_b = img_b;
        ua.pitch = (long long)pitch;
        ua.dst_a = ws(h->in_off[0]);
        ua.dst_b = ws(h->in_off[1]);
        ua.dst_pitch = h->in_pitch;
        ua.row_bytes = c.width * (user_fmt == PIX_U8 ? 1 : (user_fmt == PIX_U16 ? 2 : 4));
        ua.H = c.height;
        TraceScope ts(h, st, "upload", geom_of(c.width, c.height, 0, 0, 0, 0, 0, n));
        CK(launch_upload(ua, n, st), "upload launch");
        img_a = ua.dst_a;
        img_b = ua.dst_b;
        img_pitch = h->in_pitch;
    }

    bool pass0_pred = false;
    if (!central) {
        // frame A as float, read by every full-resolution pass
        IngestArgs ia;
        ia.src = img_a;
        ia.fmt = user_fmt;
        ia.pitch = img_pitch;
        ia.W = c.width;
        ia.H = c.height;
        ia.dst = ws(h->frame_off[0][0]);
        ia.dst_pitch = p0.fpitch;
        ia.dst_margin = M;
        TraceScope ts(h, st, "ingest", geom_of(c.width, c.height, 0, 0, 0, 0, 0, n));
        CK(launch_ingest(ia, n, st), "ingest launch");
    }
    if (run_pyr) {
        for (int l = 1; l <= L; ++l) {
            const StageDef &cur = h->stages[L - l];
            for (int ab = 0; ab < 2; ++ab) {
                DownArgs d;
                if (l == 1) {
                    d.src = ab ? img_b : img_a;
                    d.fmt = user_fmt;
                    d.pitch = img_pitch;
                    d.W = c.width;
                    d.H = c.height;
                } else {
                    const StageDef &prev = h->stages[L - (l - 1)];
                    d.src = ws(h->frame_off[l - 1][ab] + interior(prev.fpitch));
                    d.fmt = PIX_F32;
                    d.pitch = prev.fpitch * 4;
                    d.W = prev.W;
                    d.H = prev.H;
                }
                d.dst = ws(h->frame_off[l][ab]);
                d.dst_pitch = cur.fpitch;
                d.dst_margin = M;
                TraceScope ts(h, st, "down/L" + std::to_string(l), geom_of(d.W, d.H, 0, 0, 0, 0, 0, n));
                CK(launch_down(d, n, st), "pyramid launch");
            }
        }
        for (int i = 0; i < L; ++i) {
            const StageDef &d = h->stages[i];
            const bool pred = i > 0;
            if (pred) {
                const StageDef &prev = h->stages[i - 1];
                const size_t np = (size_t)prev.nx * prev.ny;
                if ((rs = run_interp(prev, ws(prev.off_out), ws(prev.off_out + 4 * np), d, 1, 0)) != RPIV_OK) return rs;
            }
            const size_t in = interior(d.fpitch);
            if ((rs = run_pass(d, ws(h->frame_off[d.lvl][0] + in), ws(h->frame_off[d.lvl][1] + in), PIX_F32,
                               d.fpitch * 4, ws(h->frame_off[d.lvl][0]), pred)) != RPIV_OK)
                return rs;
            if ((rs = run_uod(d, false)) != RPIV_OK) return rs;
        }
        const StageDef &l1 = h->stages[L - 1];
        const size_t n1 = (size_t)l1.nx * l1.ny;
        if ((rs = run_interp(l1, ws(l1.off_out), ws(l1.off_out + 4 * n1), p0, 1, 0)) != RPIV_OK) return rs;
        pass0_pred = true;
    }
    if (any_pred) {
        // caller predictor on the final-pass grid; pairs without one keep the
        // pyramid result, or get zero when there is no pyramid
        const StageDef &fin = h->stages.back();
        if ((rs = run_interp(fin, tab(&io[0].pred_u), tab(&io[0].pred_v), p0, 0, run_pyr ? 0 : 1)) != RPIV_OK)
            return rs;
        pass0_pred = true;
    }
    const int np = c.n_passes;
    for (int p = 0; p < np; ++p) {
        const StageDef &d = h->stages[L + p];
        bool pred = (p == 0) ? pass0_pred : true;
        if (p > 0) {
            const StageDef &prev = h->stages[L + p - 1];
            const size_t nprev = (size_t)prev.nx * prev.ny;
            if ((rs = run_interp(prev, ws(prev.off_out), ws(prev.off_out + 4 * nprev), d, 0, 0)) != RPIV_OK) return rs;
        }
        if ((rs = run_pass(d, img_a, img_b, user_fmt, img_pitch, ws(h->frame_off[0][0]),
                           pred)) != RPIV_OK)
            return rs;
        if ((rs = run_uod(d, p == np - 1)) != RPIV_OK) return rs;
        if (p < np - 1) {
            // the next pass reads this pass's validated field from the workspace
        }
    }
    const StageDef &fin = h->stages.back();
    VortArgs va;
    va.u = tab(&io[0].u);
    va.v = tab(&io[0].v);
    va.out = tab(&io[0].vort);
    va.nx = fin.nx;
    va.ny = fin.ny;
    va.s = fin.s;
    TraceScope ts(h, st, "vort", geom_of(fin.W, fin.H, fin.w, fin.s, fin.R, fin.nx, fin.ny, n));
    CK(launch_vort(va, n, st), "vorticity launch");
    return RPIV_OK;
}

}  // namespace

// ------------------------------------------------ one pass on caller scratch --

namespace {

// Error word of the stage entry points: bit 0 is set by a kernel whose bounded
// wait gave up (its windows were reported invalid); rpiv_stage_status reads and
// clears it.  A device variable, so that no call allocates for it.
__device__ int g_stage_err;

int *stage_err_word()
{
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_stage_err) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return static_cast<int *>(p);
}

// RPIV_DEBUG_STALL=1 (a tile's region wait) or 2 (a tensor-core tile's first
// MMA wait): the stage kernels wait on a phase that nothing completes, once
// nothing is in flight, with a short limit, so that the bounded waits and
// their reporting can be tested without a device fault.  Read per call.
int debug_stall()
{
    const char *e = std::getenv("RPIV_DEBUG_STALL");
    if (!e) return 0;
    const int v = std::atoi(e);
    return (v == 1 || v == 2) ? v : 0;
}

}  // namespace

size_t rpiv::single_pass_scratch_bytes(int W, int H, int R)
{
    const int M = frame_margin(R);
    return 2 * frame_bytes(W, H, M);  // frame A (or the warped A'), warped B'
}

int rpiv::single_pass(const void *img_a, const void *img_b, size_t pitch_bytes, int fmt, int width, int height,
                      int window, int step, int radius, int precision, int deform_mode, const float *pred_u,
                      const float *pred_v, float *u, float *v, int32_t *info, void *scratch, cudaStream_t st)
{
    if (!img_a || !img_b || !u || !v || !info || !scratch) return fail(RPIV_ERR_INVALID_ARG, "null argument");
    if (reinterpret_cast<uintptr_t>(scratch) % 256)
        return fail(RPIV_ERR_INVALID_ARG, "scratch must be 256-byte aligned");  // the pass copies 16-byte aligned rows
    if ((pred_u == nullptr) != (pred_v == nullptr)) return fail(RPIV_ERR_INVALID_ARG, "pred_u and pred_v: both or neither");
    if (fmt != 0 && fmt != RPIV_U8 && fmt != RPIV_U16) return fail(RPIV_ERR_INVALID_ARG, "fmt");
    if (window < 2 || step < 1 || radius < 0 || radius > RPIV_MAX_RADIUS)
        return fail(RPIV_ERR_INVALID_ARG, "window, step or radius out of range");
    if (width > 65536 || height > 65536) return fail(RPIV_ERR_INVALID_ARG, "image size out of range");
    if (width < window + 2 * (radius + 1) || height < window + 2 * (radius + 1))
        return fail(RPIV_ERR_INVALID_ARG, "image smaller than window + 2 (radius + 1)");
    const int bpp = fmt == RPIV_U8 ? 1 : (fmt == RPIV_U16 ? 2 : 4);
    if (pitch_bytes < (size_t)width * bpp || pitch_bytes % bpp) return fail(RPIV_ERR_INVALID_ARG, "pitch_bytes");
    if (precision != RPIV_FP32 && precision != RPIV_BF16 && precision != RPIV_FP16)
        return fail(RPIV_ERR_INVALID_ARG, "precision");
    if (deform_mode != RPIV_DEFORM_B && deform_mode != RPIV_DEFORM_CENTRAL)
        return fail(RPIV_ERR_INVALID_ARG, "deform_mode");
    const int nx = grid_n(width, window, step), ny = grid_n(height, window, step);
    if (!deform_nodes_fit(window, step, nx, ny)) return fail(RPIV_ERR_UNSUPPORTED, "step too small (minimum 3)");
    PassArgs a;
    std::memset(&a, 0, sizeof(a));
    a.prec = radius == 0 ? PREC_FP32 : prec_of((rpiv_precision)precision);
    if (!pass_plan(window, step, radius, nx, ny, a.prec, &a.plan, &a.strip))
        return fail(RPIV_ERR_UNSUPPORTED, "no kernel for this radius/precision/block size");
    const int M = frame_margin(radius);
    const long long fp = frame_pitch(width, M);
    const size_t one = frame_bytes(width, height, M);
    const bool central = deform_mode == RPIV_DEFORM_CENTRAL;
    char *first = static_cast<char *>(scratch);  // frame A, or A' for the central warp
    char *bdef = first + one;
    const int pfmt = fmt == RPIV_U8 ? PIX_U8 : (fmt == RPIV_U16 ? PIX_U16 : PIX_F32);
    prepare_pass_kernels();
    if (!central) {
        IngestArgs ia;
        ia.src = ptr_direct(img_a, 0);
        ia.fmt = pfmt;
        ia.pitch = (long long)pitch_bytes;
        ia.W = width;
        ia.H = height;
        ia.dst = ptr_direct(first, 0);
        ia.dst_pitch = fp;
        ia.dst_margin = M;
        CK(launch_ingest(ia, 1, st), "ingest launch");
    }
    for (int which = central ? 0 : 1; which < 2; ++which) {
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
        da.scale = central ? (which ? 0.5f : -0.5f) : 1.0f;
        da.M = M;
        da.out = ptr_direct(which ? bdef : first, 0);
        da.out_pitch = fp;
        CK(launch_deform(da, 1, st), "deformation launch");
    }
    a.W = width;
    a.H = height;
    a.fmt = pfmt;
    a.pitch = (long long)pitch_bytes;
    a.img_a = ptr_direct(img_a, 0);
    a.img_b = ptr_direct(img_b, 0);
    a.afl = ptr_direct(central ? nullptr : first, 0);
    a.bdef = ptr_direct(bdef, 0);
    a.adef = ptr_direct(central ? first : nullptr, 0);
    a.def_pitch = fp;
    a.def_margin = M;
    a.err = stage_err_word();
    a.dbg_stall = debug_stall();
    a.spin = a.dbg_stall ? 4096 : 0;
    a.w = window;
    a.s = step;
    a.R = radius;
    a.nx = nx;
    a.ny = ny;
    a.deform = central ? 1 : 0;
    a.pred_u = ptr_direct(pred_u, 0);
    a.pred_v = ptr_direct(pred_v, 0);
    a.out_u = ptr_direct(u, 0);
    a.out_v = ptr_direct(v, 0);
    a.out_info = ptr_direct(info, 0);
    CK(launch_pass(a, 1, st), "correlation pass launch");
    g_err.clear();
    return RPIV_OK;
}

// ===================================================================== ABI ==

extern "C" {

const char *rpiv_last_error(void) { return g_err.c_str(); }

rpiv_status rpiv_config_default(rpiv_config *cfg)
{
    if (!cfg) return fail(RPIV_ERR_INVALID_ARG, "cfg is NULL");
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->width = 1024;
    cfg->height = 1024;
    cfg->fmt = RPIV_U8;
    cfg->bit_depth = 8;
    cfg->n_passes = 1;
    cfg->window[0] = 16;
    cfg->overlap[0] = 0.5f;
    cfg->search_radius[0] = 1;
    cfg->predictor_levels = 0;
    cfg->uod_threshold = 2.0f;
    cfg->uod_eps = 0.1f;
    cfg->replace_outliers = 1;
    cfg->precision = RPIV_FP32;
    cfg->deform_mode = RPIV_DEFORM_B;
    cfg->max_batch = 1;
    cfg->host_frames = 0;
    g_err.clear();
    return RPIV_OK;
}

rpiv_status rpiv_validate_config(const rpiv_config *cfg, int *nx, int *ny)
{
    std::vector<StageDef> st;
    const std::string msg = check_config(cfg, &st);
    if (!msg.empty()) return fail(RPIV_ERR_INVALID_ARG, msg);
    if (nx) *nx = st.back().nx;
    if (ny) *ny = st.back().ny;
    g_err.clear();
    return RPIV_OK;
}

rpiv_status rpiv_create(const rpiv_config *cfg, int device, rpiv_handle **out)
{
    if (!out) return fail(RPIV_ERR_INVALID_ARG, "out is NULL");
    std::vector<StageDef> st;
    const std::string msg = check_config(cfg, &st);
    if (!msg.empty()) return fail(RPIV_ERR_INVALID_ARG, msg);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return fail(RPIV_ERR_NO_DEVICE, "no CUDA device");
    }
    if (device < 0 || device >= ndev) return fail(RPIV_ERR_INVALID_ARG, "device index out of range");
    DeviceGuard dg(device);
    prepare_pass_kernels();
    rpiv_handle *h = new rpiv_handle();
    h->cfg = *cfg;
    h->device = device;
    h->stages = st;
    // per-pair workspace layout
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = up(off + bytes, 256);
        return o;
    };
    {
        int Rmax = 0;
        for (auto &d : h->stages) Rmax = std::max(Rmax, d.R);
        const int M = frame_margin(Rmax);
        h->margin = M;
        for (auto &d : h->stages) d.fpitch = frame_pitch(d.W, M);
        const bool central = cfg->deform_mode == RPIV_DEFORM_CENTRAL;
        if (!central) h->frame_off[0][0] = take(frame_bytes(cfg->width, cfg->height, M));
        int W = cfg->width, H = cfg->height;
        for (int l = 1; l <= cfg->predictor_levels; ++l) {
            W /= 2;
            H /= 2;
            h->frame_off[l][0] = take(frame_bytes(W, H, M));
            h->frame_off[l][1] = take(frame_bytes(W, H, M));
        }
        // the warped frames of the largest stage serve every stage
        h->def_off[1] = take(frame_bytes(cfg->width, cfg->height, M));
        if (central) h->def_off[0] = take(frame_bytes(cfg->width, cfg->height, M));
        if (cfg->host_frames) {
            const int bpp = cfg->fmt == RPIV_U8 ? 1 : (cfg->fmt == RPIV_U16 ? 2 : 4);
            h->in_pitch = (long long)up((size_t)cfg->width * bpp, 16);
            h->in_off[0] = take((size_t)h->in_pitch * cfg->height);
            h->in_off[1] = take((size_t)h->in_pitch * cfg->height);
        }
    }
    for (auto &d : h->stages) {
        const size_t n1 = (size_t)d.nx * d.ny;
        d.off_pred = take(8 * n1);
        d.off_raw = take(8 * n1);
        d.off_info = take(4 * n1);
        d.off_out = take(8 * n1);
        d.off_mask = take(n1);
    }
    h->pair_stride = up(off, 256);
    h->ws_bytes = h->pair_stride * cfg->max_batch;
    auto cleanup = [&](rpiv_status s, const std::string &m) {
        rpiv_destroy(h);
        return fail(s, m);
    };
    cudaError_t e = cudaMalloc(&h->ws, h->ws_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cleanup(RPIV_ERR_OOM, "workspace allocation of " + std::to_string(h->ws_bytes) + " bytes failed");
    }
    // RPIV_POISON_SCRATCH=1 (a test setting) fills the workspace with NaN
    // bytes, so that any read of a value no kernel wrote shows up as NaN
    if (poison_scratch() && cudaMemset(h->ws, 0xFF, h->ws_bytes) != cudaSuccess)
        return cleanup(RPIV_ERR_CUDA, "workspace fill failed");
    e = cudaMalloc(&h->io_dev, sizeof(PairIO) * cfg->max_batch);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cleanup(RPIV_ERR_OOM, "pointer table allocation failed");
    }
    e = cudaMalloc(&h->err_dev, sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cleanup(RPIV_ERR_OOM, "error word allocation failed");
    }
    if ((e = cudaMemset(h->err_dev, 0, sizeof(int))) != cudaSuccess) return cleanup(RPIV_ERR_CUDA, "error word reset failed");
    e = cudaHostAlloc(&h->ring, sizeof(PairIO) * cfg->max_batch * kRing, cudaHostAllocDefault);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cleanup(RPIV_ERR_OOM, "pinned pointer ring allocation failed");
    }
    for (int i = 0; i < kRing; ++i)
        if ((e = cudaEventCreateWithFlags(&h->ring_ev[i], cudaEventDisableTiming)) != cudaSuccess)
            return cleanup(RPIV_ERR_CUDA, "event creation failed");
    if ((e = cudaEventCreateWithFlags(&h->done_ev, cudaEventDisableTiming)) != cudaSuccess)
        return cleanup(RPIV_ERR_CUDA, "event creation failed");
    if ((e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return cleanup(RPIV_ERR_CUDA, "stream creation failed");
    for (int i = 1; i < rpiv_handle::kParts; ++i) {
        if ((e = cudaStreamCreateWithFlags(&h->cap_part[i], cudaStreamNonBlocking)) != cudaSuccess)
            return cleanup(RPIV_ERR_CUDA, "stream creation failed");
        if ((e = cudaEventCreateWithFlags(&h->join_ev[i], cudaEventDisableTiming)) != cudaSuccess)
            return cleanup(RPIV_ERR_CUDA, "event creation failed");
    }
    if ((e = cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming)) != cudaSuccess)
        return cleanup(RPIV_ERR_CUDA, "event creation failed");
    *out = h;
    g_err.clear();
    return RPIV_OK;
}

rpiv_status rpiv_grid_shape(const rpiv_handle *h, int *nx, int *ny)
{
    if (!h || !nx || !ny) return fail(RPIV_ERR_INVALID_ARG, "null argument");
    *nx = h->stages.back().nx;
    *ny = h->stages.back().ny;
    return RPIV_OK;
}

rpiv_status rpiv_workspace_bytes(const rpiv_handle *h, size_t *bytes)
{
    if (!h || !bytes) return fail(RPIV_ERR_INVALID_ARG, "null argument");
    *bytes = h->ws_bytes + sizeof(PairIO) * h->cfg.max_batch + h->adj_bytes;
    return RPIV_OK;
}

// Captured batches of 16 pairs and more run as parts of at least 8 pairs on
// forked streams, two by default (RPIV_SPLIT_BATCH = 1, 2 or 4 parts; read
// when a batch shape is captured).  Measured on the 64-pair 1 MP workload:
// one chain 13420, two parts 13664-13690, four parts 13346 pairs/s.
static int split_parts(int n)
{
    int parts = 2;
    if (const char *e = std::getenv("RPIV_SPLIT_BATCH")) {
        const int v = std::atoi(e);
        parts = (v == 1 || v == 2 || v == 4) ? v : (v == 0 ? 1 : 2);
    }
    while (parts > 1 && n / parts < 8) parts /= 2;
    return parts;
}

rpiv_status rpiv_process_batch(rpiv_handle *h, int n, const void *const *img_a, const void *const *img_b,
                               size_t pitch_bytes, const float *const *pred_u, const float *const *pred_v,
                               float *const *u, float *const *v, float *const *vort, uint8_t *const *mask,
                               void *cuda_stream)
{
    if (!h) return fail(RPIV_ERR_INVALID_ARG, "handle is NULL");
    if (n < 1 || n > h->cfg.max_batch)
        return fail(RPIV_ERR_INVALID_ARG, "n = " + std::to_string(n) + " outside [1, max_batch = " +
                                              std::to_string(h->cfg.max_batch) + "]");
    if (!img_a || !img_b || !u || !v) return fail(RPIV_ERR_INVALID_ARG, "img_a, img_b, u and v must be non-NULL");
    const size_t bpp = h->cfg.fmt == RPIV_U8 ? 1 : (h->cfg.fmt == RPIV_U16 ? 2 : 4);
    if (pitch_bytes < (size_t)h->cfg.width * bpp || pitch_bytes % bpp)
        return fail(RPIV_ERR_INVALID_ARG, "pitch_bytes smaller than width * bytes per pixel or misaligned");
    if ((pred_u == nullptr) != (pred_v == nullptr)) return fail(RPIV_ERR_INVALID_ARG, "pred_u and pred_v: both or neither");
    bool any_pred = false, any_nopred = false;
    for (int i = 0; i < n; ++i) {
        if (!img_a[i] || !img_b[i] || !u[i] || !v[i])
            return fail(RPIV_ERR_INVALID_ARG, "NULL image or output pointer for pair " + std::to_string(i));
        const bool hp = pred_u && pred_u[i];
        if (pred_u && ((pred_u[i] == nullptr) != (pred_v[i] == nullptr)))
            return fail(RPIV_ERR_INVALID_ARG, "pred_u/pred_v of pair " + std::to_string(i) + ": both or neither");
        if (hp) any_pred = true;
        else any_nopred = true;
    }
    DeviceGuard dg(h->device);
    if (h->cfg.host_frames) {
        // the upload kernel reads the frames through their host addresses
        for (int i = 0; i < n; ++i)
            for (const void *p : {img_a[i], img_b[i]}) {
                cudaPointerAttributes at;
                if (cudaPointerGetAttributes(&at, p) != cudaSuccess || at.type != cudaMemoryTypeHost) {
                    cudaGetLastError();
                    return fail(RPIV_ERR_INVALID_ARG, "host_frames: the image of pair " + std::to_string(i) +
                                                          " is not page-locked host memory");
                }
            }
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // pointer table for this call, staged in a pinned ring slot
    const int slot = h->ring_pos;
    h->ring_pos = (h->ring_pos + 1) % kRing;
    if (h->ring_used[slot]) CK(cudaEventSynchronize(h->ring_ev[slot]), "pointer ring wait");
    PairIO *tabh = h->ring + (size_t)slot * h->cfg.max_batch;
    for (int i = 0; i < n; ++i) {
        tabh[i].a = img_a[i];
        tabh[i].b = img_b[i];
        tabh[i].pred_u = pred_u ? pred_u[i] : nullptr;
        tabh[i].pred_v = pred_v ? pred_v[i] : nullptr;
        tabh[i].u = u[i];
        tabh[i].v = v[i];
        tabh[i].vort = vort ? vort[i] : nullptr;
        tabh[i].mask = mask ? mask[i] : nullptr;
    }
    // one call at a time on the device per handle (shared workspace)
    if (h->done_recorded) CK(cudaStreamWaitEvent(st, h->done_ev, 0), "ordering wait");
    CK(cudaMemcpyAsync(h->io_dev, tabh, sizeof(PairIO) * n, cudaMemcpyHostToDevice, st), "pointer table copy");
    CK(cudaEventRecord(h->ring_ev[slot], st), "event record");
    h->ring_used[slot] = true;
    // launch sequence: captured once per (n, predictor pattern, pitch), then replayed
    char keybuf[96];
    std::snprintf(keybuf, sizeof(keybuf), "%d/%d/%d/%zu", n, (int)any_pred, (int)any_nopred, pitch_bytes);
    const std::string key(keybuf);
    auto it = h->graphs.find(key);
    if (h->tracing) {
        rpiv_status rs = enqueue_schedule(h, n, pitch_bytes, any_pred, any_nopred, st);
        if (rs != RPIV_OK) return rs;
    } else if (it == h->graphs.end()) {
        // first use of this shape: run eagerly, then capture the same sequence
        // on the handle's private stream for later replays
        rpiv_status rs = enqueue_schedule(h, n, pitch_bytes, any_pred, any_nopred, st);
        if (rs != RPIV_OK) return rs;
        cudaGraph_t graph = nullptr;
        CK(cudaStreamSynchronize(st), "first-run synchronise");
        CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        const int parts = split_parts(n);
        if (parts > 1) {
            // independent parts on forked streams of one graph: one part's small
            // launches and wave tails overlap the others' large passes
            cudaError_t fe = cudaEventRecord(h->fork_ev, h->cap_stream);
            int forked = 1;
            for (; fe == cudaSuccess && forked < parts; ++forked)
                fe = cudaStreamWaitEvent(h->cap_part[forked], h->fork_ev, 0);
            if (fe != cudaSuccess) --forked;
            rs = fe == cudaSuccess ? RPIV_OK : cuda_fail(fe, "capture fork");
            for (int i = 0, first = 0; i < parts && rs == RPIV_OK; ++i) {
                const int cnt = n / parts + (i < n % parts ? 1 : 0);
                rs = enqueue_schedule(h, cnt, pitch_bytes, any_pred, any_nopred, i ? h->cap_part[i] : h->cap_stream,
                                      first);
                first += cnt;
            }
            // the joins also end the forked streams' parts of the capture on every path
            for (int i = 1; i < forked; ++i) {
                cudaError_t je = cudaEventRecord(h->join_ev[i], h->cap_part[i]);
                if (je == cudaSuccess) je = cudaStreamWaitEvent(h->cap_stream, h->join_ev[i], 0);
                if (je != cudaSuccess && rs == RPIV_OK) rs = cuda_fail(je, "capture join");
            }
        } else {
            rs = enqueue_schedule(h, n, pitch_bytes, any_pred, any_nopred, h->cap_stream);
        }
        cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &graph);
        if (rs != RPIV_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rs;
        }
        if (ce != cudaSuccess) return cuda_fail(ce, "end capture");
        cudaGraphExec_t exec = nullptr;
        ce = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return cuda_fail(ce, "graph instantiate");
        h->graphs[key] = exec;
    } else {
        CK(cudaGraphLaunch(it->second, st), "graph launch");
    }
    CK(cudaEventRecord(h->done_ev, st), "event record");
    h->done_recorded = true;
    return RPIV_OK;
}

rpiv_status rpiv_process_pair(rpiv_handle *h, const void *img_a, const void *img_b, size_t pitch_bytes,
                              const float *pred_u, const float *pred_v, float *u, float *v, float *vort,
                              uint8_t *mask, void *cuda_stream)
{
    if ((pred_u == nullptr) != (pred_v == nullptr)) return fail(RPIV_ERR_INVALID_ARG, "pred_u and pred_v: both or neither");
    const void *a[1] = {img_a}, *b[1] = {img_b};
    const float *pu[1] = {pred_u}, *pv[1] = {pred_v};
    float *uu[1] = {u}, *vv[1] = {v}, *oo[1] = {vort};
    uint8_t *mm[1] = {mask};
    return rpiv_process_batch(h, 1, a, b, pitch_bytes, pred_u ? pu : nullptr, pred_v ? pv : nullptr, uu, vv, oo, mm,
                              cuda_stream);
}

rpiv_status rpiv_backward(rpiv_handle *h, const void *img_a, const void *img_b, size_t pitch_bytes, const float *u,
                          const float *v, float grad_score, float *grad_u, float *grad_v, float *score_out,
                          void *cuda_stream)
{
    if (!h || !img_a || !img_b || !u || !v) return fail(RPIV_ERR_INVALID_ARG, "null argument");
    if ((grad_u == nullptr) != (grad_v == nullptr)) return fail(RPIV_ERR_INVALID_ARG, "grad_u and grad_v: both or neither");
    const size_t bpp = h->cfg.fmt == RPIV_U8 ? 1 : (h->cfg.fmt == RPIV_U16 ? 2 : 4);
    if (pitch_bytes < (size_t)h->cfg.width * bpp || pitch_bytes % bpp)
        return fail(RPIV_ERR_INVALID_ARG, "pitch_bytes smaller than width * bytes per pixel or misaligned");
    DeviceGuard dg(h->device);
    const StageDef &d = h->stages[h->cfg.predictor_levels];  // first full-resolution pass grid
    const size_t need = adjoint_workspace_bytes(d.W, d.H, d.w, d.s, d.nx, d.ny);
    if (h->adj_bytes < need) {
        // allocated on first use (not inside a stream capture)
        if (h->adj_ws) {
            cudaDeviceSynchronize();
            cudaFree(h->adj_ws);
            h->adj_ws = nullptr;
            h->adj_bytes = 0;
        }
        if (cudaMalloc(&h->adj_ws, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(RPIV_ERR_OOM, "adjoint workspace allocation failed");
        }
        h->adj_bytes = need;
        if (poison_scratch() && cudaMemset(h->adj_ws, 0xFF, need) != cudaSuccess)
            return fail(RPIV_ERR_CUDA, "adjoint workspace fill failed");
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (h->done_recorded) CK(cudaStreamWaitEvent(st, h->done_ev, 0), "ordering wait");
    AdjArgs a;
    std::memset(&a, 0, sizeof(a));
    a.W = d.W;
    a.H = d.H;
    a.fmt = h->cfg.fmt == RPIV_U8 ? PIX_U8 : (h->cfg.fmt == RPIV_U16 ? PIX_U16 : PIX_F32);
    a.pitch = (long long)pitch_bytes;
    a.img_a = ptr_direct(img_a, 0);
    a.img_b = ptr_direct(img_b, 0);
    a.w = d.w;
    a.s = d.s;
    a.nx = d.nx;
    a.ny = d.ny;
    a.u = u;
    a.v = v;
    a.ws = h->adj_ws;
    a.grad_scale = grad_score;
    a.grad_u = grad_u;
    a.grad_v = grad_v;
    a.score_out = score_out;
    CK(launch_adjoint(a, st), "adjoint launch");
    CK(cudaEventRecord(h->done_ev, st), "event record");
    h->done_recorded = true;
    return RPIV_OK;
}

rpiv_status rpiv_refine(rpiv_handle *h, const void *img_a, const void *img_b, size_t pitch_bytes, float *u, float *v,
                        int steps, float eta0, int halvings, float *hist, void *cuda_stream)
{
    if (!h || !img_a || !img_b || !u || !v) return fail(RPIV_ERR_INVALID_ARG, "null argument");
    if (steps < 0 || halvings < 0 || !(eta0 > 0.f)) return fail(RPIV_ERR_INVALID_ARG, "steps, halvings >= 0, eta0 > 0");
    DeviceGuard dg(h->device);
    const StageDef &d = h->stages[h->cfg.predictor_levels];
    const size_t n = (size_t)d.nx * d.ny;
    if (h->ref_n < n) {
        if (h->ref_ws) {
            cudaDeviceSynchronize();
            cudaFree(h->ref_ws);
            h->ref_ws = nullptr;
            h->ref_n = 0;
        }
        if (cudaMalloc(&h->ref_ws, sizeof(float) * (4 * n + 64)) != cudaSuccess) {
            cudaGetLastError();
            return fail(RPIV_ERR_OOM, "refinement buffers allocation failed");
        }
        h->ref_n = n;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    float *gu = h->ref_ws, *gv = gu + n, *cu = gv + n, *cv = cu + n, *dS = cv + n, *dgmax = dS + 32;
    auto read = [&](const float *src, float *dst) -> rpiv_status {
        CK(cudaMemcpyAsync(dst, src, sizeof(float), cudaMemcpyDeviceToHost, st), "score read");
        CK(cudaStreamSynchronize(st), "score read");
        return RPIV_OK;
    };
    rpiv_status rs;
    float S = 0.f, gmax = 0.f;
    if ((rs = rpiv_backward(h, img_a, img_b, pitch_bytes, u, v, 1.0f, gu, gv, dS, cuda_stream)) != RPIV_OK) return rs;
    CK(launch_refine_absmax(gu, gv, (int)n, dgmax, st), "gradient maximum launch");
    if ((rs = read(dS, &S)) != RPIV_OK || (rs = read(dgmax, &gmax)) != RPIV_OK) return rs;
    if (hist) hist[0] = S;
    for (int k = 0; k < steps; ++k) {
        if (gmax > 0.f) {
            double eta = (double)eta0 * std::ldexp(1.0, -k) / (double)gmax;
            for (int t = 0; t <= halvings; ++t, eta *= 0.5) {
                CK(launch_refine_axpy(u, v, gu, gv, (float)eta, cu, cv, (int)n, st), "step launch");
                if ((rs = rpiv_backward(h, img_a, img_b, pitch_bytes, cu, cv, 1.0f, nullptr, nullptr, dS,
                                        cuda_stream)) != RPIV_OK)
                    return rs;
                float Sc = 0.f;
                if ((rs = read(dS, &Sc)) != RPIV_OK) return rs;
                if (Sc > S) {
                    CK(cudaMemcpyAsync(u, cu, sizeof(float) * n, cudaMemcpyDeviceToDevice, st), "step copy");
                    CK(cudaMemcpyAsync(v, cv, sizeof(float) * n, cudaMemcpyDeviceToDevice, st), "step copy");
                    break;
                }
            }
        }
        if ((rs = rpiv_backward(h, img_a, img_b, pitch_bytes, u, v, 1.0f, gu, gv, dS, cuda_stream)) != RPIV_OK)
            return rs;
        if ((rs = read(dS, &S)) != RPIV_OK) return rs;
        if (hist) hist[k + 1] = S;
    }
    g_err.clear();
    return RPIV_OK;
}

rpiv_status rpiv_wait(rpiv_handle *h, int timeout_ms)
{
    if (!h) return fail(RPIV_ERR_INVALID_ARG, "handle is NULL");
    if (!h->done_recorded) return RPIV_OK;
    DeviceGuard dg(h->device);
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t e = cudaEventQuery(h->done_ev);
        if (e == cudaSuccess) {
            // a kernel whose bounded wait gave up reported its tiles invalid and set the word
            int err = 0;
            cudaError_t e2 = cudaMemcpyAsync(&err, h->err_dev, sizeof(int), cudaMemcpyDeviceToHost, h->cap_stream);
            if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(h->cap_stream);
            if (e2 != cudaSuccess) return cuda_fail(e2, "error word read");
            if (err) {
                cudaMemsetAsync(h->err_dev, 0, sizeof(int), h->cap_stream);
                cudaStreamSynchronize(h->cap_stream);
                return fail(RPIV_ERR_TIMEOUT, "a tile's region load did not complete within its bounded wait; "
                                              "its windows were reported invalid");
            }
            return RPIV_OK;
        }
        if (e != cudaErrorNotReady) return cuda_fail(e, "event query");
        const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0);
        if (ms.count() >= timeout_ms) return fail(RPIV_ERR_TIMEOUT, "work did not finish within the timeout");
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
}

rpiv_status rpiv_stage_status(void *cuda_stream, int timeout_ms)
{
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t e = cudaStreamQuery(st);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return cuda_fail(e, "stream query");
        const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0);
        if (ms.count() >= timeout_ms) return fail(RPIV_ERR_TIMEOUT, "stage work did not finish within the timeout");
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    int err = 0;
    const int zero = 0;
    CK(cudaMemcpyFromSymbolAsync(&err, g_stage_err, sizeof(int), 0, cudaMemcpyDeviceToHost, st), "error word read");
    CK(cudaStreamSynchronize(st), "error word read");
    if (err) {
        CK(cudaMemcpyToSymbolAsync(g_stage_err, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st), "error word reset");
        CK(cudaStreamSynchronize(st), "error word reset");
        return fail(RPIV_ERR_TIMEOUT, "a stage kernel's bounded wait gave up; its windows were reported invalid");
    }
    g_err.clear();
    return RPIV_OK;
}

rpiv_status rpiv_trace_enable(rpiv_handle *h, int enable)
{
    if (!h) return fail(RPIV_ERR_INVALID_ARG, "handle is NULL");
    h->tracing = enable != 0;
    return RPIV_OK;
}

rpiv_status rpiv_trace_read(rpiv_handle *h, rpiv_trace_record *out, int cap, int *n)
{
    if (!h || !n || (cap > 0 && !out)) return fail(RPIV_ERR_INVALID_ARG, "null argument");
    DeviceGuard dg(h->device);
    std::vector<rpiv_trace_record> recs;
    std::map<std::string, size_t> index;
    for (auto &t : h->trace_evs) {
        CK(cudaEventSynchronize(t.t1), "trace synchronise");
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, t.t0, t.t1), "trace elapsed time");
        auto it = index.find(t.name);
        if (it == index.end()) {
            rpiv_trace_record r = t.geom;
            std::snprintf(r.name, sizeof(r.name), "%s", t.name.c_str());
            r.launches = 0;
            r.total_ms = 0.f;
            index[t.name] = recs.size();
            recs.push_back(r);
            it = index.find(t.name);
        }
        recs[it->second].launches += 1;
        recs[it->second].total_ms += ms;
        h->ev_pool.push_back(t.t0);
        h->ev_pool.push_back(t.t1);
    }
    h->trace_evs.clear();
    *n = (int)recs.size();
    for (int i = 0; i < cap && i < (int)recs.size(); ++i) out[i] = recs[i];
    return RPIV_OK;
}

rpiv_status rpiv_destroy(rpiv_handle *h)
{
    if (!h) return RPIV_OK;
    {
        DeviceGuard dg(h->device);
        if (h->done_ev && h->done_recorded) cudaEventSynchronize(h->done_ev);
        for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second);
        for (auto &t : h->trace_evs) {
            cudaEventDestroy(t.t0);
            cudaEventDestroy(t.t1);
        }
        for (auto e : h->ev_pool) cudaEventDestroy(e);
        for (int i = 0; i < kRing; ++i)
            if (h->ring_ev[i]) cudaEventDestroy(h->ring_ev[i]);
        if (h->done_ev) cudaEventDestroy(h->done_ev);
        if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
        for (int i = 1; i < rpiv_handle::kParts; ++i) {
            if (h->cap_part[i]) cudaStreamDestroy(h->cap_part[i]);
            if (h->join_ev[i]) cudaEventDestroy(h->join_ev[i]);
        }
        if (h->fork_ev) cudaEventDestroy(h->fork_ev);
        if (h->ws) cudaFree(h->ws);
        if (h->err_dev) cudaFree(h->err_dev);
        if (h->ref_ws) cudaFree(h->ref_ws);
        if (h->io_dev) cudaFree(h->io_dev);
        if (h->ring) cudaFreeHost(h->ring);
        if (h->adj_ws) cudaFree(h->adj_ws);
        cudaGetLastError();
    }
    delete h;
    return RPIV_OK;
}

// -------------------------------------------------------- stage entries --

rpiv_status rpiv_stage_correlate_scratch_bytes(int width, int height, int radius, rpiv_deform deform_mode,
                                               size_t *bytes)
{
    if (!bytes || width < 1 || height < 1 || width > 65536 || height > 65536 || radius < 0 ||
        radius > RPIV_MAX_RADIUS)
        return fail(RPIV_ERR_INVALID_ARG, "bad argument");
    if (deform_mode != RPIV_DEFORM_B && deform_mode != RPIV_DEFORM_CENTRAL)
        return fail(RPIV_ERR_INVALID_ARG, "deform_mode");
    *bytes = single_pass_scratch_bytes(width, height, radius);
    return RPIV_OK;
}

rpiv_status rpiv_stage_correlate(const void *img_a, const void *img_b, size_t pitch_bytes, int fmt, int width,
                                 int height, int window, int step, int radius, rpiv_precision precision,
                                 rpiv_deform deform_mode, const float *pred_u, const float *pred_v, float *u,
                                 float *v, int32_t *info, void *scratch, size_t scratch_bytes, void *cuda_stream)
{
    if (!scratch) return fail(RPIV_ERR_INVALID_ARG, "null argument");
    if (width < 1 || height < 1 || width > 65536 || height > 65536 || radius < 0 || radius > RPIV_MAX_RADIUS)
        return fail(RPIV_ERR_INVALID_ARG, "image size or radius out of range");
    if (scratch_bytes < single_pass_scratch_bytes(width, height, radius))
        return fail(RPIV_ERR_INVALID_ARG, "scratch smaller than rpiv_stage_correlate_scratch_bytes");
    return (rpiv_status)single_pass(img_a, img_b, pitch_bytes, fmt, width, height, window, step, radius,
                                    (int)precision, (int)deform_mode, pred_u, pred_v, u, v, info, scratch,
                                    static_cast<cudaStream_t>(cuda_stream));
}

rpiv_status rpiv_stage_validate(const float *u, const float *v, const int32_t *info, int nx, int ny, float threshold,
                                float eps, int replace, float *u_out, float *v_out, uint8_t *mask, void *cuda_stream)
{
    if (!u || !v || !u_out || !v_out || nx < 1 || ny < 1) return fail(RPIV_ERR_INVALID_ARG, "null argument or empty grid");
    if (u == u_out || v == v_out) return fail(RPIV_ERR_INVALID_ARG, "input and output must not alias");
    UodArgs a;
    a.u = ptr_direct(u, 0);
    a.v = ptr_direct(v, 0);
    a.info = ptr_direct(info, 0);
    a.nx = nx;
    a.ny = ny;
    a.thr = threshold;
    a.eps = eps;
    a.replace = replace ? 1 : 0;
    a.u_out = ptr_direct(u_out, 0);
    a.v_out = ptr_direct(v_out, 0);
    a.mask = ptr_direct(mask, 0);
    CK(launch_uod(a, 1, static_cast<cudaStream_t>(cuda_stream)), "outlier test launch");
    return RPIV_OK;
}

rpiv_status rpiv_stage_interp(const float *su, const float *sv, int snx, int sny, int sw, int ss, float *du,
                              float *dv, int dnx, int dny, int dw, int ds, int levels_up, void *cuda_stream)
{
    if (!su || !sv || !du || !dv || snx < 1 || sny < 1 || dnx < 1 || dny < 1 || ss < 1 || ds < 1 || levels_up < 0 ||
        levels_up > 8)
        return fail(RPIV_ERR_INVALID_ARG, "bad argument");
    InterpArgs a;
    a.su = ptr_direct(su, 0);
    a.sv = ptr_direct(sv, 0);
    a.snx = snx;
    a.sny = sny;
    a.sw = sw;
    a.ss = ss;
    a.du = ptr_direct(du, 0);
    a.dv = ptr_direct(dv, 0);
    a.dnx = dnx;
    a.dny = dny;
    a.dw = dw;
    a.ds = ds;
    a.levels_up = levels_up;
    a.zero_if_null = 0;
    CK(launch_interp(a, 1, static_cast<cudaStream_t>(cuda_stream)), "interpolation launch");
    return RPIV_OK;
}

rpiv_status rpiv_stage_vorticity(const float *u, const float *v, int nx, int ny, int step, float *vort,
                                 void *cuda_stream)
{
    if (!u || !v || !vort || nx < 1 || ny < 1 || step < 1) return fail(RPIV_ERR_INVALID_ARG, "bad argument");
    VortArgs a;
    a.u = ptr_direct(u, 0);
    a.v = ptr_direct(v, 0);
    a.out = ptr_direct(vort, 0);
    a.nx = nx;
    a.ny = ny;
    a.s = step;
    CK(launch_vort(a, 1, static_cast<cudaStream_t>(cuda_stream)), "vorticity launch");
    return RPIV_OK;
}

rpiv_status rpiv_stage_preprocess_scratch_bytes(int width, int height, int tiles_x, int tiles_y, size_t *bytes)
{
    if (!bytes || width < 1 || height < 1 || width > 65536 || height > 65536 || tiles_x < 1 || tiles_y < 1 ||
        tiles_x > 64 || tiles_y > 64)
        return fail(RPIV_ERR_INVALID_ARG, "bad argument");
    *bytes = preprocess_scratch_bytes(width, height, tiles_x, tiles_y);
    return RPIV_OK;
}

rpiv_status rpiv_stage_preprocess(const void *img, size_t pitch_bytes, int fmt, int width, int height, int vmax,
                                  int hp_radius, int tiles_x, int tiles_y, int clip_percent, float *out,
                                  void *scratch, size_t scratch_bytes, void *cuda_stream)
{
    if (!img || !out || !scratch) return fail(RPIV_ERR_INVALID_ARG, "null argument");
    if (fmt != RPIV_U8 && fmt != RPIV_U16) return fail(RPIV_ERR_INVALID_ARG, "fmt must be RPIV_U8 or RPIV_U16");
    if (width < 1 || height < 1 || width > 65536 || height > 65536) return fail(RPIV_ERR_INVALID_ARG, "image size");
    const size_t bpp = fmt == RPIV_U8 ? 1 : 2;
    if (pitch_bytes < (size_t)width * bpp || pitch_bytes % bpp) return fail(RPIV_ERR_INVALID_ARG, "pitch_bytes");
    if (vmax < 1 || vmax > 65535) return fail(RPIV_ERR_INVALID_ARG, "vmax must be in [1, 65535]");
    if (hp_radius < 0 || hp_radius > 64) return fail(RPIV_ERR_INVALID_ARG, "hp_radius must be in [0, 64]");
    if (tiles_x < 1 || tiles_y < 1 || tiles_x > 64 || tiles_y > 64 || tiles_x > width || tiles_y > height)
        return fail(RPIV_ERR_INVALID_ARG, "tiles must be in [1, 64] and no more than the image size");
    if (clip_percent < 0) return fail(RPIV_ERR_INVALID_ARG, "clip_percent must be >= 0");
    if (scratch_bytes < preprocess_scratch_bytes(width, height, tiles_x, tiles_y))
        return fail(RPIV_ERR_INVALID_ARG, "scratch smaller than rpiv_stage_preprocess_scratch_bytes");
    PreArgs a;
    a.img = img;
    a.fmt = fmt == RPIV_U8 ? PIX_U8 : PIX_U16;
    a.pitch = (long long)pitch_bytes;
    a.W = width;
    a.H = height;
    a.vmax = vmax;
    a.hp = hp_radius;
    a.n = hp_radius > 0 ? (2 * hp_radius + 1) * (2 * hp_radius + 1) : 1;
    a.tx = tiles_x;
    a.ty = tiles_y;
    a.clip_pct = clip_percent;
    a.out = out;
    a.out_pitch = width;
    CK(launch_preprocess(a, scratch, static_cast<cudaStream_t>(cuda_stream)), "pre-processing launch");
    return RPIV_OK;
}

rpiv_status rpiv_stage_ema(const float *x, float *state, size_t n, float alpha, int init, void *cuda_stream)
{
    if (n > 0 && (!x || !state)) return fail(RPIV_ERR_INVALID_ARG, "null argument");
    if (!(alpha >= 0.f && alpha <= 1.f)) return fail(RPIV_ERR_INVALID_ARG, "alpha must be in [0, 1]");
    if (x != state && x < state + n && state < x + n) return fail(RPIV_ERR_INVALID_ARG, "x and state overlap");
    CK(launch_ema(x, state, n, alpha, init, static_cast<cudaStream_t>(cuda_stream)), "smoothing launch");
    return RPIV_OK;
}

rpiv_status rpiv_stage_downsample(const void *img, size_t pitch_bytes, int fmt, int width, int height, float *out,
                                  void *cuda_stream)
{
    if (!img || !out || width < 2 || height < 2) return fail(RPIV_ERR_INVALID_ARG, "bad argument");
    if (fmt != 0 && fmt != RPIV_U8 && fmt != RPIV_U16) return fail(RPIV_ERR_INVALID_ARG, "fmt");
    const int bpp = fmt == RPIV_U8 ? 1 : (fmt == RPIV_U16 ? 2 : 4);
    if (pitch_bytes < (size_t)width * bpp) return fail(RPIV_ERR_INVALID_ARG, "pitch_bytes");
    DownArgs a;
    a.src = ptr_direct(img, 0);
    a.fmt = fmt == RPIV_U8 ? PIX_U8 : (fmt == RPIV_U16 ? PIX_U16 : PIX_F32);
    a.pitch = (long long)pitch_bytes;
    a.W = width;
    a.H = height;
    a.dst = ptr_direct(out, 0);
    a.dst_pitch = width / 2;
    a.dst_margin = 0;
    CK(launch_down(a, 1, static_cast<cudaStream_t>(cuda_stream)), "downsample launch");
    return RPIV_OK;
}

}  // extern "C"
