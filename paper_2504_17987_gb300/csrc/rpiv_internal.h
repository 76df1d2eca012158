// Internal interfaces between the host engine (engine.cpp, capi.cpp) and the
// CUDA kernels (k_*.cu).  Not part of the public ABI (see include/rpiv.h).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda.h>
#include <cuda_runtime.h>

namespace rpiv {

enum PixFmt : int { PIX_F32 = 0, PIX_U8 = 1, PIX_U16 = 2 };
enum Prec : int { PREC_FP32 = 0, PREC_BF16 = 1, PREC_FP16 = 2 };

// Per-pair pointers of one batch call, mirrored into device memory.
struct PairIO {
    const void *a;
    const void *b;
    const float *pred_u;
    const float *pred_v;
    float *u;
    float *v;
    float *vort;
    uint8_t *mask;
};

// A per-pair pointer: either direct (base + pair * stride) or read from a
// device table (entry at base + pair * stride holds the pointer).
struct PtrRef {
    const char *base;
    long long stride;
    int indirect;
};

__host__ __device__ inline PtrRef ptr_direct(const void *p, long long stride)
{
    PtrRef r;
    r.base = static_cast<const char *>(p);
    r.stride = stride;
    r.indirect = 0;
    return r;
}

__host__ __device__ inline PtrRef ptr_table(const void *entry0, long long stride)
{
    PtrRef r;
    r.base = static_cast<const char *>(entry0);
    r.stride = stride;
    r.indirect = 1;
    return r;
}

#ifdef __CUDACC__
__device__ __forceinline__ const void *resolve(const PtrRef &r, int pair)
{
    if (r.base == nullptr) return nullptr;
    const char *p = r.base + (long long)pair * r.stride;
    if (r.indirect) return *reinterpret_cast<const void *const *>(p);
    return p;
}
#endif

// ------------------------------------------------------------ pass kernel --

struct PassPlan {
    // tiling
    int TX, TY, tiles_x, tiles_y, threads;
    int G;    // block size of the block-decomposed correlation (= gcd(w, s))
    int strip_rows;  // > 0: each CTA walks this many window rows of a one-row tile, keeping
                     // the previous block row's planes (tiles_y counts the strip segments)
    int RGx;      // row groups per block in the plane phase
    int pstride;  // floats between consecutive blocks' planes
    int box_lv, box_lh;  // outputs per running sum in the column and row box-sum passes
    int box_nv, box_nh;  // running sums per column and per row of a full tile (edge tiles skip the ones past their end)
    // shared-memory layout (byte offsets) for a full tile
    int smem_bytes;
    int off_a, a_pitch;          // A region, floats
    int off_b, b_pitch, padl;    // B' region, floats; logical column 0 at padl - (R+1)
    int off_h, h_pitch;          // C: column box sums, (S1, S2) float pairs; odd pitch >= BC, in pairs
    int off_v, v_pitch;          // V: window box sums, (S1, 1 / sqrt of the box energy) float pairs; odd pitch >= hw, in pairs
    int off_p;                   // block planes (aliases H; a two-row ring of its own in strips)
    int off_tca, tca_pitch;      // 16-bit A copy (TC path; aliases H), elements
    int off_tcb, tcb_pitch;      // two 16-bit B' copies (TC path; aliases H), elements
    int tb_rows, tb_cols;        // rows of each B' copy, columns written
    int off_stats;               // per-window mean / energy of A
    int off_red;                 // mbarrier of the bulk region loads
    int off_gst;                 // per-G x G block sum and centred sum of squares of A
    int off_c5, off_peaks, off_need, off_dpart;  // per-window stencil values, argmax, direct-sum mask and sums
    int max_windows, max_blocks;
    // tcgen05 planes (tc = 1; BF16/FP16, 50 % overlap, r = 4): two zero-banded A
    // slabs (window rows), a ring of tc_nbuf slots of shifted B' copies (one MMA
    // group of rows each), an epilogue buffer, tmem_cols TMEM columns (two rows)
    int tc;
    int off_slab, slab_rows, slab_lbo;  // bytes; slab_lbo: stride of its 8-column chunks
    int off_cp, cp_bytes, cp_lbo, tc_nbuf;  // copy ring: cp_bytes in all, chunk stride cp_lbo
    int cp_group;  // bytes per group slot of the ring
    int off_ebuf, tmem_cols;
    int off_refit;  // FP32 block planes of the refit, |s| <= 2 (25 floats per block)
    // the A and B' regions of a full tile as two tensor-map boxes (a_pitch x ah
    // and b_pitch x BR floats, each dimension at most 256): 1 when they fit
    int tma_ok, box_ah, box_br;
};

struct PassArgs {
    int W, H, fmt;
    long long pitch;       // bytes between image rows
    PtrRef img_a, img_b;
    PtrRef afl;            // frame A as float (image grown by def_margin, interior written)
    PtrRef bdef;           // warped frame B' (float, image grown by def_margin)
    PtrRef adef;           // warped frame A' for the central warp (base null: use afl)
    long long def_pitch;   // floats between rows of afl / bdef / adef (a multiple of 32)
    int def_margin;        // a multiple of 4, at least R + 1
    int *err;              // nullable: bit 0 set if a bounded wait gave up
    int spin;              // polls of a bounded wait (0: the default limit)
    int dbg_stall;         // test hook: 1 a tile's region wait, 2 its first MMA wait (tensor-core
                           // tiles) waits on a phase nothing completes, once nothing is in flight
    int w, s, R, nx, ny;
    int deform;            // 0: frame B only, 1: central
    int prec;
    PtrRef pred_u, pred_v; // predictor on this grid (base null: zero predictor)
    PtrRef out_u, out_v;   // raw field
    PtrRef out_info;       // int32: bit0 valid, bits 8..15 ky, 16..23 kx
    PassPlan plan;
    PassPlan strip;        // strip alternative to the tile plan (strip_rows 0: none); the
                           // launch takes it when the batch gives it enough CTAs
    // set at launch (attach_region_maps): 3-D tensor maps (column, row, pair)
    // of the A and B' float frames whose boxes are the plan's regions; tma = 0:
    // the regions are loaded row by row
    int tma;
    CUtensorMap tm_a, tm_b;
};
// Encodes the region tensor maps into a for a launch of n_pairs (frames at a
// uniform pair stride); leaves a.tma = 0 where the plan's boxes, the frames or
// the encoder do not allow them.
void attach_region_maps(PassArgs &a, int n_pairs);

struct DeformArgs {
    PtrRef img;
    int fmt;
    long long pitch;       // bytes between image rows
    int W, H;
    PtrRef pred_u, pred_v; // predictor grid (base null: zero displacement)
    int w, s, nx, ny;
    float scale;           // 1 (frame B), 0.5 / -0.5 (central warp of B / A)
    int M;                 // margin of the output around the image
    PtrRef out;            // float, (W + 2M) x (H + 2M), out_pitch floats per row
    long long out_pitch;
};
cudaError_t launch_deform(const DeformArgs &a, int n_pairs, cudaStream_t st);
bool deform_nodes_fit(int w, int s, int nx, int ny);

// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount,
// read once per device); launch shapes that fill the device scale with it.
int device_sm_count();

// Opts every pass-kernel instantiation in to the full shared-memory carve-out
// on the current device (once per device; never inside a stream capture).
void prepare_pass_kernels();

// Message returned by rpiv_last_error() on the calling thread.
void set_last_error(const char *msg);

// Float frames the correlation pass reads (frame A, the warped B' and A'):
// the image sits at (M, M) of a buffer whose rows are `pitch` floats apart.
// M is a multiple of 4 and at least R + 1, so a shifted window never leaves
// the frame, and the pitch is a multiple of 32 floats with at least 4 floats
// past the right margin, so that every tile row starts 16-byte aligned (for
// a window step that is a multiple of 4) and may be copied rounded up to 16
// bytes.
inline int frame_margin(int max_radius) { return (max_radius + 1 + 3) / 4 * 4; }
inline long long frame_pitch(int W, int M) { return ((long long)W + 2 * M + 4 + 31) / 32 * 32; }
inline size_t frame_bytes(int W, int H, int M)
{
    return ((size_t)frame_pitch(W, M) * (size_t)(H + 2 * M) * 4 + 255) / 256 * 256;
}

// One full-resolution correlation pass on caller scratch of at least
// single_pass_scratch_bytes(W, H, R) bytes: checks its arguments (returns a
// public rpiv_status value, with the message set), then ingests frame A (or
// warps A' for the central mode), warps B' and runs the pass on `st`.
size_t single_pass_scratch_bytes(int W, int H, int R);
int single_pass(const void *img_a, const void *img_b, size_t pitch_bytes, int fmt, int W, int H, int w, int s, int R,
                int precision, int deform_mode, const float *pred_u, const float *pred_v, float *u, float *v,
                int32_t *info, void *scratch, cudaStream_t st);

// Returns false if (w, s, R, prec) is not supported by a compiled kernel.
// Tile plan of a correlation pass; strip (nullable) receives the strip
// alternative, strip_rows 0 when the shape has none.
bool pass_plan(int w, int s, int R, int nx, int ny, int prec, PassPlan *plan, PassPlan *strip = nullptr);
cudaError_t launch_pass(const PassArgs &args, int n_pairs, cudaStream_t st);
bool pass_supported(int R, int prec);

// ------------------------------------------------------------ grid kernels --

struct UodArgs {
    PtrRef u, v, info;         // info may have null base (all valid)
    int nx, ny;
    float thr, eps;
    int replace;
    PtrRef u_out, v_out, mask; // mask may have null base per pair
};
cudaError_t launch_uod(const UodArgs &a, int n_pairs, cudaStream_t st);

struct InterpArgs {
    PtrRef su, sv;
    int snx, sny, sw, ss;
    PtrRef du, dv;
    int dnx, dny, dw, ds, levels_up;
    int zero_if_null;  // a pair whose source is null: write zeros (1) or leave the destination (0)
};
cudaError_t launch_interp(const InterpArgs &a, int n_pairs, cudaStream_t st);

struct VortArgs {
    PtrRef u, v, out;
    int nx, ny, s;
};
cudaError_t launch_vort(const VortArgs &a, int n_pairs, cudaStream_t st);

// High-pass and CLAHE pre-processing of one u8/u16 image into float.
struct PreArgs {
    const void *img;
    int fmt;              // PIX_U8 or PIX_U16
    long long pitch;      // bytes
    int W, H, vmax;
    int hp, n;            // box radius and its pixel count (hp = 0: n = 1)
    int tx, ty, clip_pct; // tiles; clip_pct <= 0: no equalisation
    float *out;
    long long out_pitch;  // floats
};
size_t preprocess_scratch_bytes(int W, int H, int tx, int ty);
cudaError_t launch_preprocess(const PreArgs &a, void *scratch, cudaStream_t st);

// state = init ? x : alpha x + (1 - alpha) state, elementwise over n floats.
cudaError_t launch_ema(const float *x, float *state, size_t n, float alpha, int init, cudaStream_t st);

struct DownArgs {
    PtrRef src;
    int fmt;
    long long pitch;     // bytes
    int W, H;            // source size
    PtrRef dst;          // float, floor(W/2) x floor(H/2) at (margin, margin) of rows dst_pitch floats apart
    long long dst_pitch; // floats
    int dst_margin;
};
cudaError_t launch_down(const DownArgs &a, int n_pairs, cudaStream_t st);

// Frame as float into the margin layout (interior only): the correlation
// pass reads frame A from it.
struct IngestArgs {
    PtrRef src;
    int fmt;
    long long pitch;     // bytes
    int W, H;
    PtrRef dst;
    long long dst_pitch; // floats
    int dst_margin;
};
cudaError_t launch_ingest(const IngestArgs &a, int n_pairs, cudaStream_t st);

// Upload of the caller's host frames (page-locked, device-accessible) into the
// workspace: per pair, frames A and B of H rows of row_bytes, source rows pitch
// bytes apart, destination rows dst_pitch bytes apart (a multiple of 16).
struct UploadArgs {
    PtrRef src_a, src_b;   // pointer table entries of the frames
    long long pitch;       // bytes between source rows
    PtrRef dst_a, dst_b;   // workspace frames
    long long dst_pitch;   // bytes between destination rows
    int row_bytes, H;
};
cudaError_t launch_upload(const UploadArgs &a, int n_pairs, cudaStream_t st);


// ---------------------------------------------------------------- adjoint --

struct AdjArgs {
    int W, H, fmt;
    long long pitch;
    PtrRef img_a, img_b;
    int w, s, nx, ny;
    const float *u, *v;    // field on the grid
    void *ws;              // workspace of adjoint_workspace_bytes, 256-byte aligned
    float grad_scale;
    float *grad_u, *grad_v, *score_out;
};
size_t adjoint_workspace_bytes(int W, int H, int w, int s, int nx, int ny);
cudaError_t launch_adjoint(const AdjArgs &a, cudaStream_t st);
// Refinement step helpers: cu = u + eta gu (and v), and max(|a|, |b|) into *out.
cudaError_t launch_refine_axpy(const float *u, const float *v, const float *gu, const float *gv, float eta, float *cu,
                               float *cv, int n, cudaStream_t st);
cudaError_t launch_refine_absmax(const float *a, const float *b, int n, float *out, cudaStream_t st);

}  // namespace rpiv
