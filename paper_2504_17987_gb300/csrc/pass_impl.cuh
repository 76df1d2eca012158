// Fused correlation pass over a tile of TX x TY interrogation windows per
// CTA (paper Sec. 2: correlation coefficients of the warped pair around the
// peak, three-point Gaussian sub-pixel interpolation).  The warped frame B'
// is produced beforehand by the deformation kernel (k_deform.cu).
//
// Work of one CTA, staged in shared memory:
//   A region   raw A over the union of the tile's windows (aw x ah)
//   B' region  raw B' over the A region grown by R+1 on each side
//   C, V       sliding box sums of B' and B'^2 (C: columns, V: rows), pairs
//              of floats; V[r][c] = (S1, 1 / sqrt(E_B)) of the w x w box with
//              top-left logical B' pixel (r, c): its sum of B' and its inverse
//              norm (0 when the box is degenerate), i.e. every window at every
//              shift in [-R-1, R+1]^2, by lookup
//   P          block planes: the A region is cut into G x G blocks
//              (G = gcd(w, s)); P_b(s) = sum_{x in b} A(x) B'(x + s).
//              A window's numerator is the sum of its (w/G)^2 block planes
//              minus mean(A) * S1(s); this regrouping is exact, and computes
//              each block once instead of once per overlapping window.
// The peak is searched on C(s) sqrt(E_A) = numerator(s) / sqrt(E_B(s)): a positive
// per-window scale leaves the argmax unchanged; the five stencil values are
// scaled back by 1 / sqrt(E_A) before the fit.
// The planes are formed with FP32 FMAs on the CUDA cores, or with BF16/FP16
// tensor-core MMAs (mma.sync, FP32 accumulate) that multiply the Toeplitz
// matrix of a B' row (rows: sx) by the A rows that meet it (columns: sy), so
// that the accumulators hold P_b(sy, sx).  The 5-point stencil of the
// Gaussian fit is evaluated in FP32 (from the FP32 planes, or by direct sums
// on the tensor-core path and for shifts R+1).
// Strips (strip_kernel): for 50 % overlap with 16 or 32 px blocks a CTA walks
// the window rows of a one-row tile and keeps the block row two window rows
// share, so each block row's planes are computed once per strip segment.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "rpiv_internal.h"

namespace rpiv {

constexpr int PASS_THREADS = 256;
constexpr float TAU_PER_PIXEL = 1e-6f;  // degenerate-window energy per pixel

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Row-major walk over a width-W region with a fixed stride and no division
// per step: start at element `start`, advance by `stride` elements.
struct Walk2D {
    int x, y, sx, sy, W;
    __device__ __forceinline__ Walk2D(int start, int stride, int W_) : W(W_)
    {
        y = start / W_;
        x = start - y * W_;
        sy = stride / W_;
        sx = stride - sy * W_;
    }
    __device__ __forceinline__ void next()
    {
        x += sx;
        y += sy;
        if (x >= W) {
            x -= W;
            ++y;
        }
    }
};

template <typename T>
__device__ __forceinline__ float ld_px(const unsigned char *img, long long pitch, int x, int y)
{
    return (float)__ldg(reinterpret_cast<const T *>(img + (long long)y * pitch) + x);
}

template <int PREC>
__device__ __forceinline__ uint16_t to_h16(float x)
{
    if (PREC == PREC_BF16) return __bfloat16_as_ushort(__float2bfloat16_rn(x));
    return __half_as_ushort(__float2half_rn(x));
}

struct TileGeom {
    int R, ND, NP;
    int w, s, G, kb;  // window, step, block size, blocks per window side (compile-time when specialised)
    int wx0, wy0, nwx, nwy, nwin;
    int aw, ah, ax0, ay0;
    int BC, BR, OFFB;
    int hw, vh;
    int nbx, nby, nb;
};

// ------------------------------------------------------- region loads --

constexpr int MBAR_SPIN_LIMIT = 1 << 22;  // bounded wait for the bulk copies

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// one contiguous global -> shared copy (16-byte aligned, multiple of 16 bytes)
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// one bounded poll: the thread may sleep up to MBAR_SUSPEND_NS until the phase
// completes, so the wait costs few issue slots
constexpr uint32_t MBAR_SUSPEND_NS = 256;

// One box of a 3-D tensor map (column, row, pair) into shared memory,
// completing on the barrier; x is a multiple of 4 floats (16 bytes), y and z
// are in range, and the box's parts past the frame read as zeros.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// The regions as two tensor-map boxes (one instruction each) when the launch
// attached the maps and both destinations sit on 128-byte boundaries.
__device__ __forceinline__ bool regions_by_tma(const PassArgs &a, const float *As, const float *Bs)
{
    return a.tma && ((smem_addr(As) | smem_addr(Bs)) & 127u) == 0;
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(MBAR_SUSPEND_NS)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ int up4(int x) { return (x + 3) & ~3; }

// A region (raw frame A, or the central-warped A') and B' region, raw values,
// from the float frames in the workspace (margin layout).  With a step that is
// a multiple of 4 every row is one 16-byte-aligned bulk copy completing on an
// mbarrier (bounded wait: on timeout the error word is set and false returned);
// otherwise plain loads.  step: the CTA's k-th load (strips load once per
// window row): the barrier is initialised at k = 0 and phase k completes it.
static __device__ __forceinline__ bool load_regions(const PassArgs &a, const TileGeom &g, int pair, float *As, float *Bs,
                                    uint64_t *bar, int step = 0)
{
    const PassPlan &P = a.plan;
    const int tid = threadIdx.x, lane = tid & 31;
    const float *asrc = (const float *)resolve(a.adef.base ? a.adef : a.afl, pair);
    const float *bsrc = (const float *)resolve(a.bdef, pair);
    const long long dp = a.def_pitch;
    const int M = a.def_margin;
    const float *a0 = asrc + (long long)(g.ay0 + M) * dp + (g.ax0 + M);
    if (g.s % 4 == 0) {
        // B' rows start at smem column 0, i.e. global column ax0 + M - padl
        const float *b0 = bsrc + (long long)(g.ay0 - (g.R + 1) + M) * dp + (g.ax0 + M - P.padl);
        const int acols = up4(g.aw), bcols = up4(g.OFFB + g.BC);
        const bool tma = regions_by_tma(a, As, Bs);
        const uint32_t bytes = tma ? (uint32_t)(P.box_ah * P.a_pitch + P.box_br * P.b_pitch) * 4u
                                   : (uint32_t)(g.ah * acols + g.BR * bcols) * 4u;
        // warp 0 alone issues the copies and polls the barrier; the other
        // warps wait at the caller's CTA barrier, which also makes the staged
        // rows visible to them, and leave the issue slots to co-resident CTAs
        if (tid >= 32) return true;
        // the async copies follow the previous step's ordinary reads of the
        // same rows (ordered by the caller's CTA barrier)
        if (lane == 0) {
            if (step == 0) mbar_init(bar, 1);
            fence_proxy_async();
        }
        __syncwarp();
        if (lane == 0) mbar_expect_tx(bar, bytes);
        __syncwarp();
        if (tma) {
            if (lane == 0) {
                tma_load_3d(As, &a.tm_a, g.ax0 + M, g.ay0 + M, pair, bar);
                tma_load_3d(Bs, &a.tm_b, g.ax0 + M - P.padl, g.ay0 - (g.R + 1) + M, pair, bar);
            }
        } else {
            for (int r = lane; r < g.ah; r += 32) bulk_copy(As + r * P.a_pitch, a0 + (long long)r * dp, acols * 4, bar);
            for (int r = lane; r < g.BR; r += 32) bulk_copy(Bs + r * P.b_pitch, b0 + (long long)r * dp, bcols * 4, bar);
        }
        uint32_t parity = (uint32_t)step & 1u;
        const int lim = a.spin > 0 ? a.spin : MBAR_SPIN_LIMIT;
        bool landed = false;
        for (int it = 0; it < lim && !landed; ++it) landed = mbar_try_wait(bar, parity);
        if (landed && a.dbg_stall == 1) {
            // test hook: every copy has landed; the next phase expects bytes
            // that nothing sends, so the wait below runs out with nothing in flight
            __syncwarp();
            if (lane == 0) mbar_expect_tx(bar, 16);
            __syncwarp();
            parity ^= 1u;
            landed = false;
            for (int it = 0; it < lim && !landed; ++it) landed = mbar_try_wait(bar, parity);
            if (!landed && lane == 0 && a.err) atomicOr(a.err, 1);
            return false;
        }
        if (landed) return true;
        if (lane == 0 && a.err) atomicOr(a.err, 1);
        // give copies still in flight a bounded chance to land before the CTA exits
        for (int it = 0; it < lim; ++it)
            if (mbar_try_wait(bar, parity)) break;
        return false;
    }
    for (Walk2D it(tid, blockDim.x, g.aw); it.y < g.ah; it.next())
        As[it.y * P.a_pitch + it.x] = a0[(long long)it.y * dp + it.x];
    const float *b1 = bsrc + (long long)(g.ay0 - (g.R + 1) + M) * dp + (g.ax0 - (g.R + 1) + M);
    for (Walk2D it(tid, blockDim.x, g.BC); it.y < g.BR; it.next())
        Bs[it.y * P.b_pitch + g.OFFB + it.x] = b1[(long long)it.y * dp + it.x];
    return true;
}

template <int PREC>
__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    if (PREC == PREC_BF16) {
        const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<const uint32_t *>(&v);
    }
    const __half2 v = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// Rows of the A slab layout of the tensor-core path: slab j (block row
// j / RG, row group j % RG) holds A rows j rows .. j rows + rows - 1 from TA
// row tc_slab_row(j); the 2R rows before each slab and after the last are
// zero, so that an MMA fragment of a used shift that reaches past its group
// reads zeros; tc_front() leading rows keep the fragments of unused shifts
// inside the array.
__device__ __forceinline__ int tc_front(int R) { return max(0, 8 * ((2 * R + 8) / 8) - 1 - 2 * R); }
__device__ __forceinline__ int tc_slab_row(int R, int rows, int j) { return tc_front(R) + 2 * R + j * (rows + 2 * R); }

// Strip loads on the bulk path (steps that are multiples of 4): one warp issues
// the copies of a step's regions without waiting, so that they overlap the end
// of the previous step; step k completes phase k of the barrier.
static __device__ __forceinline__ void issue_regions(const PassArgs &a, const TileGeom &g, int pair, float *As, float *Bs,
                                     uint64_t *bar, int step)
{
    const PassPlan &P = a.plan;
    const int lane = threadIdx.x & 31;
    const float *asrc = (const float *)resolve(a.adef.base ? a.adef : a.afl, pair);
    const float *bsrc = (const float *)resolve(a.bdef, pair);
    const long long dp = a.def_pitch;
    const int M = a.def_margin;
    const float *a0 = asrc + (long long)(g.ay0 + M) * dp + (g.ax0 + M);
    const float *b0 = bsrc + (long long)(g.ay0 - (g.R + 1) + M) * dp + (g.ax0 + M - P.padl);
    const int acols = up4(g.aw), bcols = up4(g.OFFB + g.BC);
    const bool tma = regions_by_tma(a, As, Bs);
    const uint32_t bytes = tma ? (uint32_t)(P.box_ah * P.a_pitch + P.box_br * P.b_pitch) * 4u
                               : (uint32_t)(g.ah * acols + g.BR * bcols) * 4u;
    if (lane == 0) {
        if (step == 0) mbar_init(bar, 1);
        fence_proxy_async();
    }
    __syncwarp();
    if (lane == 0) mbar_expect_tx(bar, bytes);
    __syncwarp();
    if (tma) {
        if (lane == 0) {
            tma_load_3d(As, &a.tm_a, g.ax0 + M, g.ay0 + M, pair, bar);
            tma_load_3d(Bs, &a.tm_b, g.ax0 + M - P.padl, g.ay0 - (g.R + 1) + M, pair, bar);
        }
        return;
    }
    for (int r = lane; r < g.ah; r += 32) bulk_copy(As + r * P.a_pitch, a0 + (long long)r * dp, acols * 4, bar);
    for (int r = lane; r < g.BR; r += 32) bulk_copy(Bs + r * P.b_pitch, b0 + (long long)r * dp, bcols * 4, bar);
}

// Bounded wait for step k's copies (warp 0); false after the limit, with the
// error word set once the copies in flight had their chance to land.
static __device__ __forceinline__ bool wait_regions(const PassArgs &a, uint64_t *bar, int step)
{
    const uint32_t parity = (uint32_t)step & 1u;
    const int lim = a.spin > 0 ? a.spin : MBAR_SPIN_LIMIT;
    for (int it = 0; it < lim; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    if ((threadIdx.x & 31) == 0 && a.err) atomicOr(a.err, 1);
    for (int it = 0; it < lim; ++it)
        if (mbar_try_wait(bar, parity)) break;
    return false;
}

// 16-bit copies for the tensor-core path, two columns per conversion: A in
// the slab layout, and B' twice, the second shifted one column left (TB1[x] =
// B'[x + 1]) so that every column pair of a fragment starts 4-byte aligned,
// with zeros wherever fragments reach outside the staged region.  A thread
// keeps one column pair and walks rows.  Both frames are rounded with the
// tile offset m subtracted (restored in FP32 by plane_and_peak), which keeps
// the rounded values small.
template <int PREC>
__device__ __forceinline__ void tc_copies(const PassArgs &a, const TileGeom &g, const float *As, const float *Bs, uint16_t *TA,
                          uint16_t *TB, float m)
{
    const PassPlan &P = a.plan;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int R = g.R, RG = P.RGx, rows = g.G / RG, stride = rows + 2 * R;
    const int front = tc_front(R), nslab = g.nby * RG;
    const int ta_rows = front + 2 * R + nslab * stride;
    const int apairs = g.aw >> 1;  // aw is even (G even)
    const int hpa = P.tca_pitch >> 1, lead = front + 2 * R;
    for (int c0 = 0; c0 < apairs; c0 += nt) {
        const int cols = min(apairs - c0, nt), step = nt / cols;
        const int x2 = c0 + tid % cols, ph = tid / cols;
        if (ph >= step) continue;
        uint32_t *dst = reinterpret_cast<uint32_t *>(TA) + x2;
        const float *src = As + 2 * x2;
        for (int row = ph; row < lead; row += step) dst[row * hpa] = 0u;
        // slab rows: u = j stride + r, walked with (j, r) counters
        int j = ph / stride, r = ph - (ph / stride) * stride;
        for (int u = ph; u < ta_rows - lead; u += step) {
            uint32_t v = 0u;
            if (r < rows) {
                const float2 f = *reinterpret_cast<const float2 *>(src + (j * rows + r) * P.a_pitch);
                v = pack2<PREC>(f.x - m, f.y - m);
            }
            dst[(lead + u) * hpa] = v;
            r += step;
            while (r >= stride) {
                r -= stride;
                ++j;
            }
        }
    }
    uint32_t *TB1 = reinterpret_cast<uint32_t *>(TB + P.tb_rows * P.tcb_pitch);
    uint32_t *TB0 = reinterpret_cast<uint32_t *>(TB);
    const int lo = g.OFFB, hi = g.OFFB + g.BC;  // staged columns
    const int bpairs = P.tb_cols >> 1;           // fragments of unused shifts reach past the region: zeros
    for (int c0 = 0; c0 < bpairs; c0 += nt) {
        const int cols = min(bpairs - c0, nt), step = nt / cols;
        const int x2 = c0 + tid % cols, ph = tid / cols;
        if (ph >= step) continue;
        const int x = 2 * x2;
        const bool k0 = x >= lo && x < hi, k1 = x + 1 >= lo && x + 1 < hi, k2 = x + 2 >= lo && x + 2 < hi;
        const int hpb = P.tcb_pitch >> 1;
        const float *br = Bs + ph * P.b_pitch + x;
        uint32_t *d0 = TB0 + ph * hpb + x2, *d1 = TB1 + ph * hpb + x2;
        for (int y = ph; y < g.BR; y += step) {
            const float v0 = k0 ? br[0] - m : 0.f, v1 = k1 ? br[1] - m : 0.f, v2 = k2 ? br[2] - m : 0.f;
            *d0 = pack2<PREC>(v0, v1);
            *d1 = pack2<PREC>(v1, v2);
            br += step * P.b_pitch;
            d0 += step * hpb;
            d1 += step * hpb;
        }
    }
}

// ------------------------------------------------------ box sums (C, V) --

// 1 / sqrt(E_B) of a box from its sum and sum of squares; 0 for a degenerate
// box.  E_B > tau > 0 is a normal float, so the hardware's approximate
// reciprocal square root needs no subnormal handling (flush-to-zero form).
__device__ __forceinline__ float inv_norm(float s1, float s2, float inv_n, float tau)
{
    const float EB = s2 - s1 * s1 * inv_n;
    float r = 0.f;
    if (EB > tau) asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(EB));
    return r;
}

// Packed pairs of FP32 values for the paired arithmetic (fma/add/sub.rn.f32x2:
// two IEEE operations in one instruction, each rounded as the scalar one).
__device__ __forceinline__ uint64_t pack_f2(float lo, float hi)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float lo_f2(uint64_t p) { return __uint_as_float((uint32_t)p); }
__device__ __forceinline__ float hi_f2(uint64_t p) { return __uint_as_float((uint32_t)(p >> 32)); }
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t fadd2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t fsub2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Window box sums of B' and B'^2 at every shift, in two sliding passes (box_cols, then
// box_rows once the column sums are visible to the CTA):
//   C[r][x] = sum_{y=r}^{r+w-1} (B'[y][x], B'[y][x]^2)   (threads along x: conflict free)
//   V[r][c] = sum_{x=c}^{c+w-1} C[r][x]                  (threads along r, odd pitch)
// so V[r][c] sums the w x w box whose top-left logical B' pixel is (r, c); its
// second member keeps 1 / sqrt(E_B) of the box instead of its sum of squares.
// C and V hold (S1, S2) and (S1, 1 / sqrt(E_B)) pairs: one 64-bit access per
// element, and the row pass adds both sums with one paired instruction.  Each
// thread keeps a running sum over box_lv (columns) or box_lh (rows) outputs;
// the plan sets them and the number of runs for a full tile, and an edge tile,
// never larger, skips the runs that start past its end.
// split_cols (strips, whose column runs are short: 2R + 3 outputs): one run
// per column instead, its first w-term sum split between the two half-warps
// (rows [0, w/2) and [w/2, w)); the lower half-warp then slides down the run.
// The upper half-warp starts four rows into its range and wraps, so that the
// two halves' loads fall in different banks (the B' pitch is 4 x odd floats:
// any two rows w/2 + 4 or 4 apart are 16 banks apart for w/2 a multiple of 8).
static __device__ __forceinline__ void box_cols(const PassArgs &a, const TileGeom &g, const float *Bs, float *Cs,
                                                bool split_cols)
{
    const PassPlan &P = a.plan;
    const int w = g.w, tid = threadIdx.x;
    const int cp = P.h_pitch;  // pitch of C in pairs (odd)
    float2 *C = reinterpret_cast<float2 *>(Cs);
    if (split_cols) {
        const int lane = tid & 31, hh = lane >> 4, li = lane & 15, half = w >> 1;
        for (int base = tid - lane; base < 16 * ((g.BC + 15) >> 4) * 2; base += blockDim.x) {
            const int x0 = (base >> 1) + li, x = min(x0, g.BC - 1);
            const float *col = Bs + g.OFFB + x;
            float s1 = 0.f, s2 = 0.f;
            for (int t = 0; t < half; ++t) {
                int y = t;
                if (hh) {
                    y = t + 4;
                    if (y >= half) y -= half;
                    y += half;
                }
                const float b = col[y * P.b_pitch];
                s1 += b;
                s2 = fmaf(b, b, s2);
            }
            s1 += __shfl_xor_sync(0xffffffffu, s1, 16);
            s2 += __shfl_xor_sync(0xffffffffu, s2, 16);
            if (hh == 0 && x0 < g.BC) {
                C[x] = make_float2(s1, s2);
                for (int r = 1; r < g.vh; ++r) {
                    const float bo = col[(r - 1) * P.b_pitch], bi = col[(r + w - 1) * P.b_pitch];
                    s1 += bi - bo;
                    s2 += bi * bi - bo * bo;
                    C[r * cp + x] = make_float2(s1, s2);
                }
            }
        }
    } else {
        const int Lv = P.box_lv;
        for (int it = tid; it < g.BC * P.box_nv; it += blockDim.x) {
            const int seg = it / g.BC, x = it - seg * g.BC;
            const int r_lo = seg * Lv, r_hi = min(g.vh, r_lo + Lv);
            if (r_lo >= g.vh) continue;
            const float *col = Bs + g.OFFB + x;
            float s1 = 0.f, s2 = 0.f;
            for (int y = r_lo; y < r_lo + w; ++y) {
                const float b = col[y * P.b_pitch];
                s1 += b;
                s2 = fmaf(b, b, s2);
            }
            C[r_lo * cp + x] = make_float2(s1, s2);
            for (int r = r_lo + 1; r < r_hi; ++r) {
                const float bo = col[(r - 1) * P.b_pitch], bi = col[(r + w - 1) * P.b_pitch];
                s1 += bi - bo;
                s2 += bi * bi - bo * bo;
                C[r * cp + x] = make_float2(s1, s2);
            }
        }
    }
}

// The row pass of the window box sums, from the column sums C (complete and
// visible to the CTA).
static __device__ __forceinline__ void box_rows(const PassArgs &a, const TileGeom &g, const float *Cs, float *Vs)
{
    const PassPlan &P = a.plan;
    const int w = g.w, tid = threadIdx.x;
    const int cp = P.h_pitch;  // pitch of C in pairs (odd)
    const int vp = P.v_pitch;  // pitch of V in pairs (odd, >= hw)
    const float inv_n = 1.f / (float)(w * w), tau = TAU_PER_PIXEL * (float)(w * w);
    float2 *V = reinterpret_cast<float2 *>(Vs);
    const uint64_t *Cp = reinterpret_cast<const uint64_t *>(Cs);
    const int Lh = P.box_lh;
    for (int it = tid; it < g.vh * P.box_nh; it += blockDim.x) {
        const int seg = it / g.vh, r = it - seg * g.vh;
        const int c_lo = seg * Lh, c_hi = min(g.hw, c_lo + Lh);
        if (c_lo >= g.hw) continue;
        const uint64_t *cr = Cp + r * cp;
        float2 *vr = V + r * vp;
        uint64_t s = 0ull;  // (S1, S2), +0
        for (int x = c_lo; x < c_lo + w; ++x) s = fadd2(s, cr[x]);
        vr[c_lo] = make_float2(lo_f2(s), inv_norm(lo_f2(s), hi_f2(s), inv_n, tau));
        for (int c = c_lo + 1; c < c_hi; ++c) {
            s = fadd2(s, fsub2(cr[c + w - 1], cr[c - 1]));
            vr[c] = make_float2(lo_f2(s), inv_norm(lo_f2(s), hi_f2(s), inv_n, tau));
        }
    }
}

// Both passes, with the CTA barrier between them.
static __device__ __forceinline__ void box_sums(const PassArgs &a, const TileGeom &g, const float *Bs, float *Cs, float *Vs)
{
    box_cols(a, g, Bs, Cs, false);
    __syncthreads();
    box_rows(a, g, Cs, Vs);
}

// Sum and centred sum of squares of every G x G block of A (two passes):
// bst[b] = (sum, M2).  For G a power of two from 4 to 32 one thread takes a
// block row (128-bit loads) and the G rows of a block, in aligned lanes of one
// warp, are summed by shuffles; the mean is exact scaling by 1 / G^2.
// b0: first block (a strip step after its first computes only the block row
// it adds); ring_wy >= 0: strip mode, block row by of window row ring_wy is
// kept in ring row (ring_wy + by) & 1, as the planes are.
__device__ __forceinline__ int block_slot(const TileGeom &g, int byi, int bxi, int ring_wy)
{
    return ring_wy < 0 ? byi * g.nbx + bxi : ((ring_wy + byi) & 1) * g.nbx + bxi;
}

static __device__ __forceinline__ void block_stats_rows(const PassArgs &a, const TileGeom &g, const float *As, float2 *bst,
                                                        int b0, int ring_wy)
{
    const PassPlan &P = a.plan;
    const int lane = threadIdx.x & 31;
    const int G = g.G, lg = __ffs(G) - 1;
    const float inv_n = 1.f / (float)(G * G);
    const int items = (g.nb - b0) * G;
    // warp-uniform trip count: every lane takes part in the shuffles; lanes
    // past the end repeat the last row and store nothing
    for (int base = threadIdx.x - lane; base < items; base += blockDim.x) {
        const int it = min(base + lane, items - 1);
        const int b = b0 + (it >> lg), row = it & (G - 1);
        const int byi = b / g.nbx, bxi = b - byi * g.nbx;
        const float *p = As + (byi * G + row) * P.a_pitch + bxi * G;
        float s = 0.f;
        for (int c = 0; c < G; c += 4) {
            const float4 v = *reinterpret_cast<const float4 *>(p + c);
            s += v.x;
            s += v.y;
            s += v.z;
            s += v.w;
        }
        for (int o = 1; o < G; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const float m = s * inv_n;
        float q = 0.f;
        for (int c = 0; c < G; c += 4) {
            const float4 v = *reinterpret_cast<const float4 *>(p + c);
            q = fmaf(v.x - m, v.x - m, q);
            q = fmaf(v.y - m, v.y - m, q);
            q = fmaf(v.z - m, v.z - m, q);
            q = fmaf(v.w - m, v.w - m, q);
        }
        for (int o = 1; o < G; o <<= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
        if (base + lane < items && row == 0) bst[block_slot(g, byi, bxi, ring_wy)] = make_float2(s, q);
    }
}

// Any G: one warp per block, lanes along the rows.
static __device__ __forceinline__ void block_stats(const PassArgs &a, const TileGeom &g, const float *As, float2 *bst,
                                                   int b0 = 0, int ring_wy = -1)
{
    if (g.G >= 4 && g.G <= 32 && (g.G & (g.G - 1)) == 0) {
        block_stats_rows(a, g, As, bst, b0, ring_wy);
        return;
    }
    const PassPlan &P = a.plan;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int G = g.G;
    const float n = (float)(G * G);
    for (int b = b0 + warp; b < g.nb; b += nwarps) {
        const int bxi = b % g.nbx, byi = b / g.nbx;
        const float *base = As + (byi * G) * P.a_pitch + bxi * G;
        float s = 0.f;
        for (Walk2D e(lane, 32, G); e.y < G; e.next()) s += base[e.y * P.a_pitch + e.x];
        s = warp_sum(s);
        const float m = s / n;
        float q = 0.f;
        for (Walk2D e(lane, 32, G); e.y < G; e.next()) {
            const float d = base[e.y * P.a_pitch + e.x] - m;
            q = fmaf(d, d, q);
        }
        q = warp_sum(q);
        if (lane == 0) bst[block_slot(g, byi, bxi, ring_wy)] = make_float2(s, q);
    }
}

// Window mean and energy from its blocks (parallel-variance identity):
// E = sum M2_b + n_b sum (mean_b - mean)^2, in a fixed order.
static __device__ __forceinline__ void window_stats(const PassArgs &a, const TileGeom &g, const float2 *bst, float *stats,
                                                    int ring_wy = -1)
{
    (void)a;
    const int G = g.G, kb = g.w / G;
    const float nb = (float)(G * G), n = (float)(g.w * g.w);
    for (int wi = threadIdx.x; wi < g.nwin; wi += blockDim.x) {
        const int wxi = wi % g.nwx, wyi = wi / g.nwx;
        const int bx0 = (wxi * g.s) / G, by0 = (wyi * g.s) / G;
        float s = 0.f;
        for (int yy = 0; yy < kb; ++yy)
            for (int xx = 0; xx < kb; ++xx) s += bst[block_slot(g, by0 + yy, bx0 + xx, ring_wy)].x;
        const float mean = s / n;
        float e = 0.f;
        for (int yy = 0; yy < kb; ++yy)
            for (int xx = 0; xx < kb; ++xx) {
                const float2 p = bst[block_slot(g, by0 + yy, bx0 + xx, ring_wy)];
                const float d = p.x / nb - mean;
                e += p.y + nb * d * d;
            }
        stats[2 * wi] = mean;
        stats[2 * wi + 1] = e;
    }
}

// --------------------------------------------- FP32 block planes (CUDA cores) --

// Plane items are (unit, row group) with RG a power of two: a warp takes
// 32 / RG consecutive units, the row group in the high lane bits, so that a
// quarter-warp reads consecutive shifts (bank-conflict free) and a butterfly of
// shuffles over lane distances 32 / RG, ... , 16 sums a unit's partials; row
// group 0 stores the sum.
template <int ND>
__device__ __forceinline__ void sum_row_groups(float (&acc)[ND], int lrg)
{
    for (int o = 32 >> lrg; o < 32; o <<= 1) {
#pragma unroll
        for (int d = 0; d < ND; ++d) acc[d] += __shfl_xor_sync(0xffffffffu, acc[d], o);
    }
}

// Compile-time radius: each thread owns one (block, sy, row group) and keeps
// the 2R+1 accumulators of its sx row in registers; rows are streamed from
// shared memory four columns at a time with aligned 128-bit loads.
// b0: first block (strips compute only the new block row after their first
// step); ring_wy >= 0: strip mode, block row by of window row ring_wy goes to
// ring row (ring_wy + by) & 1.
template <int R>
__device__ __forceinline__ void block_planes_fp32(const PassArgs &a, const TileGeom &g, const float *As, const float *Bs, float *Ps,
                                  int b0 = 0, int ring_wy = -1)
{
    constexpr int ND = 2 * R + 1;
    constexpr int MIS = ((-R) % 4 + 4) % 4;
    constexpr int NQ = (4 + 2 * R + MIS + 3) / 4;
    const PassPlan &P = a.plan;
    const int G = g.G, RG = P.RGx, rows = G / RG, lrg = __ffs(RG) - 1;
    const int units = (g.nb - b0) * ND;  // (block, sy)
    const int lane = threadIdx.x & 31, gi = lane >> (5 - lrg), ul = lane & ((32 >> lrg) - 1);
    // warp-uniform trip count for the shuffles; lanes past the last unit
    // repeat it and store nothing
    for (int base = (threadIdx.x - lane) >> lrg; base < units; base += blockDim.x >> lrg) {
        const int u = min(base + ul, units - 1);
        const int b = b0 + u / ND;
        const int syi = u - (b - b0) * ND;
        const int byi = b / g.nbx, bxi = b - byi * g.nbx;
        const int c0 = bxi * G, r0 = byi * G + gi * rows;
        // Two accumulator sets of packed pairs, so that every pair of B' values
        // an FMA pair reads is an aligned register pair of a 128-bit load: for
        // the columns j with MIS + j even, set E holds (d, d + 1) for even d
        // and a single d = ND - 1; otherwise set O holds a single d = 0 and the
        // pairs (d, d + 1) for odd d.  acc[d] = E[d] + O[d].
        constexpr int NPR = (ND - 1) / 2;
        uint64_t pe[NPR > 0 ? NPR : 1], po[NPR > 0 ? NPR : 1];
        float se = 0.f, so = 0.f;
#pragma unroll
        for (int q = 0; q < NPR; ++q) pe[q] = po[q] = 0ull;
        for (int y = r0; y < r0 + rows; ++y) {
            const float *arow = As + y * P.a_pitch;
            const float *brow = Bs + (y + syi + 1) * P.b_pitch + P.padl - R - MIS;
            for (int c = c0; c < c0 + G; c += 4) {
                const float4 a4 = *reinterpret_cast<const float4 *>(arow + c);
                uint64_t bp[NQ * 2];
                float bv[NQ * 4];
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const float4 t = *reinterpret_cast<const float4 *>(brow + c + 4 * q);
                    bv[4 * q] = t.x;
                    bv[4 * q + 1] = t.y;
                    bv[4 * q + 2] = t.z;
                    bv[4 * q + 3] = t.w;
                    bp[2 * q] = pack_f2(t.x, t.y);
                    bp[2 * q + 1] = pack_f2(t.z, t.w);
                }
                const float av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint64_t a2 = pack_f2(av[j], av[j]);
                    if (((MIS + j) & 1) == 0) {
#pragma unroll
                        for (int q = 0; q < NPR; ++q) pe[q] = ffma2(a2, bp[(MIS + j) / 2 + q], pe[q]);
                        se = fmaf(av[j], bv[MIS + j + ND - 1], se);
                    } else {
                        so = fmaf(av[j], bv[MIS + j], so);
#pragma unroll
                        for (int q = 0; q < NPR; ++q) po[q] = ffma2(a2, bp[(MIS + j + 1) / 2 + q], po[q]);
                    }
                }
            }
        }
        float acc[ND];
#pragma unroll
        for (int q = 0; q < NPR; ++q) {
            acc[2 * q] = lo_f2(pe[q]);
            acc[2 * q + 1] = hi_f2(pe[q]);
        }
        acc[ND - 1] = se;
        acc[0] += so;
#pragma unroll
        for (int q = 0; q < NPR; ++q) {
            acc[2 * q + 1] += lo_f2(po[q]);
            acc[2 * q + 2] += hi_f2(po[q]);
        }
        sum_row_groups<ND>(acc, lrg);
        if (base + ul < units && gi == 0) {
            const int pb = ring_wy < 0 ? b : ((ring_wy + byi) & 1) * g.nbx + bxi;
            float *out = Ps + pb * P.pstride + syi * ND;
#pragma unroll
            for (int d = 0; d < ND; ++d) out[d] = acc[d];
        }
    }
}

// Runtime radius (any R up to RPIV_MAX_RADIUS): scalar loads, sx in chunks of 8.
static __device__ __forceinline__ void block_planes_fp32_generic(const PassArgs &a, const TileGeom &g, const float *As, const float *Bs,
                                          float *Ps)
{
    const PassPlan &P = a.plan;
    const int R = g.R, ND = g.ND;
    const int G = g.G, RG = P.RGx, rows = G / RG, lrg = __ffs(RG) - 1;
    const int nch = (ND + 7) / 8;
    const int units = g.nb * ND * nch;  // (block, sy, sx chunk)
    const int lane = threadIdx.x & 31, gi = lane >> (5 - lrg), ul = lane & ((32 >> lrg) - 1);
    for (int base = (threadIdx.x - lane) >> lrg; base < units; base += blockDim.x >> lrg) {
        int rest = min(base + ul, units - 1);
        const int ch = rest % nch;
        rest /= nch;
        const int syi = rest % ND;
        const int b = rest / ND;
        const int bxi = b % g.nbx, byi = b / g.nbx;
        const int c0 = bxi * G, r0 = byi * G + gi * rows;
        const int d0 = ch * 8;
        float acc[8];
#pragma unroll
        for (int d = 0; d < 8; ++d) acc[d] = 0.f;
        for (int y = r0; y < r0 + rows; ++y) {
            const float *arow = As + y * P.a_pitch;
            const float *brow = Bs + (y + syi + 1) * P.b_pitch + P.padl - R + d0;
            for (int c = c0; c < c0 + G; ++c) {
                const float av = arow[c];
#pragma unroll
                for (int d = 0; d < 8; ++d)
                    if (d0 + d < ND) acc[d] = fmaf(av, brow[c + d], acc[d]);
            }
        }
        sum_row_groups<8>(acc, lrg);
        if (base + ul < units && gi == 0) {
            float *out = Ps + b * P.pstride + syi * ND + d0;
            for (int d = 0; d < 8 && d0 + d < ND; ++d) out[d] = acc[d];
        }
    }
}

// ------------------------------------------- tensor-core block planes --


template <int PREC>
__device__ __forceinline__ void mma_k8(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t b0)
{
    if (PREC == PREC_BF16) {
        asm volatile(
            "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a0), "r"(a1), "r"(b0));
    } else {
        asm volatile(
            "mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a0), "r"(a1), "r"(b0));
    }
}

template <int PREC>
__device__ __forceinline__ void mma_k16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                        uint32_t b0, uint32_t b1)
{
    if (PREC == PREC_BF16) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    } else {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
}

__device__ __forceinline__ uint32_t ld_pair(const uint16_t *p) { return *reinterpret_cast<const uint32_t *>(p); }

// Block planes on the tensor cores, one warp per (block, row group).  For
// every row r of B' the group meets, the MMA multiplies
//     X_r[sx][k] = B'[r][x0 + k + sx]        (a Toeplitz matrix of the row: M = sx)
// by  Y_r[k][sy] = A[r - sy][x0 + k]        (the A rows r - sy of the group: N = sy)
// over the block's columns k, so D[sx][sy] accumulates
//     sum_r sum_k A[r - sy][x0 + k] B'[r][x0 + k + sx] = P_b(sy, sx)
// directly, for every shift, across the rows.  A rows outside the group come
// from the zero bands of the slab layout, so every fragment is one load at an
// offset that only the row step changes.  16 x 8 tiles: MT tiles of sx, NT
// tiles of sy.
template <int R, int PREC>
__device__ __forceinline__ void block_planes_tc(const PassArgs &a, const TileGeom &g, const uint16_t *TA, const uint16_t *TB,
                                float *Ps)
{
    constexpr int ND = 2 * R + 1;
    constexpr int NP = ND * ND;
    constexpr int MT = (ND + 15) / 16;
    constexpr int NT = (ND + 7) / 8;
    const PassPlan &P = a.plan;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int gq = lane >> 2, tq = lane & 3;
    const int G = g.G, RG = P.RGx, rows = G / RG;
    const int ap = P.tca_pitch, bp = P.tcb_pitch;
    const uint16_t *TB1 = TB + P.tb_rows * bp;
    // smem column of Toeplitz element (m, k) of m-tile mt at block column X:
    //     padl - R + X + 16 mt + m + k;  X is even, so its parity is that of padl - R + m
    const int colbase = P.padl - R + gq + 2 * tq;
    // odd columns read the copy shifted by one (TB1[x] = B'[x + 1]) at x - 1
    const uint16_t *srcB = (colbase & 1) ? (TB1 - 1) : TB;
    const int trips = rows + 2 * R;  // B' rows a group meets
    const int items = g.nb * RG;
    for (int it = warp; it < items; it += nwarps) {
        const int b = it / RG, gi = it - b * RG;
        const int byi = b / g.nbx, bxi = b - byi * g.nbx;
        const int X0 = bxi * G;
        const int i_lo = byi * G + gi * rows;  // first A row of the group
        // step t: B' smem row i_lo + 1 + t; lane (n, gq) reads A row i_lo + t - 8 n - gq,
        // i.e. slab row t - 8 n - gq
        const uint16_t *pb = srcB + (i_lo + 1) * bp + colbase + X0;
        const uint16_t *pa[NT];
#pragma unroll
        for (int n = 0; n < NT; ++n) pa[n] = TA + (tc_slab_row(R, rows, byi * RG + gi) - 8 * n - gq) * ap + X0 + 2 * tq;
        // the row step advances every fragment pointer by one row
        float acc[MT][NT][4];
#pragma unroll
        for (int m = 0; m < MT; ++m)
#pragma unroll
            for (int n = 0; n < NT; ++n)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[m][n][e] = 0.f;
        if ((G % 16) == 0) {
#pragma unroll 2
            for (int t = 0; t < trips; ++t) {
#pragma unroll
                for (int X = 0; X < G; X += 16) {
                    uint32_t bf[NT][2];
#pragma unroll
                    for (int n = 0; n < NT; ++n) {
                        bf[n][0] = ld_pair(pa[n] + X);
                        bf[n][1] = ld_pair(pa[n] + X + 8);
                    }
#pragma unroll
                    for (int m = 0; m < MT; ++m) {
                        const uint16_t *c = pb + X + 16 * m;
                        const uint32_t a0 = ld_pair(c), a1 = ld_pair(c + 8), a3 = ld_pair(c + 16);
#pragma unroll
                        for (int n = 0; n < NT; ++n) mma_k16<PREC>(acc[m][n], a0, a1, a1, a3, bf[n][0], bf[n][1]);
                    }
                }
#pragma unroll
                for (int n = 0; n < NT; ++n) pa[n] += ap;
                pb += bp;
            }
        } else {
            // G = 8 (or another even size below 16): k8 steps; columns past
            // the block (uneven G) enter as zeros
#pragma unroll 4
            for (int t = 0; t < trips; ++t) {
#pragma unroll
                for (int X = 0; X < G; X += 8) {
                    const bool cok = (G % 8) == 0 || X + 2 * tq < G;
                    uint32_t bf[NT];
#pragma unroll
                    for (int n = 0; n < NT; ++n) bf[n] = cok ? ld_pair(pa[n] + X) : 0u;
#pragma unroll
                    for (int m = 0; m < MT; ++m) {
                        const uint16_t *c = pb + X + 16 * m;
                        const uint32_t a0 = ld_pair(c), a1 = ld_pair(c + 8);
#pragma unroll
                        for (int n = 0; n < NT; ++n) mma_k8<PREC>(acc[m][n], a0, a1, bf[n]);
                    }
                }
#pragma unroll
                for (int n = 0; n < NT; ++n) pa[n] += ap;
                pb += bp;
            }
        }
        // D[m][n] of tile (mt, nt) is P_b(sy = 8 nt + n - R, sx = 16 mt + m - R)
        float *out = Ps + b * P.pstride + gi * NP;
#pragma unroll
        for (int m = 0; m < MT; ++m)
#pragma unroll
            for (int n = 0; n < NT; ++n)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int sx = 16 * m + gq + (e >= 2 ? 8 : 0) - R;
                    const int sy = 8 * n + 2 * tq + (e & 1) - R;
                    if (sx <= R && sy <= R) out[(sy + R) * ND + (sx + R)] = acc[m][n][e];
                }
    }
}

// Tensor-core path with RG > 1: the row groups' partial planes of a block
// (consecutive, NP floats apart) are summed into the first, in a fixed order.
static __device__ __forceinline__ void reduce_row_groups(const PassArgs &a, const TileGeom &g, float *Ps)
{
    const int RG = a.plan.RGx, NP = g.NP, ps = a.plan.pstride;
    for (int e = threadIdx.x; e < g.nb * NP; e += blockDim.x) {
        const int b = e / NP, q = e - b * NP;
        float *p = Ps + b * ps + q;
        float v = p[0];
        for (int t = 1; t < RG; ++t) v += p[t * NP];
        p[0] = v;
    }
}

// ----------------------------------------------- assembly and sub-pixel --

// Three-point Gaussian fit on a log scale, with the parabola as a fallback;
// lm, l0, lp are the logs of the values that are positive (only used when
// all three are).  Both forms are unchanged when the three values share a
// positive factor.  The fit takes the hardware's approximate logarithm and
// divide (__logf: absolute error below 2^-21.4 on [0.5, 2], 3 ulp elsewhere;
// __fdividef: 2 ulp for the denominators here, |den| < 2^126): an error of
// about 1e-6 in the logs moves the offset by about 1e-6 / |den| px.
__device__ __forceinline__ float gauss3f(float cm, float c0, float cp, float lm, float l0, float lp)
{
    float d = 0.f;
    bool ok = false;
    if (cm > 0.f && c0 > 0.f && cp > 0.f) {
        const float den = 2.f * lm - 4.f * l0 + 2.f * lp;
        if (den < 0.f) {
            d = __fdividef(lm - lp, den);
            ok = true;
        }
    }
    if (!ok) {
        const float den = 2.f * cm - 4.f * c0 + 2.f * cp;
        if (den < 0.f) {
            d = __fdividef(cm - cp, den);
            ok = true;
        }
    }
    if (!ok) return 0.f;
    return fminf(fmaxf(d, -1.f), 1.f);
}

// C(s) sqrt(E_A) from the numerator sum A B' over the window, its mean of A and
// the box's sum S1 and 1 / sqrt(E_B); a degenerate box gives +0.
__device__ __forceinline__ float scaled_zncc(float num, float muA, float S1, float nB)
{
    return (num - muA * S1) * nB + 0.f;
}

// Order-preserving key of a float that is not NaN (-0 and +0 are equal once
// canonicalised by scaled_zncc); 0 is left for "no value".
__device__ __forceinline__ uint32_t ord_key(float f)
{
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float log_pos(float c) { return c > 0.f ? __logf(c) : 0.f; }

// Outputs of one window: predictor + integer peak + sub-pixel offsets, the
// info word (bit 0 valid, ky and kx as int8 in bits 8..15 and 16..23); a
// degenerate window passes the predictor through with info 0.
struct WinOut {
    const PassArgs *a;  // the kernel's parameters: pointers are read at the write
    int pair;
    // the predictor at node k (read early, so that its latency overlaps the fit)
    __device__ __forceinline__ float2 pred(int k) const
    {
        const float *pu = (const float *)resolve(a->pred_u, pair);
        const float *pv = (const float *)resolve(a->pred_v, pair);
        return make_float2(pu ? pu[k] : 0.f, pv ? pv[k] : 0.f);
    }
    __device__ __forceinline__ void put(int k, bool ok, int ky, int kx, float dx, float dy) const
    {
        put(k, ok, ky, kx, dx, dy, pred(k));
    }
    __device__ __forceinline__ void put(int k, bool ok, int ky, int kx, float dx, float dy, float2 p) const
    {
        float *ou = (float *)resolve(a->out_u, pair);
        float *ov = (float *)resolve(a->out_v, pair);
        int32_t *oi = (int32_t *)resolve(a->out_info, pair);
        const float pu0 = p.x, pv0 = p.y;
        if (!ok) {
            ou[k] = pu0;
            ov[k] = pv0;
            oi[k] = 0;
            return;
        }
        ou[k] = pu0 + (float)kx + dx;
        ov[k] = pv0 + (float)ky + dy;
        oi[k] = 1 | ((int)(uint8_t)(int8_t)ky << 8) | ((int)(uint8_t)(int8_t)kx << 16);
    }
};

__device__ __forceinline__ WinOut win_out(const PassArgs &a, int pair)
{
    WinOut o;
    o.a = &a;
    o.pair = pair;
    return o;
}

__device__ __forceinline__ void stencil_shift(int p, int ky, int kx, int &sy, int &sx)
{
    // 0 centre, 1 -x, 2 +x, 3 -y, 4 +y
    sy = ky + (p == 3 ? -1 : (p == 4 ? 1 : 0));
    sx = kx + (p == 1 ? -1 : (p == 2 ? 1 : 0));
}

struct WinShared {
    float *c5;    // [nwin][5] stencil values (plane-supplied ones), scaled by sqrt(E_A)
    int *peaks;   // [nwin] plane index of the argmax
    int *need;    // [nwin] bit p set: stencil point p needs a direct FP32 sum
    float *dpart; // [nwin][ng][5] direct numerators per row group
};

// One warp per window: scaled plane from the block planes and box sums, argmax
// (ties keep the smallest row-major index) by two warp reductions, plane values
// of the stencil.  Degenerate windows (E_A <= tau) are skipped: the finalize
// step passes the predictor through for them.
// RC >= 0: compile-time radius; each lane decodes the shifts it owns
// (q = lane + 32 j) once, into plane and box-sum offsets kept in registers.
// ONE_PLANE: one plane per block (FP32 planes), so the block stride is NP.
// ring_wy >= 0: strip mode, the window's block rows yy sit in ring rows
// (ring_wy + yy) & 1.  Returns whether this thread stored a nonzero
// direct-sum mask (some window needs the direct stencil).
template <int RC, bool ONE_PLANE>
static __device__ __forceinline__ bool plane_and_peak(const PassArgs &a, const TileGeom &g, const float *Ps, const float *Vs,
                                      const float *stats, bool tc, const WinShared &ws, int ring_wy = -1,
                                      float moff = 0.f)
{
    const PassPlan &P = a.plan;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int R = RC >= 0 ? RC : g.R;
    const int ND = 2 * R + 1, NP = ND * ND;
    const int kb = g.kb, sg = g.s / g.G;  // blocks per window side, per step
    const int ps = ONE_PLANE ? NP : P.pstride, rs = g.nbx * ps;
    const float tau = TAU_PER_PIXEL * (float)(g.w * g.w);
    const int cp = P.v_pitch;
    const float2 *VV = reinterpret_cast<const float2 *>(Vs);
    constexpr uint32_t NONE = 0xffffffffu;
    // shifts owned by this lane: plane offset q and box-sum offset, per j
    constexpr int NQ = RC >= 0 ? ((2 * RC + 1) * (2 * RC + 1) + 31) / 32 : 1;
    int qv[NQ], vv[NQ];
    if (RC >= 0) {
#pragma unroll
        for (int j = 0; j < NQ; ++j) {
            const int q = min(lane + 32 * j, NP - 1);
            const int qy = q / ND, qx = q - qy * ND;
            qv[j] = q;
            vv[j] = (qy - R) * cp + (qx - R);
        }
    }
    auto block_sum = [&](const float *pb, int q) {
        float num = 0.f;
        for (int yy = 0; yy < kb; ++yy) {
            const int ro = ring_wy < 0 ? yy * rs : ((ring_wy + yy) & 1) * rs;
            for (int xx = 0; xx < kb; ++xx) num += pb[ro + xx * ps + q];
        }
        return num;
    };
    // tensor-core planes are sums of (A - m)(B' - m): the numerator of the
    // definition is P - (mu_A - m)(S1 - n m)
    const float nm = (float)(g.w * g.w) * moff;
    auto coef = [&](float num, float muA, float S1, float nB) {
        return tc ? (num - (muA - moff) * (S1 - nm)) * nB + 0.f : scaled_zncc(num, muA, S1, nB);
    };
    bool any_need = false;
    for (Walk2D wk(warp, nwarps, g.nwx); wk.y < g.nwy; wk.next()) {
        const int wxi = wk.x, wyi = wk.y, wi = wyi * g.nwx + wxi;
        const float muA = stats[2 * wi], EA = stats[2 * wi + 1];
        if (!(EA > tau)) {
            if (lane == 0) {
                ws.peaks[wi] = NP / 2;
                ws.need[wi] = 0;
            }
            continue;
        }
        const float *pb = Ps + ((ring_wy < 0 ? wyi * sg * g.nbx : 0) + wxi * sg) * ps;
        const float2 *vb = VV + (wyi * g.s + R + 1) * cp + wxi * g.s + R + 1;
        float best = 0.f;
        uint32_t bq = NONE;
        // ascending q: the first of equal values stays; NaN never wins
        auto offer = [&](float c, int q) {
            if (c > best || (bq == NONE && c == c)) {
                best = c;
                bq = (uint32_t)q;
            }
        };
        if (RC >= 0) {
#pragma unroll
            for (int j = 0; j < NQ; ++j) {
                if (j < NQ - 1 || lane + 32 * j < NP)
                    offer(coef(block_sum(pb, qv[j]), muA, vb[vv[j]].x, vb[vv[j]].y), qv[j]);
            }
        } else {
            for (int q = lane; q < NP; q += 32) {
                const int qy = q / ND, vo = (qy - R) * cp + (q - qy * ND - R);
                offer(coef(block_sum(pb, q), muA, vb[vo].x, vb[vo].y), q);
            }
        }
        const uint32_t key = bq == NONE ? 0u : ord_key(best);
        const uint32_t kmax = __reduce_max_sync(0xffffffffu, key);
        const uint32_t qmin = __reduce_min_sync(0xffffffffu, (key == kmax && bq != NONE) ? bq : NONE);
        const int bidx = qmin < (uint32_t)NP ? (int)qmin : NP / 2;  // no finite value: zero shift
        const int ky = bidx / ND - R, kx = bidx % ND - R;
        if (lane < 5) {
            int sy, sx;
            stencil_shift(lane, ky, kx, sy, sx);
            const bool inside = sy >= -R && sy <= R && sx >= -R && sx <= R;
            const bool direct = tc || !inside;
            float c = 0.f;
            if (!direct) {
                const int q = (sy + R) * ND + (sx + R), vo = sy * cp + sx;
                c = scaled_zncc(block_sum(pb, q), muA, vb[vo].x, vb[vo].y);
            }
            ws.c5[wi * 5 + lane] = c;
            const unsigned bits = __ballot_sync(0x1fu, direct);
            if (lane == 0) {
                ws.peaks[wi] = bidx;
                ws.need[wi] = (int)bits;
                any_need |= bits != 0u;
            }
        }
    }
    return any_need;
}

// FP32 planes, compile-time radius: two windows per warp, one per half-warp
// (window 2 pw + h for half h), 16 lanes over the shifts q = lane + 16 j, so
// that the per-window set-up, reduction and stencil work is shared by two
// windows.  The half's argmax takes two reductions over its 16 lanes (order
// key, then q): the largest value, ties to the smallest row-major index, NaN
// never winning.  Results as plane_and_peak.
template <int RC>
static __device__ __forceinline__ bool plane_and_peak_pairs(const PassArgs &a, const TileGeom &g, const float *Ps,
                                            const float *Vs, const float *stats, const WinShared &ws,
                                            int ring_wy = -1)
{
    constexpr int R = RC, ND = 2 * RC + 1, NP = ND * ND;
    constexpr int NQ = (NP + 15) / 16;
    constexpr uint32_t NONE = 0xffffffffu;
    const PassPlan &P = a.plan;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int h = lane >> 4, hl = lane & 15;
    const int kb = g.kb, sg = g.s / g.G;
    const int ps = NP, rs = g.nbx * ps;
    const float tau = TAU_PER_PIXEL * (float)(g.w * g.w);
    const int cp = P.v_pitch;
    const float2 *VV = reinterpret_cast<const float2 *>(Vs);
    int qv[NQ], vv[NQ];
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
        const int q = min(hl + 16 * j, NP - 1);
        const int qy = q / ND, qx = q - qy * ND;
        qv[j] = q;
        vv[j] = (qy - R) * cp + (qx - R);
    }
    auto block_sum = [&](const float *pb, int q) {
        float num = 0.f;
        for (int yy = 0; yy < kb; ++yy) {
            const int ro = ring_wy < 0 ? yy * rs : ((ring_wy + yy) & 1) * rs;
            for (int xx = 0; xx < kb; ++xx) num += pb[ro + xx * ps + q];
        }
        return num;
    };
    const int npairs = (g.nwin + 1) >> 1;
    bool any_need = false;
    for (int pw = warp; pw < npairs; pw += nwarps) {
        const int wi = 2 * pw + h;
        const bool has = wi < g.nwin;  // the second half of an odd tile's last pair idles
        const int wic = has ? wi : g.nwin - 1;
        const int wyi = wic / g.nwx, wxi = wic - wyi * g.nwx;
        const float muA = stats[2 * wic], EA = stats[2 * wic + 1];
        const bool live = has && EA > tau;  // degenerate windows: finalize passes the predictor
        const float *pb = Ps + ((ring_wy < 0 ? wyi * sg * g.nbx : 0) + wxi * sg) * ps;
        const float2 *vb = VV + (wyi * g.s + R + 1) * cp + wxi * g.s + R + 1;
        float best = 0.f;
        uint32_t bq = NONE;
        if (live) {
#pragma unroll
            for (int j = 0; j < NQ; ++j) {
                if (j < NQ - 1 || hl + 16 * j < NP) {
                    const float c = scaled_zncc(block_sum(pb, qv[j]), muA, vb[vv[j]].x, vb[vv[j]].y);
                    // ascending q: the first of equal values stays; NaN never wins
                    if (c > best || (bq == NONE && c == c)) {
                        best = c;
                        bq = (uint32_t)qv[j];
                    }
                }
            }
        }
        // the half's argmax: the largest order key, then the smallest q among
        // the lanes that hold it, by two reductions over the half's 16 lanes
        // (each half waits only for its own lanes; both halves run them)
        const uint32_t hmask = 0xffffu << (16 * h);
        const uint32_t key = bq == NONE ? 0u : ord_key(best);
        const uint32_t kmax = __reduce_max_sync(hmask, key);
        const uint32_t kq = __reduce_min_sync(hmask, (key == kmax && bq != NONE) ? bq : NONE);
        const int bidx = kq < (uint32_t)NP ? (int)kq : NP / 2;  // no finite value: zero shift
        const int ky = bidx / ND - R, kx = bidx % ND - R;
        float c = 0.f;
        bool direct = false;
        if (hl < 5 && live) {
            int sy, sx;
            stencil_shift(hl, ky, kx, sy, sx);
            direct = !(sy >= -R && sy <= R && sx >= -R && sx <= R);
            if (!direct) {
                const int q = (sy + R) * ND + (sx + R), vo = sy * cp + sx;
                c = scaled_zncc(block_sum(pb, q), muA, vb[vo].x, vb[vo].y);
            }
        }
        const unsigned bits = (__ballot_sync(0xffffffffu, direct) >> (16 * h)) & 0x1fu;
        if (has && hl < 5) ws.c5[wi * 5 + hl] = c;
        if (has && hl == 0) {
            ws.peaks[wi] = live ? bidx : NP / 2;
            ws.need[wi] = live ? (int)bits : 0;
            any_need |= live && bits != 0u;
        }
    }
    return any_need;
}

// Row groups per window in the direct stencil: enough (window, group) items
// for the CTA's warps when a tile has fewer windows than warps.
__device__ __forceinline__ int stencil_groups(int nwin, int w, int nwarps) { return min(max(1, nwarps / nwin), w); }

// Direct FP32 numerators of the stencil points the plane cannot supply: one
// warp per (window, row group), lanes over the group's pixels, five
// accumulators; dpart[(wi ng + gr) 5 + p] holds a group's partial sum.
static __device__ __forceinline__ void stencil_direct(const PassArgs &a, const TileGeom &g, const float *As, const float *Bs,
                                      const WinShared &ws)
{
    const PassPlan &P = a.plan;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int w = g.w, R = g.R, ND = g.ND;
    const int ng = stencil_groups(g.nwin, w, nwarps);
    const int bpt = P.b_pitch;
    for (int it = warp; it < g.nwin * ng; it += nwarps) {
        const int wi = it / ng, gr = it - wi * ng;
        const int need = ws.need[wi];
        if (!need) continue;
        const int q = ws.peaks[wi];
        const int ky = q / ND - R, kx = q % ND - R;
        const int wyi = wi / g.nwx, wxi = wi - wyi * g.nwx;
        const int r0 = gr * w / ng, r1 = (gr + 1) * w / ng;
        const float *abase = As + (wyi * g.s + r0) * P.a_pitch + wxi * g.s;
        // B' at A pixel (r, x) and shift (sy, sx): row r + sy + R + 1, column x + sx + padl
        const float *bbase = Bs + (wyi * g.s + r0 + ky + R + 1) * bpt + P.padl + wxi * g.s + kx;
        float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (need == 0x1f) {
            for (Walk2D e(lane, 32, w); e.y < r1 - r0; e.next()) {
                const float av = abase[e.y * P.a_pitch + e.x];
                const float *bb = bbase + e.y * bpt + e.x;
                acc[0] = fmaf(av, bb[0], acc[0]);
                acc[1] = fmaf(av, bb[-1], acc[1]);
                acc[2] = fmaf(av, bb[1], acc[2]);
                acc[3] = fmaf(av, bb[-bpt], acc[3]);
                acc[4] = fmaf(av, bb[bpt], acc[4]);
            }
        } else {
            for (Walk2D e(lane, 32, w); e.y < r1 - r0; e.next()) {
                const float av = abase[e.y * P.a_pitch + e.x];
                const float *bb = bbase + e.y * bpt + e.x;
                if (need & 1) acc[0] = fmaf(av, bb[0], acc[0]);
                if (need & 2) acc[1] = fmaf(av, bb[-1], acc[1]);
                if (need & 4) acc[2] = fmaf(av, bb[1], acc[2]);
                if (need & 8) acc[3] = fmaf(av, bb[-bpt], acc[3]);
                if (need & 16) acc[4] = fmaf(av, bb[bpt], acc[4]);
            }
        }
#pragma unroll
        for (int p = 0; p < 5; ++p)
            if (need & (1 << p)) acc[p] = warp_sum(acc[p]);
        if (lane < 5) {
            float v = acc[0];
#pragma unroll
            for (int p = 1; p < 5; ++p)
                if (lane == p) v = acc[p];
            ws.dpart[it * 5 + lane] = v;
        }
    }
}

// Stencil values, Gaussian fit and outputs (one thread per window).
static __device__ __forceinline__ void finalize(const PassArgs &a, const TileGeom &g, const float *Vs, const float *stats,
                                const WinShared &ws, int pair)
{
    const PassPlan &P = a.plan;
    const int w = g.w, R = g.R, ND = g.ND;
    const int ng = stencil_groups(g.nwin, w, blockDim.x >> 5);
    const int cp = P.v_pitch;
    const float2 *VV = reinterpret_cast<const float2 *>(Vs);
    const WinOut out = win_out(a, pair);
    const float tau = TAU_PER_PIXEL * (float)(w * w);
    for (int wi = threadIdx.x; wi < g.nwin; wi += blockDim.x) {
        const int wyi = wi / g.nwx, wxi = wi - wyi * g.nwx;
        const int k = (g.wy0 + wyi) * a.nx + (g.wx0 + wxi);
        const float2 p0 = out.pred(k);
        const float muA = stats[2 * wi], EA = stats[2 * wi + 1];
        if (!(EA > tau)) {
            out.put(k, false, 0, 0, 0.f, 0.f, p0);
            continue;
        }
        const int q = ws.peaks[wi], need = ws.need[wi];
        const int ky = q / ND - R, kx = q % ND - R;
        const float inv_a = rsqrtf(EA);
        float c5[5], l5[5];
#pragma unroll
        for (int p = 0; p < 5; ++p) {
            float c;
            if (need & (1 << p)) {
                int sy, sx;
                stencil_shift(p, ky, kx, sy, sx);
                float num = 0.f;
                for (int gr = 0; gr < ng; ++gr) num += ws.dpart[(wi * ng + gr) * 5 + p];
                const int vo = (wyi * g.s + R + 1 + sy) * cp + wxi * g.s + R + 1 + sx;
                c = scaled_zncc(num, muA, VV[vo].x, VV[vo].y);
            } else {
                c = ws.c5[wi * 5 + p];
            }
            c5[p] = c * inv_a;
            l5[p] = log_pos(c5[p]);
        }
        const float dx = gauss3f(c5[1], c5[0], c5[2], l5[1], l5[0], l5[2]);
        const float dy = gauss3f(c5[3], c5[0], c5[4], l5[3], l5[0], l5[4]);
        out.put(k, true, ky, kx, dx, dy, p0);
    }
}

// A tile whose region load did not complete: its windows are reported
// invalid (the predictor passes through, info 0), as for a degenerate window,
// so that the outlier test replaces them; the error word carries the event.
static __device__ __forceinline__ void invalid_tile(const PassArgs &a, const TileGeom &g, int pair)
{
    const float *pu = (const float *)resolve(a.pred_u, pair);
    const float *pv = (const float *)resolve(a.pred_v, pair);
    float *ou = (float *)resolve(a.out_u, pair);
    float *ov = (float *)resolve(a.out_v, pair);
    int32_t *oi = (int32_t *)resolve(a.out_info, pair);
    for (int wi = threadIdx.x; wi < g.nwin; wi += blockDim.x) {
        const int k = (g.wy0 + wi / g.nwx) * a.nx + (g.wx0 + wi % g.nwx);
        ou[k] = pu ? pu[k] : 0.f;
        ov[k] = pv ? pv[k] : 0.f;
        oi[k] = 0;
    }
}

// ------------------------------------------------------------- the kernel --

// GC > 0: a kernel specialised for blocks of GC pixels, windows of 2 GC and
// steps of GC (50 % overlap), so that window, step and block loops unroll.
// FP32 kernels up to r = 4 are bounded to five CTAs per SM (48 registers),
// except the 64 px windows and the 16 px windows at r = 4, whose tiles are
// planned for three.
template <int RC, int PREC, int GC>
__global__ void __launch_bounds__(PASS_THREADS,
                                  (PREC == PREC_FP32 && (RC >= 0 && RC <= 4) && GC != 32 && !(GC == 8 && RC == 4)) ? 5 : 3)
    pass_kernel(const __grid_constant__ PassArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const PassPlan &P = a.plan;
    TileGeom g;
    g.R = RC >= 0 ? RC : a.R;
    g.ND = 2 * g.R + 1;
    g.NP = g.ND * g.ND;
    g.G = GC > 0 ? GC : P.G;
    g.w = GC > 0 ? 2 * GC : a.w;
    g.s = GC > 0 ? GC : a.s;
    g.kb = g.w / g.G;
    const int pair = blockIdx.z;
    const int s = g.s, w = g.w;
    g.wx0 = blockIdx.x * P.TX;
    g.wy0 = blockIdx.y * P.TY;
    g.nwx = min(P.TX, a.nx - g.wx0);
    g.nwy = min(P.TY, a.ny - g.wy0);
    g.nwin = g.nwx * g.nwy;
    g.aw = (g.nwx - 1) * s + w;
    g.ah = (g.nwy - 1) * s + w;
    g.ax0 = g.wx0 * s;
    g.ay0 = g.wy0 * s;
    g.BC = g.aw + 2 * (g.R + 1);
    g.BR = g.ah + 2 * (g.R + 1);
    g.OFFB = P.padl - (g.R + 1);
    g.hw = g.BC - w + 1;
    g.vh = g.BR - w + 1;
    g.nbx = g.aw / g.G;
    g.nby = g.ah / g.G;
    g.nb = g.nbx * g.nby;

    float *As = reinterpret_cast<float *>(smem + P.off_a);
    float *Bs = reinterpret_cast<float *>(smem + P.off_b);
    float *Cs = reinterpret_cast<float *>(smem + P.off_h);
    float *Vs = reinterpret_cast<float *>(smem + P.off_v);
    float *Ps = reinterpret_cast<float *>(smem + P.off_p);
    float *stats = reinterpret_cast<float *>(smem + P.off_stats);
    float2 *bst = reinterpret_cast<float2 *>(smem + P.off_gst);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + P.off_red);
    uint16_t *TA = reinterpret_cast<uint16_t *>(smem + P.off_tca);
    uint16_t *TB = reinterpret_cast<uint16_t *>(smem + P.off_tcb);
    WinShared ws;
    ws.c5 = reinterpret_cast<float *>(smem + P.off_c5);
    ws.peaks = reinterpret_cast<int *>(smem + P.off_peaks);
    ws.need = reinterpret_cast<int *>(smem + P.off_need);
    ws.dpart = reinterpret_cast<float *>(smem + P.off_dpart);

    // 1: A and B' regions
    // every thread leaves together if any thread's bounded wait gave up (error word set)
    const bool loaded = load_regions(a, g, pair, As, Bs, bar);
    if (__syncthreads_or(!loaded)) {
        invalid_tile(a, g, pair);
        return;
    }

    // 2: A window statistics, box sums of B' for every window and shift
    block_stats(a, g, As, bst);
    box_sums(a, g, Bs, Cs, Vs);  // contains a barrier between its two passes
    __syncthreads();
    window_stats(a, g, bst, stats);
    float moff = 0.f;
    if (PREC != PREC_FP32) {
        // tile offset: the mean of the A region, from the block sums in a fixed
        // order (kept after the region loads' barrier)
        float *off_slot = reinterpret_cast<float *>(bar + 1);
        if ((threadIdx.x >> 5) == 0) {
            const int lane = threadIdx.x & 31;
            float sum = 0.f;
            for (int b = lane; b < g.nb; b += 32) sum += bst[b].x;
            sum = warp_sum(sum);
            if (lane == 0) *off_slot = sum / (float)(g.aw * g.ah);
        }
        __syncthreads();
        moff = *off_slot;
        // 16-bit copies of the regions for the tensor cores, over the dead C region
        tc_copies<PREC>(a, g, As, Bs, TA, TB, moff);
        __syncthreads();
    }

    // 3: block planes (alias the dead C region)
    if (PREC == PREC_FP32) {
        if (RC >= 0)
            block_planes_fp32<(RC >= 0 ? RC : 0)>(a, g, As, Bs, Ps);
        else
            block_planes_fp32_generic(a, g, As, Bs, Ps);
    } else {
        block_planes_tc<(RC >= 0 ? RC : 0), PREC>(a, g, TA, TB, Ps);
    }
    __syncthreads();
    if (PREC != PREC_FP32 && P.RGx > 1) {
        reduce_row_groups(a, g, Ps);
        __syncthreads();
    }

    // 4: plane, argmax, FP32 stencil, Gaussian fit, outputs
    constexpr bool tc = PREC != PREC_FP32;
    // two windows per warp once the tile has at least two per warp (16 px
    // tiles: 1.207 -> 1.198 ms per 64-pair launch; with fewer windows the
    // warps left idle cost more than the shared set-up saves)
    bool needs;
    if (PREC == PREC_FP32 && RC >= 0 && g.nwin >= 2 * (int)(blockDim.x >> 5))
        needs = plane_and_peak_pairs<(RC >= 0 ? RC : 0)>(a, g, Ps, Vs, stats, ws);
    else
        needs = plane_and_peak<RC, PREC == PREC_FP32>(a, g, Ps, Vs, stats, tc, ws, -1, moff);
    // the direct stencil and its barrier only when some window needs them
    // (peaks at the edge of the search, and every window on the 16-bit path)
    if (__syncthreads_or(needs)) {
        stencil_direct(a, g, As, Bs, ws);
        __syncthreads();
    }
    finalize(a, g, Vs, stats, ws, pair);
}

// A strip: one CTA walks P.strip_rows window rows of a one-row tile of TX
// windows (50 % overlap, blocks of GC px: a window is 2 x 2 blocks).  Each step
// loads its regions (the rows it shares with the previous step come from L2),
// recomputes the box sums, computes the statistics and the planes of the block
// row it adds (both block rows on its first step) into two-row rings, and takes
// the block row it shares with the previous window row from the rings.  The
// next step's copies are issued once the regions are last read (after the
// direct stencil, when a window needs it), so that they overlap the fit.  GC is
// a multiple of 4: every region row is one bulk copy.
template <int RC, int GC>
__global__ void __launch_bounds__(PASS_THREADS, GC == 32 ? 3 : 4) strip_kernel(const __grid_constant__ PassArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const PassPlan &P = a.plan;
    TileGeom g;
    g.R = RC;
    g.ND = 2 * RC + 1;
    g.NP = g.ND * g.ND;
    g.G = GC;
    g.w = 2 * GC;
    g.s = GC;
    g.kb = 2;
    const int pair = blockIdx.z;
    const int s = g.s, w = g.w;
    g.wx0 = blockIdx.x * P.TX;
    g.nwx = min(P.TX, a.nx - g.wx0);
    g.nwy = 1;
    g.nwin = g.nwx;
    g.aw = (g.nwx - 1) * s + w;
    g.ah = w;
    g.ax0 = g.wx0 * s;
    g.BC = g.aw + 2 * (g.R + 1);
    g.BR = g.ah + 2 * (g.R + 1);
    g.OFFB = P.padl - (g.R + 1);
    g.hw = g.BC - w + 1;
    g.vh = g.BR - w + 1;
    g.nbx = g.aw / g.G;
    g.nby = 2;
    g.nb = 2 * g.nbx;

    float *As = reinterpret_cast<float *>(smem + P.off_a);
    float *Bs = reinterpret_cast<float *>(smem + P.off_b);
    float *Cs = reinterpret_cast<float *>(smem + P.off_h);
    float *Vs = reinterpret_cast<float *>(smem + P.off_v);
    float *Ps = reinterpret_cast<float *>(smem + P.off_p);
    float *stats = reinterpret_cast<float *>(smem + P.off_stats);
    float2 *bst = reinterpret_cast<float2 *>(smem + P.off_gst);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + P.off_red);
    WinShared ws;
    ws.c5 = reinterpret_cast<float *>(smem + P.off_c5);
    ws.peaks = reinterpret_cast<int *>(smem + P.off_peaks);
    ws.need = reinterpret_cast<int *>(smem + P.off_need);
    ws.dpart = reinterpret_cast<float *>(smem + P.off_dpart);

    const int wy_begin = blockIdx.y * P.strip_rows, wy_end = min(a.ny, wy_begin + P.strip_rows);
    g.wy0 = wy_begin;
    g.ay0 = wy_begin * s;
    if (threadIdx.x < 32) issue_regions(a, g, pair, As, Bs, bar, 0);
    for (int wy = wy_begin; wy < wy_end; ++wy) {
        const int k = wy - wy_begin;
        g.wy0 = wy;
        g.ay0 = wy * s;
        // 1: A and B' regions of this window row (issued the step before)
        const bool loaded = threadIdx.x < 32 ? wait_regions(a, bar, k) : true;
        if (__syncthreads_or(!loaded)) {
            for (int r = wy; r < wy_end; ++r) {
                g.wy0 = r;
                invalid_tile(a, g, pair);
            }
            return;
        }
        // 2: statistics and box sums of the row
        block_stats(a, g, As, bst, k == 0 ? 0 : g.nbx, wy);
        box_cols(a, g, Bs, Cs, true);
        __syncthreads();
        // 3: the row pass of the box sums and the window statistics beside the
        // planes of the block row this step adds: the planes' ring lies apart
        // from the column sums, so no barrier separates them (the warps with
        // row items take their plane items after them)
        box_rows(a, g, Cs, Vs);
        window_stats(a, g, bst, stats, wy);
        block_planes_fp32<RC>(a, g, As, Bs, Ps, k == 0 ? 0 : g.nbx, wy);
        __syncthreads();
        // 4: plane, argmax, FP32 stencil, Gaussian fit, outputs
        // the direct stencil and its barrier only when some window needs them
        if (__syncthreads_or(plane_and_peak<RC, true>(a, g, Ps, Vs, stats, false, ws, wy))) {
            stencil_direct(a, g, As, Bs, ws);
            __syncthreads();
        }
        // the regions are read no more in this step: the next step's copies go
        // out now, behind the CTA barrier that ordered the reads, from warp 1,
        // so that they do not wait for the fit that warp 0's first lanes run
        // (warp 0 initialised the barrier before the loop and waits on it)
        if (wy + 1 < wy_end && threadIdx.x >= 32 && threadIdx.x < 64) {
            TileGeom gn = g;
            gn.wy0 = wy + 1;
            gn.ay0 = (wy + 1) * s;
            issue_regions(a, gn, pair, As, Bs, bar, k + 1);
        }
        finalize(a, g, Vs, stats, ws, pair);
        // the next step overwrites the sums and the window buffers
        __syncthreads();
    }
}

}  // namespace rpiv
