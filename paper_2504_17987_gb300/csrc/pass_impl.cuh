// Fused correlation pass: image deformation, zero-normalised correlation
// plane over a +-R search, integer peak, FP32 5-point refit and three-point
// Gaussian fit, for a tile of TX x TY interrogation windows per CTA
// (paper Sec. 2: warp the pair by the predictor, correlation coefficients on
// a stencil around the peak, Gaussian sub-pixel interpolation).
//
// Layout of the work in one CTA (all staged in shared memory):
//   A region   A - mu_T over the union of the tile's windows (aw x ah)
//   B' region  B(x + d(x)) - mu_T over the A region grown by R+1 on each side
//   H, V       sliding box sums of B' and B'^2: V[r][c] is the sum over the
//              w x w box with top-left (r, c), i.e. sum_x B'(x + s) of every
//              window at every shift s in [-R-1, R+1]^2 by lookup
//   P          block partial planes: the A region is cut into G x G blocks
//              (G = gcd(w, s)); P_b(s) = sum_{x in b} A_c(x) B'_c(x + s).
//              A window's numerator is the sum of its (w/G)^2 block planes
//              minus mean(A_c) * sum B'_c(x + s); this regrouping is exact,
//              and it computes each block once instead of once per
//              overlapping window.
//   The plane is formed either with FP32 FMAs on the CUDA cores, or with
//   BF16/FP16 tensor-core MMAs (mma.sync m16n8k8, FP32 accumulate) whose
//   accumulator tile D[i][j] (i = B' row, j = A row of an 8-row sub-block)
//   holds shift sy = i - j - R on its diagonals.  The argmax is taken on the
//   plane; the 5-point stencil for the Gaussian fit is evaluated in FP32
//   (from the FP32 block planes, or directly on the TC path).
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

// Node index i0 (local to the grid) and weight t of node i0+1 for an image
// position along one axis; outside the node hull the border node is used.
__device__ __forceinline__ void axis_w(int pos, int n, float c0, int s, int &i0, float &t)
{
    if (n <= 1) {
        i0 = 0;
        t = 0.f;
        return;
    }
    float f = ((float)pos - c0) / (float)s;
    f = fminf(fmaxf(f, 0.f), (float)(n - 1));
    int ia = (int)floorf(f);
    if (ia > n - 2) ia = n - 2;
    i0 = ia;
    t = f - (float)ia;
}

template <typename T>
__device__ __forceinline__ float ld_px(const unsigned char *img, long long pitch, int x, int y)
{
    return (float)__ldg(reinterpret_cast<const T *>(img + (long long)y * pitch) + x);
}

// Bilinear sample of the image at (x + dx, y + dy), clamp-to-edge; x, y integer.
template <typename T>
__device__ __forceinline__ float sample_img(const unsigned char *img, long long pitch, int W, int H, int x, int y,
                                            float dx, float dy)
{
    // non-finite or absurd displacements are clamped so that the integer
    // arithmetic below cannot overflow
    dx = isfinite(dx) ? fminf(fmaxf(dx, -1048576.f), 1048576.f) : 0.f;
    dy = isfinite(dy) ? fminf(fmaxf(dy, -1048576.f), 1048576.f) : 0.f;
    const float fx = floorf(dx), fy = floorf(dy);
    const float tx = dx - fx, ty = dy - fy;
    const int ix = x + (int)fx, iy = y + (int)fy;
    const int x0 = min(max(ix, 0), W - 1), x1 = min(max(ix + 1, 0), W - 1);
    const int y0 = min(max(iy, 0), H - 1), y1 = min(max(iy + 1, 0), H - 1);
    const float b00 = ld_px<T>(img, pitch, x0, y0), b10 = ld_px<T>(img, pitch, x1, y0);
    const float b01 = ld_px<T>(img, pitch, x0, y1), b11 = ld_px<T>(img, pitch, x1, y1);
    const float top = b00 + tx * (b10 - b00);
    const float bot = b01 + tx * (b11 - b01);
    return top + ty * (bot - top);
}

struct TileGeom {
    int R, ND, NP;
    int wx0, wy0, nwx, nwy, nwin;
    int aw, ah, ax0, ay0;
    int BC, BR, OFFB;
    int hw, vh;
    int nbx, nby, nb;
    int nodes_w;  // nodes per row in the local node grid
    int i_lo, j_lo;
};

// ----------------------------------------------------------- phases 0..2 --

template <typename T>
__device__ void load_and_deform(const PassArgs &a, const TileGeom &g, const unsigned char *imgA,
                                const unsigned char *imgB, bool has_pred, const float *nodes, const int *ti,
                                const float *tf, float *As, float *Bs, float *red, float &muT_out)
{
    const PassPlan &P = a.plan;
    const int tid = threadIdx.x;
    const int R = g.R;
    // field at a B'-region pixel (logical column bx, row by)
    auto field = [&](int bx, int by, float &du, float &dv) {
        if (!has_pred) {
            du = 0.f;
            dv = 0.f;
            return;
        }
        const int i0 = ti[bx], j0 = ti[g.BC + by];
        const float tx = tf[bx], ty = tf[g.BC + by];
        const int i1 = i0 + (a.nx > 1 ? 1 : 0), j1 = j0 + (a.ny > 1 ? 1 : 0);
        const float *nu = nodes, *nv = nodes + P.node_cap;
        const int q = g.nodes_w;
        float t0 = nu[j0 * q + i0] + tx * (nu[j0 * q + i1] - nu[j0 * q + i0]);
        float t1 = nu[j1 * q + i0] + tx * (nu[j1 * q + i1] - nu[j1 * q + i0]);
        du = t0 + ty * (t1 - t0);
        t0 = nv[j0 * q + i0] + tx * (nv[j0 * q + i1] - nv[j0 * q + i0]);
        t1 = nv[j1 * q + i0] + tx * (nv[j1 * q + i1] - nv[j1 * q + i0]);
        dv = t0 + ty * (t1 - t0);
    };
    // A region (central mode: A warped by -d/2)
    float local = 0.f;
    const int na = g.aw * g.ah;
    for (int e = tid; e < na; e += blockDim.x) {
        const int y = e / g.aw, x = e - y * g.aw;
        float val;
        if (a.deform == 1 && has_pred) {
            float du, dv;
            field(x + R + 1, y + R + 1, du, dv);
            val = sample_img<T>(imgA, a.pitch, a.W, a.H, g.ax0 + x, g.ay0 + y, -0.5f * du, -0.5f * dv);
        } else {
            val = ld_px<T>(imgA, a.pitch, g.ax0 + x, g.ay0 + y);
        }
        As[y * P.a_pitch + x] = val;
        local += val;
    }
    // tile mean of A: the common offset removed from A and B' (ZNCC is
    // invariant to it; it keeps the FP32 box sums well conditioned)
    local = warp_sum(local);
    if ((tid & 31) == 0) red[tid >> 5] = local;
    __syncthreads();
    if (tid < 32) {
        float v = tid < (int)(blockDim.x >> 5) ? red[tid] : 0.f;
        v = warp_sum(v);
        if (tid == 0) red[32] = v / (float)na;
    }
    __syncthreads();
    const float muT = red[32];
    muT_out = muT;
    for (int e = tid; e < na; e += blockDim.x) {
        const int y = e / g.aw, x = e - y * g.aw;
        As[y * P.a_pitch + x] -= muT;
    }
    const float scale = (a.deform == 1) ? 0.5f : 1.0f;
    const int nbp = g.BC * g.BR;
    for (int e = tid; e < nbp; e += blockDim.x) {
        const int by = e / g.BC, bx = e - by * g.BC;
        float du, dv;
        field(bx, by, du, dv);
        const int x = g.ax0 - (R + 1) + bx, y = g.ay0 - (R + 1) + by;
        Bs[by * P.b_pitch + g.OFFB + bx] = sample_img<T>(imgB, a.pitch, a.W, a.H, x, y, scale * du, scale * dv) - muT;
    }
}

// ------------------------------------------------------ box sums (H, V) --

static __device__ void box_sums(const PassArgs &a, const TileGeom &g, const float *Bs, float *Hs, float *Vs)
{
    const PassPlan &P = a.plan;
    const int w = a.w, tid = threadIdx.x;
    // H[r][c] = sum_{x=c}^{c+w-1} B'[r][x] (logical columns), segments of 8
    const int nseg = (g.hw + 7) / 8;
    for (int it = tid; it < g.BR * nseg; it += blockDim.x) {
        const int by = it / nseg, seg = it - by * nseg;
        const int c_lo = seg * 8, c_hi = min(g.hw, c_lo + 8);
        const float *row = Bs + by * P.b_pitch + g.OFFB;
        float s1 = 0.f, s2 = 0.f;
        for (int x = c_lo; x < c_lo + w; ++x) {
            const float b = row[x];
            s1 += b;
            s2 = fmaf(b, b, s2);
        }
        float *h1 = Hs + by * P.h_pitch;
        float *h2 = Hs + (g.BR + by) * P.h_pitch;
        h1[c_lo] = s1;
        h2[c_lo] = s2;
        for (int c = c_lo + 1; c < c_hi; ++c) {
            const float bo = row[c - 1], bi = row[c + w - 1];
            s1 += bi - bo;
            s2 += bi * bi - bo * bo;
            h1[c] = s1;
            h2[c] = s2;
        }
    }
    __syncthreads();
    // V[r][c] = sum_{y=r}^{r+w-1} H[y][c], segments of 8 rows
    const int nsegv = (g.vh + 7) / 8;
    for (int it = tid; it < g.hw * nsegv; it += blockDim.x) {
        const int c = it / nsegv, seg = it - c * nsegv;
        const int r_lo = seg * 8, r_hi = min(g.vh, r_lo + 8);
        const float *h1 = Hs + c, *h2 = Hs + g.BR * P.h_pitch + c;
        float s1 = 0.f, s2 = 0.f;
        for (int y = r_lo; y < r_lo + w; ++y) {
            s1 += h1[y * P.h_pitch];
            s2 += h2[y * P.h_pitch];
        }
        float *v1 = Vs + c, *v2 = Vs + g.vh * P.h_pitch + c;
        v1[r_lo * P.h_pitch] = s1;
        v2[r_lo * P.h_pitch] = s2;
        for (int r = r_lo + 1; r < r_hi; ++r) {
            s1 += h1[(r + w - 1) * P.h_pitch] - h1[(r - 1) * P.h_pitch];
            s2 += h2[(r + w - 1) * P.h_pitch] - h2[(r - 1) * P.h_pitch];
            v1[r * P.h_pitch] = s1;
            v2[r * P.h_pitch] = s2;
        }
    }
}

// Per-window mean and energy of A_c (two-pass, one warp per window).
static __device__ void window_stats(const PassArgs &a, const TileGeom &g, const float *As, float *stats)
{
    const PassPlan &P = a.plan;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int w = a.w, n = w * w;
    for (int wi = warp; wi < g.nwin; wi += nwarps) {
        const int wxi = wi % g.nwx, wyi = wi / g.nwx;
        const float *base = As + (wyi * a.s) * P.a_pitch + wxi * a.s;
        float s = 0.f;
        for (int e = lane; e < n; e += 32) s += base[(e / w) * P.a_pitch + (e % w)];
        const float mean = warp_sum(s) / (float)n;
        float q = 0.f;
        for (int e = lane; e < n; e += 32) {
            const float d = base[(e / w) * P.a_pitch + (e % w)] - mean;
            q = fmaf(d, d, q);
        }
        q = warp_sum(q);
        if (lane == 0) {
            stats[2 * wi] = mean;
            stats[2 * wi + 1] = q;
        }
    }
}

// --------------------------------------------- FP32 block planes (CUDA cores) --

// Compile-time radius: each thread owns one (block, sy, row group) and keeps
// the 2R+1 accumulators of its sx row in registers; rows are streamed from
// shared memory four columns at a time with aligned 128-bit loads.
template <int R>
__device__ void block_planes_fp32(const PassArgs &a, const TileGeom &g, const float *As, const float *Bs, float *Ps)
{
    constexpr int ND = 2 * R + 1;
    constexpr int NP = ND * ND;
    constexpr int MIS = ((-R) % 4 + 4) % 4;
    constexpr int NQ = (4 + 2 * R + MIS + 3) / 4;
    const PassPlan &P = a.plan;
    const int G = P.G, RG = P.RGx, rows = G / RG;
    const int items = g.nb * ND * RG;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int syi = it % ND;
        const int rest = it / ND;
        const int gi = rest % RG;
        const int b = rest / RG;
        const int bxi = b % g.nbx, byi = b / g.nbx;
        const int c0 = bxi * G, r0 = byi * G + gi * rows;
        float acc[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) acc[d] = 0.f;
        for (int y = r0; y < r0 + rows; ++y) {
            const float *arow = As + y * P.a_pitch;
            const float *brow = Bs + (y + syi + 1) * P.b_pitch + P.padl - R - MIS;
            for (int c = c0; c < c0 + G; c += 4) {
                const float4 a4 = *reinterpret_cast<const float4 *>(arow + c);
                float bv[NQ * 4];
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const float4 t = *reinterpret_cast<const float4 *>(brow + c + 4 * q);
                    bv[4 * q] = t.x;
                    bv[4 * q + 1] = t.y;
                    bv[4 * q + 2] = t.z;
                    bv[4 * q + 3] = t.w;
                }
                const float av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
#pragma unroll
                    for (int d = 0; d < ND; ++d) acc[d] = fmaf(av[j], bv[MIS + j + d], acc[d]);
                }
            }
        }
        float *out = Ps + (size_t)(b * RG + gi) * NP + syi * ND;
#pragma unroll
        for (int d = 0; d < ND; ++d) out[d] = acc[d];
    }
}

// Runtime radius (any R up to RPIV_MAX_RADIUS): scalar loads, sx in chunks of 8.
static __device__ void block_planes_fp32_generic(const PassArgs &a, const TileGeom &g, const float *As, const float *Bs,
                                          float *Ps)
{
    const PassPlan &P = a.plan;
    const int R = g.R, ND = g.ND, NP = g.NP;
    const int G = P.G, RG = P.RGx, rows = G / RG;
    const int nch = (ND + 7) / 8;
    const int items = g.nb * ND * RG * nch;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        int rest = it;
        const int ch = rest % nch;
        rest /= nch;
        const int syi = rest % ND;
        rest /= ND;
        const int gi = rest % RG;
        const int b = rest / RG;
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
        float *out = Ps + (size_t)(b * RG + gi) * NP + syi * ND + d0;
        for (int d = 0; d < 8 && d0 + d < ND; ++d) out[d] = acc[d];
    }
}

// ------------------------------------------- tensor-core block planes --

template <int PREC>
__device__ __forceinline__ uint16_t to_h16(float x)
{
    if (PREC == PREC_BF16) return __bfloat16_as_ushort(__float2bfloat16_rn(x));
    return __half_as_ushort(__float2half_rn(x));
}

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

// 16-bit copies for the tensor-core path: A_c, and B'_c twice (the second
// shifted by one column so that every pair of columns starts 4-byte aligned).
template <int PREC>
__device__ void tc_convert(const PassArgs &a, const TileGeom &g, const float *As, const float *Bs, uint16_t *TA,
                           uint16_t *TB)
{
    const PassPlan &P = a.plan;
    const int tid = threadIdx.x;
    const int arows = ((g.ah + 7) / 8) * 8 + 8;
    for (int e = tid; e < arows * P.tca_pitch; e += blockDim.x) {
        const int y = e / P.tca_pitch, x = e - y * P.tca_pitch;
        const float v = (y < g.ah && x < g.aw) ? As[y * P.a_pitch + x] : 0.f;
        TA[e] = to_h16<PREC>(v);
    }
    const int brows = g.BR + 32;
    const int lo = g.OFFB, hi = g.OFFB + g.BC;
    uint16_t *TB1 = TB + brows * P.tcb_pitch;
    for (int e = tid; e < brows * P.tcb_pitch; e += blockDim.x) {
        const int y = e / P.tcb_pitch, x = e - y * P.tcb_pitch;
        const float v0 = (y < g.BR && x >= lo && x < hi) ? Bs[y * P.b_pitch + x] : 0.f;
        const float v1 = (y < g.BR && x + 1 >= lo && x + 1 < hi) ? Bs[y * P.b_pitch + x + 1] : 0.f;
        TB[e] = to_h16<PREC>(v0);
        TB1[e] = to_h16<PREC>(v1);
    }
}

// One warp per (block, 8-row sub-block).  For each chunk of at most 9 shifts
// sx the accumulators D[i][j] (i: B' row offset, j: A row offset) are summed
// over the sub-block's 8-column chunks; shift sy = i - j - R is recovered from
// the diagonals through a per-warp scratch buffer.
template <int R, int PREC>
__device__ void block_planes_tc(const PassArgs &a, const TileGeom &g, const uint16_t *TA, const uint16_t *TB,
                                float *scratch, float *Ps)
{
    constexpr int ND = 2 * R + 1;
    constexpr int NP = ND * ND;
    constexpr int MT = (8 + 2 * R + 15) / 16;
    constexpr int SXC = ND < 9 ? ND : 9;
    const PassPlan &P = a.plan;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int gq = lane >> 2, tq = lane & 3;
    const int G = P.G;
    const int nsb = (G + 7) / 8, nkc = (G + 7) / 8;
    const int brows = g.BR + 32;
    const uint16_t *TB1 = TB + brows * P.tcb_pitch;
    float *scr = scratch + warp * (SXC * ND * 8);
    const int items = g.nb * nsb;
    for (int it = warp; it < items; it += nwarps) {
        const int b = it / nsb, sb = it - b * nsb;
        const int bxi = b % g.nbx, byi = b / g.nbx;
        const int Y0 = byi * G + sb * 8;  // first A row of the sub-block (A-region coords)
        const int X0 = bxi * G;
        const bool row_ok = (sb * 8 + gq) < G;
        for (int sx0 = -R; sx0 <= R; sx0 += SXC) {
            float acc[SXC][MT][4];
#pragma unroll
            for (int q = 0; q < SXC; ++q)
#pragma unroll
                for (int m = 0; m < MT; ++m)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[q][m][e] = 0.f;
            for (int kc = 0; kc < nkc; ++kc) {
                const int X = X0 + kc * 8;
                const bool col_ok = (kc * 8 + 2 * tq) < G;
                const uint32_t bfrag =
                    (row_ok && col_ok)
                        ? *reinterpret_cast<const uint32_t *>(TA + (Y0 + gq) * P.tca_pitch + X + 2 * tq)
                        : 0u;
#pragma unroll
                for (int q = 0; q < SXC; ++q) {
                    const int sx = sx0 + q;
                    if (sx > R) break;
                    // smem column of A column X + 2tq at shift sx; pick the copy that makes it even
                    const int col = X + 2 * tq + sx + P.padl;
                    const uint16_t *src = (col & 1) ? TB1 : TB;
                    const int c2 = col & ~1;
#pragma unroll
                    for (int m = 0; m < MT; ++m) {
                        // B' logical row of A row Y0 + i - R is Y0 + i + 1
                        const int r0 = Y0 + 1 + 16 * m + gq;
                        const uint32_t a0 = *reinterpret_cast<const uint32_t *>(src + r0 * P.tcb_pitch + c2);
                        const uint32_t a1 = *reinterpret_cast<const uint32_t *>(src + (r0 + 8) * P.tcb_pitch + c2);
                        mma_k8<PREC>(acc[q][m], a0, a1, bfrag);
                    }
                }
            }
            // scatter the diagonals d = i - j in [0, 2R] to scr[q][d][j]
#pragma unroll
            for (int q = 0; q < SXC; ++q) {
#pragma unroll
                for (int m = 0; m < MT; ++m) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int i = 16 * m + gq + ((e & 2) ? 8 : 0);
                        const int j = 2 * tq + (e & 1);
                        const int d = i - j;
                        if (d >= 0 && d < ND) scr[(q * ND + d) * 8 + j] = acc[q][m][e];
                    }
                }
            }
            __syncwarp();
            const int nq = min(SXC, R - sx0 + 1);
            for (int o = lane; o < nq * ND; o += 32) {
                const int q = o / ND, d = o - q * ND;
                const float4 lo4 = *reinterpret_cast<const float4 *>(scr + (q * ND + d) * 8);
                const float4 hi4 = *reinterpret_cast<const float4 *>(scr + (q * ND + d) * 8 + 4);
                const float sum = ((lo4.x + lo4.y) + (lo4.z + lo4.w)) + ((hi4.x + hi4.y) + (hi4.z + hi4.w));
                // plane index: sy = d - R -> row d; sx = sx0 + q -> column sx0 + q + R
                Ps[(size_t)(b * nsb + sb) * NP + d * ND + (sx0 + q + R)] = sum;
            }
            __syncwarp();
        }
    }
}

// ----------------------------------------------- assembly and sub-pixel --

__device__ __forceinline__ float gauss3f(float cm, float c0, float cp)
{
    float d = 0.f;
    bool ok = false;
    if (cm > 0.f && c0 > 0.f && cp > 0.f) {
        const float lm = logf(cm), l0 = logf(c0), lp = logf(cp);
        const float den = 2.f * lm - 4.f * l0 + 2.f * lp;
        if (den < 0.f) {
            d = (lm - lp) / den;
            ok = true;
        }
    }
    if (!ok) {
        const float den = 2.f * cm - 4.f * c0 + 2.f * cp;
        if (den < 0.f) {
            d = (cm - cp) / den;
            ok = true;
        }
    }
    if (!ok) return 0.f;
    return fminf(fmaxf(d, -1.f), 1.f);
}

struct WinRef {
    int wxi, wyi;       // tile-local window index
    float muA, EA;
    float inv_n, tau;
};

__device__ __forceinline__ float zncc_from(float num, const WinRef &wr, float S1, float S2)
{
    const float Nc = num - wr.muA * S1;
    const float EB = S2 - S1 * S1 * wr.inv_n;
    if (!(wr.EA > wr.tau) || !(EB > wr.tau)) return 0.f;
    return Nc / sqrtf(wr.EA * EB);
}

// numerator of one window at shift (sy, sx) by direct FP32 summation (warp-wide)
static __device__ float direct_num(const PassArgs &a, const TileGeom &g, const float *As, const float *Bs, const WinRef &wr,
                            int sy, int sx)
{
    const PassPlan &P = a.plan;
    const int lane = threadIdx.x & 31, w = a.w, n = w * w;
    const float *abase = As + (wr.wyi * a.s) * P.a_pitch + wr.wxi * a.s;
    const float *bbase = Bs + (wr.wyi * a.s + sy + g.R + 1) * P.b_pitch + P.padl + wr.wxi * a.s + sx;
    float acc = 0.f;
    for (int e = lane; e < n; e += 32) {
        const int y = e / w, x = e - y * w;
        acc = fmaf(abase[y * P.a_pitch + x], bbase[y * P.b_pitch + x], acc);
    }
    return warp_sum(acc);
}

__device__ __forceinline__ float plane_num(const PassArgs &a, const TileGeom &g, const float *Ps, const WinRef &wr,
                                           int q)
{
    const PassPlan &P = a.plan;
    const int G = P.G, kb = a.w / G, RG = P.RGx;
    const int bx0 = (wr.wxi * a.s) / G, by0 = (wr.wyi * a.s) / G;
    float sum = 0.f;
    for (int yy = 0; yy < kb; ++yy)
        for (int xx = 0; xx < kb; ++xx) {
            const float *pb = Ps + (size_t)((by0 + yy) * g.nbx + bx0 + xx) * RG * g.NP + q;
            for (int gi = 0; gi < RG; ++gi) sum += pb[(size_t)gi * g.NP];
        }
    return sum;
}

// Window assembly, argmax, 5-point FP32 stencil, Gaussian fit; one warp per window.
static __device__ void assemble(const PassArgs &a, const TileGeom &g, const float *As, const float *Bs, const float *Vs,
                         const float *Ps, const float *stats, bool tc, int pair)
{
    const PassPlan &P = a.plan;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int R = g.R, ND = g.ND, NP = g.NP;
    const float n = (float)(a.w * a.w);
    const float *pu = (const float *)resolve(a.pred_u, pair);
    const float *pv = (const float *)resolve(a.pred_v, pair);
    float *ou = (float *)resolve(a.out_u, pair);
    float *ov = (float *)resolve(a.out_v, pair);
    int32_t *oi = (int32_t *)resolve(a.out_info, pair);
    const float *V1 = Vs, *V2 = Vs + g.vh * P.h_pitch;
    for (int wi = warp; wi < g.nwin; wi += nwarps) {
        WinRef wr;
        wr.wxi = wi % g.nwx;
        wr.wyi = wi / g.nwx;
        wr.muA = stats[2 * wi];
        wr.EA = stats[2 * wi + 1];
        wr.inv_n = 1.f / n;
        wr.tau = TAU_PER_PIXEL * n;
        const int gi = (g.wy0 + wr.wyi), gj = (g.wx0 + wr.wxi);
        const int k = gi * a.nx + gj;
        const float pu0 = pu ? pu[k] : 0.f, pv0 = pv ? pv[k] : 0.f;
        const int vr0 = wr.wyi * a.s + R + 1, vc0 = wr.wxi * a.s + R + 1;
        auto S1at = [&](int sy, int sx) { return V1[(vr0 + sy) * P.h_pitch + vc0 + sx]; };
        auto S2at = [&](int sy, int sx) { return V2[(vr0 + sy) * P.h_pitch + vc0 + sx]; };
        if (!(wr.EA > wr.tau)) {
            if (lane == 0) {
                ou[k] = pu0;
                ov[k] = pv0;
                oi[k] = 0;
            }
            continue;
        }
        float best = -INFINITY;
        int bidx = 0x7fffffff;
        for (int q = lane; q < NP; q += 32) {
            const int sy = q / ND - R, sx = q % ND - R;
            const float c = zncc_from(plane_num(a, g, Ps, wr, q), wr, S1at(sy, sx), S2at(sy, sx));
            if (c > best || (c == best && q < bidx)) {
                best = c;
                bidx = q;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oq = __shfl_xor_sync(0xffffffffu, bidx, o);
            if (ob > best || (ob == best && oq < bidx)) {
                best = ob;
                bidx = oq;
            }
        }
        const int ky = bidx / ND - R, kx = bidx % ND - R;
        // 5-point stencil in FP32: centre, -x, +x, -y, +y
        float c5[5];
        const int dys[5] = {0, 0, 0, -1, 1}, dxs[5] = {0, -1, 1, 0, 0};
#pragma unroll
        for (int p = 0; p < 5; ++p) {
            const int sy = ky + dys[p], sx = kx + dxs[p];
            float num;
            if (!tc && sy >= -R && sy <= R && sx >= -R && sx <= R)
                num = plane_num(a, g, Ps, wr, (sy + R) * ND + (sx + R));
            else
                num = direct_num(a, g, As, Bs, wr, sy, sx);
            c5[p] = zncc_from(num, wr, S1at(sy, sx), S2at(sy, sx));
        }
        if (lane == 0) {
            const float dx = gauss3f(c5[1], c5[0], c5[2]);
            const float dy = gauss3f(c5[3], c5[0], c5[4]);
            ou[k] = pu0 + (float)kx + dx;
            ov[k] = pv0 + (float)ky + dy;
            oi[k] = 1 | ((int)(uint8_t)(int8_t)ky << 8) | ((int)(uint8_t)(int8_t)kx << 16);
        }
    }
}

// ------------------------------------------------------------- the kernel --

template <int RC, int PREC>
__global__ void __launch_bounds__(PASS_THREADS) pass_kernel(const PassArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const PassPlan &P = a.plan;
    TileGeom g;
    g.R = RC >= 0 ? RC : a.R;
    g.ND = 2 * g.R + 1;
    g.NP = g.ND * g.ND;
    const int pair = blockIdx.z;
    const int s = a.s, w = a.w;
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
    g.nbx = g.aw / P.G;
    g.nby = g.ah / P.G;
    g.nb = g.nbx * g.nby;

    float *nodes = reinterpret_cast<float *>(smem + P.off_nodes);
    int *ti = reinterpret_cast<int *>(smem + P.off_tabs);
    float *tf = reinterpret_cast<float *>(ti + g.BC + g.BR);
    float *As = reinterpret_cast<float *>(smem + P.off_a);
    float *Bs = reinterpret_cast<float *>(smem + P.off_b);
    float *Hs = reinterpret_cast<float *>(smem + P.off_h);
    float *Vs = reinterpret_cast<float *>(smem + P.off_v);
    float *Ps = reinterpret_cast<float *>(smem + P.off_p);
    float *stats = reinterpret_cast<float *>(smem + P.off_stats);
    float *red = reinterpret_cast<float *>(smem + P.off_red);

    const unsigned char *imgA = (const unsigned char *)resolve(a.img_a, pair);
    const unsigned char *imgB = (const unsigned char *)resolve(a.img_b, pair);
    const float *pu = (const float *)resolve(a.pred_u, pair);
    const float *pv = (const float *)resolve(a.pred_v, pair);
    const bool has_pred = (pu != nullptr) && (pv != nullptr);
    const int tid = threadIdx.x;
    const float c0 = 0.5f * (float)(w - 1);

    // phase 0: grid weights of every region column/row and the predictor nodes
    {
        int ilo, ihi, jlo, jhi;
        float t;
        axis_w(g.ax0 - (g.R + 1), a.nx, c0, s, ilo, t);
        axis_w(g.ax0 - (g.R + 1) + g.BC - 1, a.nx, c0, s, ihi, t);
        axis_w(g.ay0 - (g.R + 1), a.ny, c0, s, jlo, t);
        axis_w(g.ay0 - (g.R + 1) + g.BR - 1, a.ny, c0, s, jhi, t);
        ihi = min(ihi + 1, a.nx - 1);
        jhi = min(jhi + 1, a.ny - 1);
        g.i_lo = ilo;
        g.j_lo = jlo;
        g.nodes_w = ihi - ilo + 1;
        const int nh = jhi - jlo + 1;
        for (int bx = tid; bx < g.BC; bx += blockDim.x) {
            int i0;
            float tt;
            axis_w(g.ax0 - (g.R + 1) + bx, a.nx, c0, s, i0, tt);
            ti[bx] = i0 - ilo;
            tf[bx] = tt;
        }
        for (int by = tid; by < g.BR; by += blockDim.x) {
            int j0;
            float tt;
            axis_w(g.ay0 - (g.R + 1) + by, a.ny, c0, s, j0, tt);
            ti[g.BC + by] = j0 - jlo;
            tf[g.BC + by] = tt;
        }
        if (has_pred) {
            for (int e = tid; e < g.nodes_w * nh; e += blockDim.x) {
                const int jj = e / g.nodes_w, ii = e - jj * g.nodes_w;
                const int gk = (jlo + jj) * a.nx + ilo + ii;
                nodes[e] = pu[gk];
                nodes[P.node_cap + e] = pv[gk];
            }
        }
    }
    __syncthreads();

    // phases 1-2: A region, tile mean, deformed B' region
    float muT;
    if (a.fmt == PIX_U8)
        load_and_deform<uint8_t>(a, g, imgA, imgB, has_pred, nodes, ti, tf, As, Bs, red, muT);
    else if (a.fmt == PIX_U16)
        load_and_deform<uint16_t>(a, g, imgA, imgB, has_pred, nodes, ti, tf, As, Bs, red, muT);
    else
        load_and_deform<float>(a, g, imgA, imgB, has_pred, nodes, ti, tf, As, Bs, red, muT);
    __syncthreads();

    // phase 3-4: box sums of B' for every window and shift; A window statistics
    window_stats(a, g, As, stats);
    box_sums(a, g, Bs, Hs, Vs);
    __syncthreads();

    // phase 5: block partial planes (aliases the dead H region)
    if (PREC == PREC_FP32) {
        if (RC >= 0)
            block_planes_fp32<(RC >= 0 ? RC : 0)>(a, g, As, Bs, Ps);
        else
            block_planes_fp32_generic(a, g, As, Bs, Ps);
    } else {
        uint16_t *TA = reinterpret_cast<uint16_t *>(smem + P.off_tca);
        uint16_t *TB = reinterpret_cast<uint16_t *>(smem + P.off_tcb);
        float *scr = reinterpret_cast<float *>(smem + P.off_scr);
        tc_convert<PREC>(a, g, As, Bs, TA, TB);
        __syncthreads();
        block_planes_tc<(RC >= 0 ? RC : 0), PREC>(a, g, TA, TB, scr, Ps);
    }
    __syncthreads();

    // phase 6: per-window plane, argmax, refit, Gaussian fit, outputs
    assemble(a, g, As, Bs, Vs, Ps, stats, PREC != PREC_FP32, pair);
}

}  // namespace rpiv
