// Adjoint of the zero-shift correlation score with respect to the
// displacement grid (differentiation of the deformation step of paper Sec. 2).
//
//   S = sum_w C_w(0),  C_w = sum a~ b~ / sqrt(E_A E_B),  B'(x) = B(x + d(x)),
//   d(x) = sum_k phi_k(x) d_k  (bilinear weights, border value outside the hull)
//   dC_w/dB'(x) = a~(x)/sqrt(E_A E_B) - C_w b~(x)/E_B
//   dS/dd_k = sum_x phi_k(x) grad B(x + d(x)) sum_{w containing x} dC_w/dB'(x)
//
// Deterministic kernels, no floating-point atomics:
//   1. one thread per pixel: d(x), B'(x) and the in-cell gradient of B at the
//      deformed position                                        -> bp, gxy
//   2. one warp per G x G block (G = gcd(w, s), so that every window is a
//      union of blocks): means of A and B' and their centred second moments
//                                                                 -> blk
//   3. one thread per window: the window's moments combined from its blocks
//      (pairwise update of centred moments), C_w             -> win_stats
//   4. one thread per pixel: grad B times the sum over its windows of
//      dC_w/dB'                                                   -> pix_g
//   5. the node sums, separable in the bilinear weights: one thread per
//      (image row, node column) sums its row of the node's support along x,
//      then one thread per node sums those along y             -> grad
//   plus a single-block fixed-order sum of C_w for the score.
// Each pixel's deformation is evaluated once (not once per overlapping
// window), and the window sums reuse each block across the windows that
// contain it.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "rpiv_internal.h"

namespace rpiv {

namespace {

constexpr float kTauPerPixel = 1e-6f;

__device__ __forceinline__ float wsum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void axis_wt(int pos, int n, float c0, int s, int &i0, int &i1, float &t)
{
    if (n <= 1) {
        i0 = i1 = 0;
        t = 0.f;
        return;
    }
    float f = ((float)pos - c0) / (float)s;
    f = fminf(fmaxf(f, 0.f), (float)(n - 1));
    int ia = (int)floorf(f);
    if (ia > n - 2) ia = n - 2;
    i0 = ia;
    i1 = ia + 1;
    t = f - (float)ia;
}

// bilinear weight of node i at a pixel position along one axis
__device__ __forceinline__ float node_wt(int pos, int i, int n, float c0, int s)
{
    int i0, i1;
    float t;
    axis_wt(pos, n, c0, s, i0, i1, t);
    return (i0 == i ? 1.f - t : 0.f) + (i1 == i && i1 != i0 ? t : 0.f);
}

__device__ __forceinline__ void field(const AdjArgs &a, int x, int y, float &du, float &dv)
{
    const float c0 = 0.5f * (float)(a.w - 1);
    int i0, i1, j0, j1;
    float tx, ty;
    axis_wt(x, a.nx, c0, a.s, i0, i1, tx);
    axis_wt(y, a.ny, c0, a.s, j0, j1, ty);
    const float *u = a.u, *v = a.v;
    float t0 = u[j0 * a.nx + i0] + tx * (u[j0 * a.nx + i1] - u[j0 * a.nx + i0]);
    float t1 = u[j1 * a.nx + i0] + tx * (u[j1 * a.nx + i1] - u[j1 * a.nx + i0]);
    du = t0 + ty * (t1 - t0);
    t0 = v[j0 * a.nx + i0] + tx * (v[j0 * a.nx + i1] - v[j0 * a.nx + i0]);
    t1 = v[j1 * a.nx + i0] + tx * (v[j1 * a.nx + i1] - v[j1 * a.nx + i0]);
    dv = t0 + ty * (t1 - t0);
}

template <typename T>
__device__ __forceinline__ float px(const unsigned char *img, long long pitch, int x, int y)
{
    return (float)__ldg(reinterpret_cast<const T *>(img + (long long)y * pitch) + x);
}

// B' = bilinear(B) at (x + du, y + dv), clamp-to-edge, and its in-cell gradient.
template <typename T>
__device__ __forceinline__ float deformed(const AdjArgs &a, const unsigned char *B, int x, int y, float du, float dv,
                                          float *gx, float *gy)
{
    du = isfinite(du) ? fminf(fmaxf(du, -1048576.f), 1048576.f) : 0.f;
    dv = isfinite(dv) ? fminf(fmaxf(dv, -1048576.f), 1048576.f) : 0.f;
    const float fx = floorf(du), fy = floorf(dv);
    const float tx = du - fx, ty = dv - fy;
    const int ix = x + (int)fx, iy = y + (int)fy;
    const int x0 = min(max(ix, 0), a.W - 1), x1 = min(max(ix + 1, 0), a.W - 1);
    const int y0 = min(max(iy, 0), a.H - 1), y1 = min(max(iy + 1, 0), a.H - 1);
    const float b00 = px<T>(B, a.pitch, x0, y0), b10 = px<T>(B, a.pitch, x1, y0);
    const float b01 = px<T>(B, a.pitch, x0, y1), b11 = px<T>(B, a.pitch, x1, y1);
    *gx = (1.f - ty) * (b10 - b00) + ty * (b11 - b01);
    *gy = (1.f - tx) * (b01 - b00) + tx * (b11 - b10);
    const float top = b00 + tx * (b10 - b00), bot = b01 + tx * (b11 - b01);
    return top + ty * (bot - top);
}

// Workspace carve-up (floats, each part 256-byte aligned).
struct AdjWs {
    float *win_stats;  // 8 per window: mean A, mean B', 1/sqrt(E_A E_B), C/E_B, C
    float *blk;        // 8 per block: mean A, mean B', centred A.A, B'.B', A.B'
    float *bp;         // B' per pixel
    float2 *gxy;       // grad B at the deformed position per pixel
    float2 *pix_g;     // dS/dB' times grad B per pixel
    float2 *rows;      // per (image row, node column): the node's support summed along x
};

__host__ __device__ inline size_t up64(size_t n) { return (n + 63) & ~(size_t)63; }

__host__ __device__ inline int gcd_i(int a, int b)
{
    while (b) {
        const int t = a % b;
        a = b;
        b = t;
    }
    return a;
}

struct BlockGrid {
    int G, nbx, nby;  // block size; blocks across the windows' union
};

__host__ __device__ inline BlockGrid block_grid(int w, int s, int nx, int ny)
{
    BlockGrid b;
    b.G = gcd_i(w, s);
    b.nbx = ((nx - 1) * s + w) / b.G;
    b.nby = ((ny - 1) * s + w) / b.G;
    return b;
}

__host__ __device__ inline size_t ws_floats(int W, int H, int w, int s, int nx, int ny, AdjWs *out, float *base)
{
    const BlockGrid bg = block_grid(w, s, nx, ny);
    size_t off = 0;
    const size_t o_win = off;
    off += up64(8ull * nx * ny);
    const size_t o_blk = off;
    off += up64(8ull * bg.nbx * bg.nby);
    const size_t o_bp = off;
    off += up64((size_t)W * H);
    const size_t o_gxy = off;
    off += up64(2ull * W * H);
    const size_t o_pix = off;
    off += up64(2ull * W * H);
    const size_t o_rows = off;
    off += up64(2ull * H * nx);
    if (out) {
        out->win_stats = base + o_win;
        out->blk = base + o_blk;
        out->bp = base + o_bp;
        out->gxy = reinterpret_cast<float2 *>(base + o_gxy);
        out->pix_g = reinterpret_cast<float2 *>(base + o_pix);
        out->rows = reinterpret_cast<float2 *>(base + o_rows);
    }
    return off;
}

// 1: the deformed frame and the gradient of B under it, once per pixel
template <typename T>
__global__ void adj_deform_kernel(const AdjArgs a, const AdjWs ws)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= a.W) return;
    const unsigned char *B = (const unsigned char *)resolve(a.img_b, 0);
    float du, dv, gx, gy;
    field(a, x, y, du, dv);
    const long long p = (long long)y * a.W + x;
    ws.bp[p] = deformed<T>(a, B, x, y, du, dv, &gx, &gy);
    ws.gxy[p] = make_float2(gx, gy);
}

// 2: per G x G block, by one warp: means, then centred second moments
template <typename T>
__global__ void adj_block_kernel(const AdjArgs a, const AdjWs ws, const BlockGrid bg)
{
    const int lane = threadIdx.x & 31;
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= bg.nbx * bg.nby) return;
    const unsigned char *A = (const unsigned char *)resolve(a.img_a, 0);
    const int by = b / bg.nbx, bx = b - by * bg.nbx;
    const int G = bg.G, n = G * G, x0 = bx * G, y0 = by * G;
    float sa = 0.f, sb = 0.f;
    for (int e = lane; e < n; e += 32) {
        const int x = x0 + e % G, y = y0 + e / G;
        sa += px<T>(A, a.pitch, x, y);
        sb += ws.bp[(long long)y * a.W + x];
    }
    const float ma = wsum(sa) / (float)n, mb = wsum(sb) / (float)n;
    float caa = 0.f, cbb = 0.f, cab = 0.f;
    for (int e = lane; e < n; e += 32) {
        const int x = x0 + e % G, y = y0 + e / G;
        const float at = px<T>(A, a.pitch, x, y) - ma;
        const float bt = ws.bp[(long long)y * a.W + x] - mb;
        caa = fmaf(at, at, caa);
        cbb = fmaf(bt, bt, cbb);
        cab = fmaf(at, bt, cab);
    }
    caa = wsum(caa);
    cbb = wsum(cbb);
    cab = wsum(cab);
    if (lane == 0) {
        float *o = ws.blk + 8ll * b;
        o[0] = ma;
        o[1] = mb;
        o[2] = caa;
        o[3] = cbb;
        o[4] = cab;
    }
}

// 3: per window, its (w/G)^2 blocks combined: equal-size parts, so the mean
// is the mean of the block means, and each centred moment gains
// G^2 (mean_k - mean)(mean'_k - mean') per block
__global__ void adj_win_kernel(const AdjArgs a, const AdjWs ws, const BlockGrid bg)
{
    const int win = blockIdx.x * blockDim.x + threadIdx.x;
    if (win >= a.nx * a.ny) return;
    const int j = win / a.nx, i = win - j * a.nx;
    const int G = bg.G, kb = a.w / G, bx0 = i * a.s / G, by0 = j * a.s / G;
    float ma = 0.f, mb = 0.f;
    for (int q = 0; q < kb; ++q)
        for (int p = 0; p < kb; ++p) {
            const float *o = ws.blk + 8ll * ((by0 + q) * bg.nbx + bx0 + p);
            ma += o[0];
            mb += o[1];
        }
    ma /= (float)(kb * kb);
    mb /= (float)(kb * kb);
    const float nb = (float)(G * G);
    float ea = 0.f, eb = 0.f, num = 0.f;
    for (int q = 0; q < kb; ++q)
        for (int p = 0; p < kb; ++p) {
            const float *o = ws.blk + 8ll * ((by0 + q) * bg.nbx + bx0 + p);
            const float da = o[0] - ma, db = o[1] - mb;
            ea += fmaf(nb * da, da, o[2]);
            eb += fmaf(nb * db, db, o[3]);
            num += fmaf(nb * da, db, o[4]);
        }
    float *st = ws.win_stats + 8ll * win;
    const float tau = kTauPerPixel * (float)(a.w * a.w);
    const bool ok = ea > tau && eb > tau;
    const float rs = ok ? 1.f / sqrtf(ea * eb) : 0.f;
    const float C = ok ? num * rs : 0.f;
    st[0] = ma;
    st[1] = mb;
    st[2] = rs;
    st[3] = ok ? C / eb : 0.f;
    st[4] = C;
}

// 4: per pixel, grad B times the sum of dC_w/dB' over the windows that hold it
template <typename T>
__global__ void adj_pix_kernel(const AdjArgs a, const AdjWs ws)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= a.W) return;
    const unsigned char *A = (const unsigned char *)resolve(a.img_a, 0);
    const int w = a.w, s = a.s;
    const int ilo = max(0, (x - w + s) / s), ihi = min(a.nx - 1, x / s);
    const int jlo = max(0, (y - w + s) / s), jhi = min(a.ny - 1, y / s);
    const long long p = (long long)y * a.W + x;
    float g = 0.f;
    if (ilo <= ihi && jlo <= jhi) {
        const float b = ws.bp[p];
        const float av = px<T>(A, a.pitch, x, y);
        for (int j = jlo; j <= jhi; ++j)
            for (int i = ilo; i <= ihi; ++i) {
                const float *st = ws.win_stats + 8 * (j * a.nx + i);
                g += (av - st[0]) * st[2] - st[3] * (b - st[1]);
            }
    }
    const float2 gr = ws.gxy[p];
    ws.pix_g[p] = make_float2(g * gr.x, g * gr.y);
}

// support of node i along an axis of n nodes: the pixels strictly between its
// neighbours, extended to the image border for the first and last node
__device__ __forceinline__ void support(int i, int n, float c0, int s, int len, int &lo, int &hi)
{
    lo = (i == 0) ? 0 : max(0, (int)floorf(c0 + (float)((i - 1) * s)) + 1);
    hi = (i == n - 1) ? len - 1 : min(len - 1, (int)ceilf(c0 + (float)((i + 1) * s)) - 1);
}

// 5a: per (image row y, node column i): sum over x of the x weight times pix_g
__global__ void adj_rows_kernel(const AdjArgs a, const AdjWs ws)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (i >= a.nx) return;
    const float c0 = 0.5f * (float)(a.w - 1);
    int xl, xh;
    support(i, a.nx, c0, a.s, a.W, xl, xh);
    const float2 *row = ws.pix_g + (long long)y * a.W;
    float gu = 0.f, gv = 0.f;
    for (int x = xl; x <= xh; ++x) {
        const float wx = node_wt(x, i, a.nx, c0, a.s);
        if (wx == 0.f) continue;
        gu = fmaf(wx, row[x].x, gu);
        gv = fmaf(wx, row[x].y, gv);
    }
    ws.rows[(long long)y * a.nx + i] = make_float2(gu, gv);
}

// 5b: per node: sum over y of the y weight times the row sums
__global__ void adj_node_kernel(const AdjArgs a, const AdjWs ws)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.nx * a.ny) return;
    const int j = k / a.nx, i = k - j * a.nx;
    const float c0 = 0.5f * (float)(a.w - 1);
    int yl, yh;
    support(j, a.ny, c0, a.s, a.H, yl, yh);
    float gu = 0.f, gv = 0.f;
    for (int y = yl; y <= yh; ++y) {
        const float wy = node_wt(y, j, a.ny, c0, a.s);
        if (wy == 0.f) continue;
        const float2 r = ws.rows[(long long)y * a.nx + i];
        gu = fmaf(wy, r.x, gu);
        gv = fmaf(wy, r.y, gv);
    }
    if (a.grad_u) a.grad_u[k] = a.grad_scale * gu;
    if (a.grad_v) a.grad_v[k] = a.grad_scale * gv;
}

__global__ void adj_score_kernel(const AdjArgs a, const AdjWs ws)
{
    __shared__ float part[32];
    const int n = a.nx * a.ny;
    float s = 0.f;
    for (int k = threadIdx.x; k < n; k += blockDim.x) s += ws.win_stats[8 * k + 4];
    s = wsum(s);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.f;
        v = wsum(v);
        if (threadIdx.x == 0 && a.score_out) *a.score_out = v;
    }
}

template <typename T>
cudaError_t run(const AdjArgs &a, cudaStream_t st)
{
    AdjWs ws;
    ws_floats(a.W, a.H, a.w, a.s, a.nx, a.ny, &ws, reinterpret_cast<float *>(a.ws));
    const BlockGrid bg = block_grid(a.w, a.s, a.nx, a.ny);
    const int nwin = a.nx * a.ny, nblk = bg.nbx * bg.nby;
    adj_deform_kernel<T><<<dim3((a.W + 255) / 256, a.H), 256, 0, st>>>(a, ws);
    adj_block_kernel<T><<<(nblk * 32 + 255) / 256, 256, 0, st>>>(a, ws, bg);
    adj_win_kernel<<<(nwin + 127) / 128, 128, 0, st>>>(a, ws, bg);
    if (a.score_out) adj_score_kernel<<<1, 1024, 0, st>>>(a, ws);
    if (a.grad_u || a.grad_v) {
        adj_pix_kernel<T><<<dim3((a.W + 255) / 256, a.H), 256, 0, st>>>(a, ws);
        adj_rows_kernel<<<dim3((a.nx + 127) / 128, a.H), 128, 0, st>>>(a, ws);
        adj_node_kernel<<<(nwin + 127) / 128, 128, 0, st>>>(a, ws);
    }
    return cudaGetLastError();
}

}  // namespace

// ------------------------------------------------ refinement step helpers --

namespace {

// cu = u + eta gu, cv = v + eta gv (FP32, one element per thread)
__global__ void refine_axpy_kernel(const float *u, const float *v, const float *gu, const float *gv, float eta,
                                   float *cu, float *cv, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    cu[i] = fmaf(eta, gu[i], u[i]);
    cv[i] = fmaf(eta, gv[i], v[i]);
}

// out = max(|a|, |b|) over n elements: one CTA, fixed order (max is exact)
__global__ void refine_absmax_kernel(const float *a, const float *b, int n, float *out)
{
    __shared__ float part[32];
    float m = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmaxf(m, fmaxf(fabsf(a[i]), fabsf(b[i])));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) *out = m;
    }
}

}  // namespace

cudaError_t launch_refine_axpy(const float *u, const float *v, const float *gu, const float *gv, float eta, float *cu,
                               float *cv, int n, cudaStream_t st)
{
    refine_axpy_kernel<<<(n + 255) / 256, 256, 0, st>>>(u, v, gu, gv, eta, cu, cv, n);
    return cudaGetLastError();
}

cudaError_t launch_refine_absmax(const float *a, const float *b, int n, float *out, cudaStream_t st)
{
    refine_absmax_kernel<<<1, 1024, 0, st>>>(a, b, n, out);
    return cudaGetLastError();
}

size_t adjoint_workspace_bytes(int W, int H, int w, int s, int nx, int ny)
{
    return sizeof(float) * ws_floats(W, H, w, s, nx, ny, nullptr, nullptr) + 256;
}

cudaError_t launch_adjoint(const AdjArgs &a, cudaStream_t st)
{
    if (a.fmt == PIX_U8) return run<uint8_t>(a, st);
    if (a.fmt == PIX_U16) return run<uint16_t>(a, st);
    return run<float>(a, st);
}

}  // namespace rpiv
