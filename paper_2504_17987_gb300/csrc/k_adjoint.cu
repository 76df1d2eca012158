// Adjoint of the zero-shift correlation score with respect to the
// displacement grid (differentiation of the deformation step of paper Sec. 2).
//
//   S = sum_w C_w(0),  C_w = sum a~ b~ / sqrt(E_A E_B),  B'(x) = B(x + d(x)),
//   d(x) = sum_k phi_k(x) d_k  (bilinear weights, border value outside the hull)
//   dC_w/dB'(x) = a~(x)/sqrt(E_A E_B) - C_w b~(x)/E_B
//   dS/dd_k = sum_x phi_k(x) grad B(x + d(x)) sum_{w containing x} dC_w/dB'(x)
//
// Three deterministic kernels, no floating-point atomics; deformed windows are
// recomputed from the images instead of being stored:
//   1. one warp per window: mean/energy of A and B', C_w       -> win_stats
//   2. one thread per pixel: grad B at the deformed position times the sum
//      over its windows of dC_w/dB'                           -> pix_g
//   3. one thread per grid node: weighted sum of pix_g over the node's
//      bilinear support                                          -> grad
//   plus a single-block fixed-order sum of C_w for the score.
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
    if (gx) {
        *gx = (1.f - ty) * (b10 - b00) + ty * (b11 - b01);
        *gy = (1.f - tx) * (b01 - b00) + tx * (b11 - b10);
    }
    const float top = b00 + tx * (b10 - b00), bot = b01 + tx * (b11 - b01);
    return top + ty * (bot - top);
}

template <typename T>
__global__ void adj_win_kernel(const AdjArgs a)
{
    const int lane = threadIdx.x & 31;
    const int win = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (win >= a.nx * a.ny) return;
    const unsigned char *A = (const unsigned char *)resolve(a.img_a, 0);
    const unsigned char *B = (const unsigned char *)resolve(a.img_b, 0);
    const int j = win / a.nx, i = win - j * a.nx;
    const int x0 = i * a.s, y0 = j * a.s, w = a.w, n = w * w;
    float sa = 0.f, sb = 0.f;
    for (int e = lane; e < n; e += 32) {
        const int x = x0 + e % w, y = y0 + e / w;
        float du, dv;
        field(a, x, y, du, dv);
        sa += px<T>(A, a.pitch, x, y);
        sb += deformed<T>(a, B, x, y, du, dv, nullptr, nullptr);
    }
    const float ma = wsum(sa) / (float)n, mb = wsum(sb) / (float)n;
    float ea = 0.f, eb = 0.f, num = 0.f;
    for (int e = lane; e < n; e += 32) {
        const int x = x0 + e % w, y = y0 + e / w;
        float du, dv;
        field(a, x, y, du, dv);
        const float at = px<T>(A, a.pitch, x, y) - ma;
        const float bt = deformed<T>(a, B, x, y, du, dv, nullptr, nullptr) - mb;
        ea = fmaf(at, at, ea);
        eb = fmaf(bt, bt, eb);
        num = fmaf(at, bt, num);
    }
    ea = wsum(ea);
    eb = wsum(eb);
    num = wsum(num);
    if (lane == 0) {
        float *st = a.win_stats + 8 * win;
        const float tau = kTauPerPixel * (float)n;
        const bool ok = ea > tau && eb > tau;
        const float rs = ok ? 1.f / sqrtf(ea * eb) : 0.f;
        const float C = ok ? num * rs : 0.f;
        st[0] = ma;
        st[1] = mb;
        st[2] = rs;
        st[3] = ok ? C / eb : 0.f;
        st[4] = C;
    }
}

template <typename T>
__global__ void adj_pix_kernel(const AdjArgs a)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= a.W || y >= a.H) return;
    const unsigned char *A = (const unsigned char *)resolve(a.img_a, 0);
    const unsigned char *B = (const unsigned char *)resolve(a.img_b, 0);
    const int w = a.w, s = a.s;
    const int ilo = max(0, (x - w + s) / s), ihi = min(a.nx - 1, x / s);
    const int jlo = max(0, (y - w + s) / s), jhi = min(a.ny - 1, y / s);
    float g = 0.f;
    float gx = 0.f, gy = 0.f;
    if (ilo <= ihi && jlo <= jhi) {
        float du, dv;
        field(a, x, y, du, dv);
        const float b = deformed<T>(a, B, x, y, du, dv, &gx, &gy);
        const float av = px<T>(A, a.pitch, x, y);
        for (int j = jlo; j <= jhi; ++j)
            for (int i = ilo; i <= ihi; ++i) {
                const float *st = a.win_stats + 8 * (j * a.nx + i);
                g += (av - st[0]) * st[2] - st[3] * (b - st[1]);
            }
    }
    float *o = a.pix_g + 2 * ((long long)y * a.W + x);
    o[0] = g * gx;
    o[1] = g * gy;
}

__global__ void adj_node_kernel(const AdjArgs a)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.nx * a.ny) return;
    const int j = k / a.nx, i = k - j * a.nx;
    const float c0 = 0.5f * (float)(a.w - 1);
    // support along each axis: pixels strictly between the neighbouring nodes,
    // extended to the image border for the first and last node
    const int xl = (i == 0) ? 0 : max(0, (int)floorf(c0 + (float)((i - 1) * a.s)) + 1);
    const int xh = (i == a.nx - 1) ? a.W - 1 : min(a.W - 1, (int)ceilf(c0 + (float)((i + 1) * a.s)) - 1);
    const int yl = (j == 0) ? 0 : max(0, (int)floorf(c0 + (float)((j - 1) * a.s)) + 1);
    const int yh = (j == a.ny - 1) ? a.H - 1 : min(a.H - 1, (int)ceilf(c0 + (float)((j + 1) * a.s)) - 1);
    float gu = 0.f, gv = 0.f;
    for (int y = yl; y <= yh; ++y) {
        int j0, j1;
        float ty;
        axis_wt(y, a.ny, c0, a.s, j0, j1, ty);
        const float wy = (j0 == j ? 1.f - ty : 0.f) + (j1 == j && j1 != j0 ? ty : 0.f);
        if (wy == 0.f) continue;
        for (int x = xl; x <= xh; ++x) {
            int i0, i1;
            float tx;
            axis_wt(x, a.nx, c0, a.s, i0, i1, tx);
            const float wx = (i0 == i ? 1.f - tx : 0.f) + (i1 == i && i1 != i0 ? tx : 0.f);
            if (wx == 0.f) continue;
            const float *p = a.pix_g + 2 * ((long long)y * a.W + x);
            gu = fmaf(wx * wy, p[0], gu);
            gv = fmaf(wx * wy, p[1], gv);
        }
    }
    if (a.grad_u) a.grad_u[k] = a.grad_scale * gu;
    if (a.grad_v) a.grad_v[k] = a.grad_scale * gv;
}

__global__ void adj_score_kernel(const AdjArgs a)
{
    __shared__ float part[32];
    const int n = a.nx * a.ny;
    float s = 0.f;
    for (int k = threadIdx.x; k < n; k += blockDim.x) s += a.win_stats[8 * k + 4];
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
    const int nwin = a.nx * a.ny;
    adj_win_kernel<T><<<(nwin * 32 + 255) / 256, 256, 0, st>>>(a);
    if (a.score_out) adj_score_kernel<<<1, 1024, 0, st>>>(a);
    if (a.grad_u || a.grad_v) {
        adj_pix_kernel<T><<<dim3((a.W + 255) / 256, a.H), 256, 0, st>>>(a);
        adj_node_kernel<<<(nwin + 127) / 128, 128, 0, st>>>(a);
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

size_t adjoint_workspace_bytes(int W, int H, int nx, int ny)
{
    return sizeof(float) * (8ull * nx * ny + 2ull * W * H) + 256;
}

cudaError_t launch_adjoint(const AdjArgs &a, cudaStream_t st)
{
    if (a.fmt == PIX_U8) return run<uint8_t>(a, st);
    if (a.fmt == PIX_U16) return run<uint16_t>(a, st);
    return run<float>(a, st);
}

}  // namespace rpiv
