// Per-node kernels of the vector grid and the image pyramid:
//   - universal outlier detection with median replacement (paper Sec. 2,
//     Westerweel & Scarano 2005; threshold 2 and 0.1 px regulariser, Sec. 3.1)
//   - grid-to-grid bilinear interpolation (pass-to-pass predictor, pyramid)
//   - vorticity omega = dv/dx - du/dy (paper Sec. 1-2, displayed field)
//   - 2x2 box downsampling of the image pyramid (coarse-to-fine predictor)
#include <algorithm>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "rpiv_internal.h"

namespace rpiv {

// ------------------------------------------------------------------ UOD --

constexpr int UOD_TILE = 16;
constexpr int UOD_IN = UOD_TILE + 4;    // values with a 2-node halo
constexpr int UOD_FLAG = UOD_TILE + 2;  // flags with a 1-node halo

__device__ __forceinline__ void cswap(float &a, float &b)
{
    const float lo = fminf(a, b), hi = fmaxf(a, b);
    a = lo;
    b = hi;
}

// Sorts 8 values ascending (Batcher's odd-even merge network, 19 exchanges).
__device__ __forceinline__ void sort8(float (&v)[8])
{
    cswap(v[0], v[1]); cswap(v[2], v[3]); cswap(v[4], v[5]); cswap(v[6], v[7]);
    cswap(v[0], v[2]); cswap(v[1], v[3]); cswap(v[4], v[6]); cswap(v[5], v[7]);
    cswap(v[1], v[2]); cswap(v[5], v[6]);
    cswap(v[0], v[4]); cswap(v[1], v[5]); cswap(v[2], v[6]); cswap(v[3], v[7]);
    cswap(v[2], v[4]); cswap(v[3], v[5]);
    cswap(v[1], v[2]); cswap(v[3], v[4]); cswap(v[5], v[6]);
}

// Median of the first c entries (c in 1..8) of v once sorted; the rest must
// be +inf.  v is left sorted.
__device__ __forceinline__ float median_sorted(float (&v)[8], int c)
{
    sort8(v);
    if (c == 8) return 0.5f * (v[3] + v[4]);  // every neighbour present: the usual case
    float m = v[0];
#pragma unroll
    for (int q = 1; q < 8; ++q)
        if (q == c / 2) m = v[q];
    if ((c & 1) == 0) {
        float lo = v[0];
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (q == c / 2 - 1) lo = v[q];
        m = 0.5f * (lo + m);
    }
    return m;
}

__global__ void __launch_bounds__(256) uod_kernel(const UodArgs a)
{
    __shared__ float su[UOD_IN][UOD_IN], sv[UOD_IN][UOD_IN];
    __shared__ unsigned char sok[UOD_IN][UOD_IN];   // 1 if the node exists
    __shared__ unsigned char sbad[UOD_FLAG][UOD_FLAG];
    const int pair = blockIdx.z;
    const float *u = (const float *)resolve(a.u, pair);
    const float *v = (const float *)resolve(a.v, pair);
    const int32_t *info = (const int32_t *)resolve(a.info, pair);
    float *uo = (float *)resolve(a.u_out, pair);
    float *vo = (float *)resolve(a.v_out, pair);
    uint8_t *mask = (uint8_t *)resolve(a.mask, pair);
    const int i0 = blockIdx.x * UOD_TILE - 2, j0 = blockIdx.y * UOD_TILE - 2;
    const int tid = threadIdx.x;
    for (int e = tid; e < UOD_IN * UOD_IN; e += blockDim.x) {
        const int jj = e / UOD_IN, ii = e % UOD_IN;
        const int i = i0 + ii, j = j0 + jj;
        const bool ok = i >= 0 && j >= 0 && i < a.nx && j < a.ny;
        su[jj][ii] = ok ? u[j * a.nx + i] : 0.f;
        sv[jj][ii] = ok ? v[j * a.nx + i] : 0.f;
        sok[jj][ii] = ok ? 1 : 0;
    }
    __syncthreads();
    // detection on the tile plus a 1-node halo
    for (int e = tid; e < UOD_FLAG * UOD_FLAG; e += blockDim.x) {
        const int jj = e / UOD_FLAG + 1, ii = e % UOD_FLAG + 1;
        const int i = i0 + ii, j = j0 + jj;
        unsigned char bad = 0;
        if (sok[jj][ii]) {
            if (info && !(info[j * a.nx + i] & 1)) bad = 1;
            // the neighbours in a fixed order, +inf where a node is missing:
            // sorting puts the c present values first, in the same order as
            // any packing of them would
            float nu[8], nv[8];
            int c = 0, q = 0;
#pragma unroll
            for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
                for (int di = -1; di <= 1; ++di) {
                    if (di == 0 && dj == 0) continue;
                    const bool ok = sok[jj + dj][ii + di];
                    nu[q] = ok ? su[jj + dj][ii + di] : INFINITY;
                    nv[q] = ok ? sv[jj + dj][ii + di] : INFINITY;
                    c += ok ? 1 : 0;
                    ++q;
                }
            if (c > 0) {
                // nu, nv sorted in place: the residuals of their first c entries
                const float um = median_sorted(nu, c);
                const float vm = median_sorted(nv, c);
#pragma unroll
                for (int q2 = 0; q2 < 8; ++q2) {
                    nu[q2] = q2 < c ? fabsf(nu[q2] - um) : INFINITY;
                    nv[q2] = q2 < c ? fabsf(nv[q2] - vm) : INFINITY;
                }
                const float rmu = median_sorted(nu, c);
                const float rmv = median_sorted(nv, c);
                const float r0u = fabsf(su[jj][ii] - um) / (rmu + a.eps);
                const float r0v = fabsf(sv[jj][ii] - vm) / (rmv + a.eps);
                if (r0u > a.thr || r0v > a.thr) bad = 1;
                // a non-finite value is always an outlier
                if (!isfinite(su[jj][ii]) || !isfinite(sv[jj][ii])) bad = 1;
            }
        }
        sbad[jj - 1][ii - 1] = bad;
    }
    __syncthreads();
    // replacement on the tile
    {
        const int ii = tid % UOD_TILE + 2, jj = tid / UOD_TILE + 2;
        const int i = i0 + ii, j = j0 + jj;
        if (tid < UOD_TILE * UOD_TILE && i < a.nx && j < a.ny) {
            const int k = j * a.nx + i;
            float ru = su[jj][ii], rv = sv[jj][ii];
            const bool bad = sbad[jj - 1][ii - 1];
            if (bad && a.replace) {
                float nu[8], nv[8];
                int c = 0, q = 0;
#pragma unroll
                for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
                    for (int di = -1; di <= 1; ++di) {
                        if (di == 0 && dj == 0) continue;
                        const bool ok = sok[jj + dj][ii + di] && !sbad[jj + dj - 1][ii + di - 1];
                        nu[q] = ok ? su[jj + dj][ii + di] : INFINITY;
                        nv[q] = ok ? sv[jj + dj][ii + di] : INFINITY;
                        c += ok ? 1 : 0;
                        ++q;
                    }
                if (c > 0) {
                    ru = median_sorted(nu, c);
                    rv = median_sorted(nv, c);
                }
            }
            uo[k] = ru;
            vo[k] = rv;
            if (mask) mask[k] = bad ? 0 : 1;
        }
    }
}

cudaError_t launch_uod(const UodArgs &a, int n_pairs, cudaStream_t st)
{
    dim3 grid((a.nx + UOD_TILE - 1) / UOD_TILE, (a.ny + UOD_TILE - 1) / UOD_TILE, n_pairs);
    uod_kernel<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// --------------------------------------------------------------- interp --

__device__ __forceinline__ void axis_wf(float pos, int n, float c0, int s, int &i0, int &i1, float &t)
{
    if (n <= 1) {
        i0 = i1 = 0;
        t = 0.f;
        return;
    }
    float f = (pos - c0) / (float)s;
    f = fminf(fmaxf(f, 0.f), (float)(n - 1));
    int ia = (int)floorf(f);
    if (ia > n - 2) ia = n - 2;
    i0 = ia;
    i1 = ia + 1;
    t = f - (float)ia;
}

__global__ void interp_kernel(const InterpArgs a)
{
    const int pair = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.dnx * a.dny) return;
    const float *su = (const float *)resolve(a.su, pair);
    const float *sv = (const float *)resolve(a.sv, pair);
    float *du = (float *)resolve(a.du, pair);
    float *dv = (float *)resolve(a.dv, pair);
    if (!su || !sv) {
        if (a.zero_if_null) {
            du[k] = 0.f;
            dv[k] = 0.f;
        }
        return;
    }
    const int j = k / a.dnx, i = k - j * a.dnx;
    const float f = (float)(1 << a.levels_up);
    const float X = (float)(i * a.ds) + 0.5f * (float)(a.dw - 1);
    const float Y = (float)(j * a.ds) + 0.5f * (float)(a.dw - 1);
    const float xs = (X + 0.5f) / f - 0.5f, ys = (Y + 0.5f) / f - 0.5f;
    const float c0 = 0.5f * (float)(a.sw - 1);
    int i0, i1, j0, j1;
    float tx, ty;
    axis_wf(xs, a.snx, c0, a.ss, i0, i1, tx);
    axis_wf(ys, a.sny, c0, a.ss, j0, j1, ty);
    float t0 = su[j0 * a.snx + i0] + tx * (su[j0 * a.snx + i1] - su[j0 * a.snx + i0]);
    float t1 = su[j1 * a.snx + i0] + tx * (su[j1 * a.snx + i1] - su[j1 * a.snx + i0]);
    du[k] = f * (t0 + ty * (t1 - t0));
    t0 = sv[j0 * a.snx + i0] + tx * (sv[j0 * a.snx + i1] - sv[j0 * a.snx + i0]);
    t1 = sv[j1 * a.snx + i0] + tx * (sv[j1 * a.snx + i1] - sv[j1 * a.snx + i0]);
    dv[k] = f * (t0 + ty * (t1 - t0));
}

cudaError_t launch_interp(const InterpArgs &a, int n_pairs, cudaStream_t st)
{
    const int n = a.dnx * a.dny;
    dim3 grid((n + 255) / 256, n_pairs);
    interp_kernel<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------ vorticity --

__global__ void vort_kernel(const VortArgs a)
{
    const int pair = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.nx * a.ny) return;
    const float *u = (const float *)resolve(a.u, pair);
    const float *v = (const float *)resolve(a.v, pair);
    float *o = (float *)resolve(a.out, pair);
    if (!o) return;
    const int j = k / a.nx, i = k - j * a.nx;
    const int nx = a.nx, ny = a.ny;
    const float s = (float)a.s;
    float dvdx = 0.f, dudy = 0.f;
    if (nx > 1) {
        if (i == 0) dvdx = (v[j * nx + 1] - v[j * nx]) / s;
        else if (i == nx - 1) dvdx = (v[j * nx + i] - v[j * nx + i - 1]) / s;
        else dvdx = (v[j * nx + i + 1] - v[j * nx + i - 1]) / (2.f * s);
    }
    if (ny > 1) {
        if (j == 0) dudy = (u[nx + i] - u[i]) / s;
        else if (j == ny - 1) dudy = (u[j * nx + i] - u[(j - 1) * nx + i]) / s;
        else dudy = (u[(j + 1) * nx + i] - u[(j - 1) * nx + i]) / (2.f * s);
    }
    o[k] = dvdx - dudy;
}

__global__ void ema_kernel(const float *__restrict__ x, float *state, size_t n, float alpha, int init)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float xi = x[i];
        state[i] = init ? xi : alpha * xi + (1.f - alpha) * state[i];
    }
}

cudaError_t launch_ema(const float *x, float *state, size_t n, float alpha, int init, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const size_t blocks = std::min<size_t>((n + 255) / 256, (size_t)device_sm_count() * 8);
    ema_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, state, n, alpha, init);
    return cudaGetLastError();
}

cudaError_t launch_vort(const VortArgs &a, int n_pairs, cudaStream_t st)
{
    const int n = a.nx * a.ny;
    dim3 grid((n + 255) / 256, n_pairs);
    vort_kernel<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------- downsample --

template <typename T>
__device__ __forceinline__ float ldp(const unsigned char *img, long long pitch, int x, int y)
{
    return (float)__ldg(reinterpret_cast<const T *>(img + (long long)y * pitch) + x);
}

template <typename T>
__device__ __forceinline__ float box2(const unsigned char *img, long long pitch, int x, int y)
{
    // (a + b + c + d) / 4 is exact in FP32 for integer (or quarter-integer) pixels
    return 0.25f * ((ldp<T>(img, pitch, 2 * x, 2 * y) + ldp<T>(img, pitch, 2 * x + 1, 2 * y)) +
                    (ldp<T>(img, pitch, 2 * x, 2 * y + 1) + ldp<T>(img, pitch, 2 * x + 1, 2 * y + 1)));
}

// Eight consecutive source pixels of a row from pixel p (p a multiple of 8):
// one 8-byte (u8), 16-byte (u16) or two 16-byte (float) loads.
template <typename T>
__device__ __forceinline__ void load8(const unsigned char *row, int p, float (&v)[8])
{
    if (sizeof(T) == 1) {
        const uint2 u = __ldg(reinterpret_cast<const uint2 *>(row) + p / 8);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            v[i] = (float)((u.x >> (8 * i)) & 0xffu);
            v[4 + i] = (float)((u.y >> (8 * i)) & 0xffu);
        }
    } else if (sizeof(T) == 2) {
        const uint4 u = __ldg(reinterpret_cast<const uint4 *>(row) + p / 8);
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            v[2 * i] = (float)(w[i] & 0xffffu);
            v[2 * i + 1] = (float)(w[i] >> 16);
        }
    } else {
        const float4 f0 = __ldg(reinterpret_cast<const float4 *>(row) + p / 4);
        const float4 f1 = __ldg(reinterpret_cast<const float4 *>(row) + p / 4 + 1);
        v[0] = f0.x; v[1] = f0.y; v[2] = f0.z; v[3] = f0.w;
        v[4] = f1.x; v[5] = f1.y; v[6] = f1.z; v[7] = f1.w;
    }
}

// Four consecutive outputs per thread (x0 = 4 k): their 2 x 8 source pixels by
// one vector load per source row and one 16-byte store, where the source rows
// and the destination row are aligned for them (checked per pair); the row's
// last outputs and unaligned rows take the scalar form.  Same sums, in the
// same order, either way.
template <typename T>
__device__ __forceinline__ void down_row4(const unsigned char *src, long long pitch, int x0, int y, int W2, float *d,
                                          bool vec)
{
    if (vec && x0 + 4 <= W2) {
        float r0[8], r1[8];
        load8<T>(src + (long long)(2 * y) * pitch, 2 * x0, r0);
        load8<T>(src + (long long)(2 * y + 1) * pitch, 2 * x0, r1);
        float o[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) o[i] = 0.25f * ((r0[2 * i] + r0[2 * i + 1]) + (r1[2 * i] + r1[2 * i + 1]));
        *reinterpret_cast<float4 *>(d) = make_float4(o[0], o[1], o[2], o[3]);
        return;
    }
    for (int k = 0; k < 4 && x0 + k < W2; ++k) d[k] = box2<T>(src, pitch, x0 + k, y);
}

__global__ void __launch_bounds__(256) down_kernel(const DownArgs a)
{
    const int pair = blockIdx.z;
    const int W2 = a.W / 2, H2 = a.H / 2;
    const int x0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x), y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x0 >= W2 || y >= H2) return;
    const unsigned char *src = (const unsigned char *)resolve(a.src, pair);
    float *dst = (float *)resolve(a.dst, pair);
    float *d = dst + (long long)(y + a.dst_margin) * a.dst_pitch + (x0 + a.dst_margin);
    const int bpp = a.fmt == PIX_U8 ? 1 : (a.fmt == PIX_U16 ? 2 : 4);
    const int align = bpp == 1 ? 8 : 16;
    const bool vec = ((reinterpret_cast<uintptr_t>(src) | (uintptr_t)a.pitch) % align) == 0 &&
                     (reinterpret_cast<uintptr_t>(d) % 16) == 0;
    if (a.fmt == PIX_U8) down_row4<uint8_t>(src, a.pitch, x0, y, W2, d, vec);
    else if (a.fmt == PIX_U16) down_row4<uint16_t>(src, a.pitch, x0, y, W2, d, vec);
    else down_row4<float>(src, a.pitch, x0, y, W2, d, vec);
}

// Eight consecutive pixels per thread: one 8-byte (u8), 16-byte (u16) or two
// 16-byte (float) loads and two 16-byte stores where the source row and the
// destination are aligned for them (checked per pair on the device), scalar
// accesses otherwise.
template <typename T>
__device__ __forceinline__ void ingest_row8(const unsigned char *row, int x, int W, float *d, bool vec)
{
    if (vec && x + 8 <= W) {
        float v[8];
        load8<T>(row, x, v);
        *reinterpret_cast<float4 *>(d) = make_float4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<float4 *>(d + 4) = make_float4(v[4], v[5], v[6], v[7]);
        return;
    }
    for (int k = 0; k < 8 && x + k < W; ++k) d[k] = (float)__ldg(reinterpret_cast<const T *>(row) + x + k);
}

__global__ void ingest_kernel(const IngestArgs a)
{
    const int pair = blockIdx.z;
    const int x = 8 * (blockIdx.x * blockDim.x + threadIdx.x), y = blockIdx.y;
    if (x >= a.W) return;
    const unsigned char *src = (const unsigned char *)resolve(a.src, pair);
    float *dst = (float *)resolve(a.dst, pair);
    const int bpp = a.fmt == PIX_U8 ? 1 : (a.fmt == PIX_U16 ? 2 : 4);
    const unsigned char *row = src + (long long)y * a.pitch;
    float *d = dst + (long long)(y + a.dst_margin) * a.dst_pitch + (x + a.dst_margin);
    const uintptr_t align = bpp == 1 ? 8 : 16;
    const bool vec = ((reinterpret_cast<uintptr_t>(row) % align) == 0) && ((reinterpret_cast<uintptr_t>(d) % 16) == 0);
    if (a.fmt == PIX_U8) ingest_row8<uint8_t>(row, x, a.W, d, vec);
    else if (a.fmt == PIX_U16) ingest_row8<uint16_t>(row, x, a.W, d, vec);
    else ingest_row8<float>(row, x, a.W, d, vec);
}

// One CTA copies UPLOAD_ROWS rows of one frame of one pair: 16-byte words
// where the source row starts on a 16-byte boundary, bytes otherwise.
constexpr int UPLOAD_ROWS = 8;

__global__ void __launch_bounds__(256) upload_kernel(const UploadArgs a)
{
    const int pair = blockIdx.z, which = blockIdx.y;
    const unsigned char *src = (const unsigned char *)resolve(which ? a.src_b : a.src_a, pair);
    unsigned char *dst = (unsigned char *)resolve(which ? a.dst_b : a.dst_a, pair);
    const int nw = a.row_bytes >> 4;
    for (int r = 0; r < UPLOAD_ROWS; ++r) {
        const int y = blockIdx.x * UPLOAD_ROWS + r;
        if (y >= a.H) return;
        const unsigned char *s = src + (long long)y * a.pitch;
        unsigned char *d = dst + (long long)y * a.dst_pitch;
        if (((uintptr_t)s & 15) == 0) {
            for (int i = threadIdx.x; i < nw; i += blockDim.x)
                reinterpret_cast<uint4 *>(d)[i] = reinterpret_cast<const uint4 *>(s)[i];
            for (int i = (nw << 4) + threadIdx.x; i < a.row_bytes; i += blockDim.x) d[i] = s[i];
        } else {
            for (int i = threadIdx.x; i < a.row_bytes; i += blockDim.x) d[i] = s[i];
        }
    }
}

cudaError_t launch_upload(const UploadArgs &a, int n_pairs, cudaStream_t st)
{
    dim3 grid((a.H + UPLOAD_ROWS - 1) / UPLOAD_ROWS, 2, n_pairs);
    upload_kernel<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_ingest(const IngestArgs &a, int n_pairs, cudaStream_t st)
{
    dim3 grid((a.W + 8 * 128 - 1) / (8 * 128), a.H, n_pairs);
    ingest_kernel<<<grid, 128, 0, st>>>(a);
    return cudaGetLastError();
}

// 256 threads per CTA: up to 128 along a row (four outputs each), the rest
// over rows
cudaError_t launch_down(const DownArgs &a, int n_pairs, cudaStream_t st)
{
    const int W2 = a.W / 2, H2 = a.H / 2;
    if (W2 < 1 || H2 < 1) return cudaSuccess;
    const int quads = (W2 + 3) / 4;
    const int tx = std::min(128, (quads + 31) / 32 * 32), ty = 256 / tx;
    dim3 block(tx, ty);
    dim3 grid((quads + tx - 1) / tx, (H2 + ty - 1) / ty, n_pairs);
    down_kernel<<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace rpiv
