// Image deformation by the predictor (paper Sec. 2: the pre-processed pair is
// warped by the current displacement estimate before the correlation).
//
//   out(x, y) = I(x + c du(x, y), y + c dv(x, y))     bilinear, clamp-to-edge
//
// where (du, dv) is the bilinear interpolation of the predictor grid at the
// pixel (border values continued outside the node hull), c = 1 for the
// frame-B-only warp and +-1/2 for the central warp of either frame.  The output
// covers the image grown by a margin M on every side, because correlation
// shifts reach M pixels outside the windows; it is written once per pixel
// and read by the correlation pass of the same grid.
#include <algorithm>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "rpiv_internal.h"

namespace rpiv {

namespace {

constexpr int DTX = 64, DTY = 32;  // output pixels per CTA
constexpr int DROWS = DTY / 4;     // rows per thread (256 threads = 64 columns x 4 row phases)
constexpr int NODE_CAP = 512;      // nodes a tile can touch (checked on the host)

__device__ __forceinline__ void axis_weight(int pos, int n, float c0, int s, int &i0, float &t)
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
__device__ __forceinline__ float tap(const unsigned char *img, long long pitch, int x, int y)
{
    return (float)__ldg(reinterpret_cast<const T *>(img + (long long)y * pitch) + x);
}

template <typename T>
__device__ void deform_tile(const DeformArgs &a, const unsigned char *img, const float *pu, const float *pv,
                            float *out)
{
    __shared__ float nu[NODE_CAP], nv[NODE_CAP];
    __shared__ int cix[DTX], riy[DTY];
    __shared__ float ctx[DTX], rty[DTY];
    const int x0 = blockIdx.x * DTX - a.M, y0 = blockIdx.y * DTY - a.M;
    const float c0 = 0.5f * (float)(a.w - 1);
    const bool has = pu != nullptr && pv != nullptr;
    int ilo = 0, jlo = 0, nwn = 1;
    if (has) {
        int ihi, jhi;
        float t;
        axis_weight(x0, a.nx, c0, a.s, ilo, t);
        axis_weight(x0 + DTX - 1, a.nx, c0, a.s, ihi, t);
        axis_weight(y0, a.ny, c0, a.s, jlo, t);
        axis_weight(y0 + DTY - 1, a.ny, c0, a.s, jhi, t);
        ihi = min(ihi + 1, a.nx - 1);
        jhi = min(jhi + 1, a.ny - 1);
        nwn = ihi - ilo + 1;
        const int nhn = jhi - jlo + 1;
        for (int e = threadIdx.x; e < nwn * nhn; e += blockDim.x) {
            const int jj = e / nwn, ii = e - jj * nwn;
            nu[e] = pu[(jlo + jj) * a.nx + ilo + ii];
            nv[e] = pv[(jlo + jj) * a.nx + ilo + ii];
        }
        for (int e = threadIdx.x; e < DTX; e += blockDim.x) {
            int i0;
            float t;
            axis_weight(x0 + e, a.nx, c0, a.s, i0, t);
            cix[e] = i0 - ilo;
            ctx[e] = t;
        }
        for (int e = threadIdx.x; e < DTY; e += blockDim.x) {
            int j0;
            float t;
            axis_weight(y0 + e, a.ny, c0, a.s, j0, t);
            riy[e] = j0 - jlo;
            rty[e] = t;
        }
    }
    __syncthreads();
    const int di = a.nx > 1 ? 1 : 0, dj = a.ny > 1 ? 1 : 0;
    const int lx = threadIdx.x % DTX, ly0 = threadIdx.x / DTX;
    const int x = x0 + lx;
    // all rows of a thread are unrolled so that their 4 DROWS gathers are in
    // flight together; rows and columns past the grown image are computed on
    // clamped coordinates and not stored
    float res[DROWS];
#pragma unroll
    for (int k = 0; k < DROWS; ++k) {
        const int ly = ly0 + 4 * k, y = y0 + ly;
        float du = 0.f, dv = 0.f;
        if (has) {
            const int i0 = cix[lx], j0 = riy[ly];
            const float tx = ctx[lx], ty = rty[ly];
            const int k00 = j0 * nwn + i0, k01 = k00 + dj * nwn;
            float t0 = nu[k00] + tx * (nu[k00 + di] - nu[k00]);
            float t1 = nu[k01] + tx * (nu[k01 + di] - nu[k01]);
            du = a.scale * (t0 + ty * (t1 - t0));
            t0 = nv[k00] + tx * (nv[k00 + di] - nv[k00]);
            t1 = nv[k01] + tx * (nv[k01 + di] - nv[k01]);
            dv = a.scale * (t0 + ty * (t1 - t0));
            // NaN or absurd predictor values are clamped so the index math cannot overflow
            du = fminf(fmaxf(du, -1048576.f), 1048576.f);
            dv = fminf(fmaxf(dv, -1048576.f), 1048576.f);
        }
        const float fx = floorf(du), fy = floorf(dv);
        const float tx = du - fx, ty = dv - fy;
        const int ix = x + (int)fx, iy = y + (int)fy;
        const int xa = min(max(ix, 0), a.W - 1), xb = min(max(ix + 1, 0), a.W - 1);
        const int ya = min(max(iy, 0), a.H - 1), yb = min(max(iy + 1, 0), a.H - 1);
        const float b00 = tap<T>(img, a.pitch, xa, ya), b10 = tap<T>(img, a.pitch, xb, ya);
        const float b01 = tap<T>(img, a.pitch, xa, yb), b11 = tap<T>(img, a.pitch, xb, yb);
        const float top = b00 + tx * (b10 - b00), bot = b01 + tx * (b11 - b01);
        res[k] = top + ty * (bot - top);
    }
    if (x < a.W + a.M) {
#pragma unroll
        for (int k = 0; k < DROWS; ++k) {
            const int y = y0 + ly0 + 4 * k;
            if (y < a.H + a.M) out[(long long)(y + a.M) * a.out_pitch + (x + a.M)] = res[k];
        }
    }
}

__global__ void __launch_bounds__(256) deform_kernel(const DeformArgs a)
{
    const int pair = blockIdx.z;
    const unsigned char *img = (const unsigned char *)resolve(a.img, pair);
    const float *pu = (const float *)resolve(a.pred_u, pair);
    const float *pv = (const float *)resolve(a.pred_v, pair);
    float *out = (float *)resolve(a.out, pair);
    if (a.fmt == PIX_U8) deform_tile<uint8_t>(a, img, pu, pv, out);
    else if (a.fmt == PIX_U16) deform_tile<uint16_t>(a, img, pu, pv, out);
    else deform_tile<float>(a, img, pu, pv, out);
}

}  // namespace

bool deform_nodes_fit(int w, int s, int nx, int ny)
{
    (void)w;
    // nodes touched by a DTX x DTY tile along each axis, plus the neighbour node
    const int cx = DTX / s + 3, cy = DTY / s + 3;
    return std::min(cx, nx) * std::min(cy, ny) <= NODE_CAP;
}

cudaError_t launch_deform(const DeformArgs &a, int n_pairs, cudaStream_t st)
{
    const int WE = a.W + 2 * a.M, HE = a.H + 2 * a.M;
    dim3 grid((WE + DTX - 1) / DTX, (HE + DTY - 1) / DTY, n_pairs);
    deform_kernel<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace rpiv
