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

// A tile is DTX x DTY output pixels: 64 x 128 when the batch fills the GPU
// (the per-tile set-up is spread over more pixels), 64 x 64 otherwise.
constexpr int DTX = 64, DTY_MAX = 128;
constexpr int DROWS = 4;            // rows per thread and slice (256 threads = 64 columns x 4 row phases)
constexpr int SLICE = 4 * DROWS;    // rows per slice
// Nodes and node rows a tile can touch, for steps >= 3 and for steps >= 8
// (checked on the host).  The shared arrays are sized by these caps: the
// smaller ones leave more of the SM's combined L1 / shared memory to the L1
// that serves the gathers.
constexpr int NODE_CAP = 1152, NODE_CAP_S8 = 256;
constexpr int nrow_cap(int dty, int min_step) { return dty / min_step + 4; }

// cell index and weight of a pixel position along one axis of the node grid
// (node i at c0 + i s; positions outside the hull take the border value)
// (the division stays: a rounded reciprocal of a step that is not a power of
// two would bias every weight the same way, up to 1e-5 px at 4k columns)
__device__ __forceinline__ void axis_weight(int pos, int n, float c0, float s, int &i0, float &t)
{
    if (n <= 1) {
        i0 = 0;
        t = 0.f;
        return;
    }
    float f = ((float)pos - c0) / s;
    f = fminf(fmaxf(f, 0.f), (float)(n - 1));
    int ia = (int)floorf(f);
    if (ia > n - 2) ia = n - 2;
    i0 = ia;
    t = f - (float)ia;
}

__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Exact float of a pixel: integers below 2^23 placed in the mantissa under the
// exponent of 2^23, minus 2^23 (two full-rate instructions instead of a
// conversion).
__device__ __forceinline__ float pix(uint8_t v) { return __uint_as_float(0x4B000000u | (uint32_t)v) - 8388608.f; }
__device__ __forceinline__ float pix(uint16_t v) { return __uint_as_float(0x4B000000u | (uint32_t)v) - 8388608.f; }
__device__ __forceinline__ float pix(float v) { return v; }

// floor of d (|d| < 2^22) as a float and as an int: the integer of the floored
// value read from the mantissa of fl + 1.5 * 2^23
__device__ __forceinline__ void floor_split(float d, float &fl, int &i)
{
    fl = floorf(d);
    i = __float_as_int(fl + 12582912.f) - 0x4B400000;
}

// The tile in slices of SLICE rows; within a slice all rows of a thread are
// unrolled so that their gathers are in flight together; rows and columns
// past the grown image are computed on clamped coordinates and not stored.
// CLAMP: the taps are clamped to the image (tiles near its border or with a
// displacement range reaching outside); otherwise the four taps of a pixel
// are read from one base pointer.  Off: the integer type of pixel offsets.
template <int DTY, typename T, typename Off, bool CLAMP>
__device__ __forceinline__ void deform_rows(const DeformArgs &a, const T *base, float *out, int djo, Off pe, int x,
                                            int y0, int lx, int ly0, const float2 *cuv, const int2 *rinfo)
{
    // warps whose 32 columns, and slices whose rows, lie past the grown
    // image store nothing: skip them (uniform per warp)
    if (x - (int)(threadIdx.x & 31) >= a.W + a.M) return;
    for (int half = 0; half < DTY / SLICE; ++half) {
        if (y0 + SLICE * half >= a.H + a.M) break;
        float res[DROWS];
#pragma unroll
        for (int k = 0; k < DROWS; ++k) {
            const int ly = SLICE * half + ly0 + 4 * k, y = y0 + ly;
            const int2 ri = rinfo[ly];
            const float ty = __int_as_float(ri.y);
            const float2 n0 = cuv[ri.x + lx], n1 = cuv[ri.x + djo + lx];
            float du = fmaf(ty, n1.x - n0.x, n0.x), dv = fmaf(ty, n1.y - n0.y, n0.y);
            if (CLAMP) {
                // NaN or absurd predictor values are clamped so the index math cannot overflow
                du = fminf(fmaxf(du, -1048576.f), 1048576.f);
                dv = fminf(fmaxf(dv, -1048576.f), 1048576.f);
            }
            float fx, fy;
            int ix, iy;
            floor_split(du, fx, ix);
            floor_split(dv, fy, iy);
            const float tx = du - fx, tyy = dv - fy;
            float b00, b10, b01, b11;
            if (CLAMP) {
                const int xl = x + ix, yl = y + iy;
                const int xa = min(max(xl, 0), a.W - 1), xb = min(max(xl + 1, 0), a.W - 1);
                const int ya = min(max(yl, 0), a.H - 1), yb = min(max(yl + 1, 0), a.H - 1);
                const T *ra = base + (Off)ya * pe, *rb = base + (Off)yb * pe;
                b00 = pix(__ldg(ra + xa));
                b10 = pix(__ldg(ra + xb));
                b01 = pix(__ldg(rb + xa));
                b11 = pix(__ldg(rb + xb));
            } else {
                const T *q = base + ((Off)(y + iy) * pe + (Off)(x + ix));
                b00 = pix(__ldg(q));
                b10 = pix(__ldg(q + 1));
                b01 = pix(__ldg(q + pe));
                b11 = pix(__ldg(q + pe + 1));
            }
            const float top = b00 + tx * (b10 - b00), bot = b01 + tx * (b11 - b01);
            res[k] = top + tyy * (bot - top);
        }
        if (x < a.W + a.M) {
            float *o = out + (long long)(y0 + SLICE * half + ly0 + a.M) * a.out_pitch + (x + a.M);
#pragma unroll
            for (int k = 0; k < DROWS; ++k) {
                const int y = y0 + SLICE * half + ly0 + 4 * k;
                if (y < a.H + a.M) o[(long long)(4 * k) * a.out_pitch] = res[k];
            }
        }
    }
}

template <int DTY, typename T, typename Off>
__device__ __forceinline__ void deform_rows_any(const DeformArgs &a, const T *base, float *out, bool inside, int djo,
                                                Off pe, int x, int y0, int lx, int ly0, const float2 *cuv,
                                                const int2 *rinfo)
{
    if (inside)
        deform_rows<DTY, T, Off, false>(a, base, out, djo, pe, x, y0, lx, ly0, cuv, rinfo);
    else
        deform_rows<DTY, T, Off, true>(a, base, out, djo, pe, x, y0, lx, ly0, cuv, rinfo);
}

// The field is bilinear in the nodes: the tile first interpolates every node
// row it touches along x at each of its columns, already scaled (cuv), and
// stores per row its node-row offset and weight (rinfo), so that a pixel needs
// one interpolation along y.  A tile whose taps provably stay inside the image
// (its displacement lies within the range of its nodes, a convex combination)
// skips the clamping; either way every tap is the clamp-to-edge sample.
template <typename T, int DTY, int MIN_STEP>
__device__ void deform_tile(const DeformArgs &a, const unsigned char *img, const float *pu, const float *pv,
                            float *out)
{
    constexpr int NCAP = MIN_STEP >= 8 ? NODE_CAP_S8 : NODE_CAP;
    __shared__ float nu[NCAP], nv[NCAP];
    __shared__ float2 cuv[nrow_cap(DTY, MIN_STEP) * DTX];
    __shared__ int2 rinfo[DTY];
    __shared__ float red[4][8];
    const int x0 = blockIdx.x * DTX - a.M, y0 = blockIdx.y * DTY - a.M;
    const float c0 = 0.5f * (float)(a.w - 1), sf = (float)a.s;
    const bool has = pu != nullptr && pv != nullptr;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int lx = threadIdx.x % DTX, ly0 = threadIdx.x / DTX;
    const int x = x0 + lx;
    float umin = 0.f, umax = 0.f, vmin = 0.f, vmax = 0.f;
    bool any_nan = false;
    int djo = 0;
    if (has) {
        int ilo, ihi, jlo, jhi;
        float t;
        axis_weight(x0, a.nx, c0, sf, ilo, t);
        axis_weight(x0 + DTX - 1, a.nx, c0, sf, ihi, t);
        axis_weight(y0, a.ny, c0, sf, jlo, t);
        axis_weight(y0 + DTY - 1, a.ny, c0, sf, jhi, t);
        ihi = min(ihi + 1, a.nx - 1);
        jhi = min(jhi + 1, a.ny - 1);
        const int nwn = ihi - ilo + 1, nhn = jhi - jlo + 1;
        float lu0 = INFINITY, lu1 = -INFINITY, lv0 = INFINITY, lv1 = -INFINITY;
        bool nan_seen = false;
        for (int e = threadIdx.x; e < nwn * nhn; e += blockDim.x) {
            const int jj = e / nwn, ii = e - jj * nwn;
            const float fu = pu[(jlo + jj) * a.nx + ilo + ii], fv = pv[(jlo + jj) * a.nx + ilo + ii];
            nu[e] = fu;
            nv[e] = fv;
            nan_seen |= (fu != fu) || (fv != fv);
            lu0 = fminf(lu0, fu);
            lu1 = fmaxf(lu1, fu);
            lv0 = fminf(lv0, fv);
            lv1 = fmaxf(lv1, fv);
        }
        lu0 = warp_min(lu0);
        lu1 = warp_max(lu1);
        lv0 = warp_min(lv0);
        lv1 = warp_max(lv1);
        if (lane == 0) {
            red[0][warp] = lu0;
            red[1][warp] = lu1;
            red[2][warp] = lv0;
            red[3][warp] = lv1;
        }
        for (int e = threadIdx.x; e < DTY; e += blockDim.x) {
            int j0;
            axis_weight(y0 + e, a.ny, c0, sf, j0, t);
            rinfo[e] = make_int2((j0 - jlo) * DTX, __float_as_int(t));
        }
        any_nan = __syncthreads_or(nan_seen);
        // node rows interpolated along x at this thread's column, scaled
        {
            int i0;
            float tx;
            axis_weight(x, a.nx, c0, sf, i0, tx);
            const int ci = i0 - ilo, di = a.nx > 1 ? 1 : 0;
            for (int jj = ly0; jj < nhn; jj += blockDim.x / DTX) {
                const float *ru = nu + jj * nwn + ci, *rv = nv + jj * nwn + ci;
                cuv[jj * DTX + lx] = make_float2(a.scale * (ru[0] + tx * (ru[di] - ru[0])),
                                                 a.scale * (rv[0] + tx * (rv[di] - rv[0])));
            }
        }
        umin = red[0][0];
        umax = red[1][0];
        vmin = red[2][0];
        vmax = red[3][0];
        for (int k = 1; k < 8; ++k) {
            umin = fminf(umin, red[0][k]);
            umax = fmaxf(umax, red[1][k]);
            vmin = fminf(vmin, red[2][k]);
            vmax = fmaxf(vmax, red[3][k]);
        }
        // the central warp scales by -1/2 for frame A: the range flips
        const float su0 = a.scale * umin, su1 = a.scale * umax, sv0 = a.scale * vmin, sv1 = a.scale * vmax;
        umin = fminf(su0, su1);
        umax = fmaxf(su0, su1);
        vmin = fminf(sv0, sv1);
        vmax = fmaxf(sv0, sv1);
        djo = a.ny > 1 ? DTX : 0;
        __syncthreads();
    } else {
        // no predictor: one zero node row, weight 0 on every row
        if (threadIdx.x < DTX) cuv[threadIdx.x] = make_float2(0.f, 0.f);
        if (threadIdx.x < DTY) rinfo[threadIdx.x] = make_int2(0, 0);
        __syncthreads();
    }
    // every tap of the tile inside the image, with a pixel to spare against rounding
    const bool inside = !any_nan && umin > -1048576.f && umax < 1048576.f && vmin > -1048576.f &&
                        vmax < 1048576.f && x0 + floorf(umin) - 1.f >= 0.f &&
                        x0 + DTX - 1 + floorf(umax) + 2.f <= (float)(a.W - 1) && y0 + floorf(vmin) - 1.f >= 0.f &&
                        y0 + DTY - 1 + floorf(vmax) + 2.f <= (float)(a.H - 1);
    const T *base = reinterpret_cast<const T *>(img);
    const long long pe = a.pitch / (long long)sizeof(T);  // row pitch in pixels (a multiple of the pixel size)
    // 32-bit pixel offsets when the whole image fits them
    if ((long long)a.H * pe < (1LL << 31))
        deform_rows_any<DTY, T, int>(a, base, out, inside, djo, (int)pe, x, y0, lx, ly0, cuv, rinfo);
    else
        deform_rows_any<DTY, T, long long>(a, base, out, inside, djo, pe, x, y0, lx, ly0, cuv, rinfo);
}

// one kernel per pixel type, so that each holds a single copy of the tile's
// shared arrays; MIN_STEP: the smallest node step its caps allow (3 or 8).
// Six CTAs per SM (40 registers).
template <typename T, int DTY, int MIN_STEP>
__global__ void __launch_bounds__(256, 8) deform_kernel(const DeformArgs a)
{
    const int pair = blockIdx.z;
    const unsigned char *img = (const unsigned char *)resolve(a.img, pair);
    const float *pu = (const float *)resolve(a.pred_u, pair);
    const float *pv = (const float *)resolve(a.pred_v, pair);
    float *out = (float *)resolve(a.out, pair);
    deform_tile<T, DTY, MIN_STEP>(a, img, pu, pv, out);
}

// nodes touched by a DTX x dty tile along each axis, plus the neighbour node,
// within the caps of the kernel for steps >= min_step
bool nodes_fit(int s, int nx, int ny, int dty, int min_step)
{
    const int cx = DTX / s + 3, cy = dty / s + 3;
    const int cap = min_step >= 8 ? NODE_CAP_S8 : NODE_CAP;
    return std::min(cx, nx) * std::min(cy, ny) <= cap && std::min(cy, ny) <= nrow_cap(dty, min_step);
}

}  // namespace

bool deform_nodes_fit(int w, int s, int nx, int ny)
{
    (void)w;
    return nodes_fit(s, nx, ny, DTY_MAX, 3);
}

template <int DTY, int MIN_STEP>
static void launch_tiles_caps(const DeformArgs &a, int n_pairs, cudaStream_t st)
{
    const int WE = a.W + 2 * a.M, HE = a.H + 2 * a.M;
    dim3 grid((WE + DTX - 1) / DTX, (HE + DTY - 1) / DTY, n_pairs);
    if (a.fmt == PIX_U8) deform_kernel<uint8_t, DTY, MIN_STEP><<<grid, 256, 0, st>>>(a);
    else if (a.fmt == PIX_U16) deform_kernel<uint16_t, DTY, MIN_STEP><<<grid, 256, 0, st>>>(a);
    else deform_kernel<float, DTY, MIN_STEP><<<grid, 256, 0, st>>>(a);
}

// the small-cap kernel whenever the grid fits its caps (no predictor: one
// zero node row)
template <int DTY>
static void launch_tiles(const DeformArgs &a, int n_pairs, cudaStream_t st)
{
    const bool has = a.pred_u.base != nullptr && a.pred_v.base != nullptr;
    if (!has || nodes_fit(a.s, a.nx, a.ny, DTY, 8)) launch_tiles_caps<DTY, 8>(a, n_pairs, st);
    else launch_tiles_caps<DTY, 3>(a, n_pairs, st);
}

// 64 x 128 tiles when they still make two full waves (five CTAs per SM on
// 152 SMs): 0.235 -> 0.215 ms per 64-pair 1 MP launch; a single pair keeps the
// finer grid of 64 x 64 tiles
cudaError_t launch_deform(const DeformArgs &a, int n_pairs, cudaStream_t st)
{
    const long long WE = a.W + 2LL * a.M, HE = a.H + 2LL * a.M;
    const long long tall = ((WE + DTX - 1) / DTX) * ((HE + DTY_MAX - 1) / DTY_MAX) * n_pairs;
    if (tall >= 2LL * device_sm_count() * 5) launch_tiles<DTY_MAX>(a, n_pairs, st);
    else launch_tiles<64>(a, n_pairs, st);
    return cudaGetLastError();
}

}  // namespace rpiv
