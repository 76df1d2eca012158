// Pre-processing before the flow estimate (paper Sec. 2): a high-pass filter
// against the static background, then contrast-limited adaptive histogram
// equalisation (CLAHE).
//
//   high-pass  d = max(0, n I - S), S the clamp-to-edge sum of I over the
//              (2 hp + 1)^2 box around the pixel, n its pixel count (hp = 0:
//              d = I, n = 1); the filtered value is d / n
//   CLAHE      256 bins over [0, vmax + 1), bin = floor(d 256 / (n (vmax + 1)));
//              per tile of N pixels the histogram is clipped at
//              L = max(1, floor(clip% N / (100 * 256))), the excess E spread as
//              E / 256 to every bin and one more to the first E mod 256 bins;
//              map[b] = cdf[b] vmax / N; a pixel blends the maps of the four
//              tiles whose centres surround it, bilinearly
//
// Box sums, bins and cumulative counts are integers, so every bin is exact.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rpiv_internal.h"

namespace rpiv {

namespace {

constexpr int NBINS = 256;

template <typename T>
__device__ __forceinline__ int px(const unsigned char *img, long long pitch, int x, int y)
{
    return (int)__ldg(reinterpret_cast<const T *>(img + (long long)y * pitch) + x);
}

// R(x, y) = sum over dx in [-hp, hp] of I(clamp(x + dx), y)
template <typename T>
__global__ void hp_rows(const PreArgs a, int *R)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= a.W) return;
    const unsigned char *img = static_cast<const unsigned char *>(a.img);
    int s = 0;
    for (int dx = -a.hp; dx <= a.hp; ++dx) s += px<T>(img, a.pitch, min(max(x + dx, 0), a.W - 1), y);
    R[(long long)y * a.W + x] = s;
}

// d = max(0, n I - S) with S the vertical clamp-to-edge sum of R (hp = 0: d = I)
template <typename T>
__global__ void hp_cols(const PreArgs a, const int *R, int *D)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= a.W) return;
    const unsigned char *img = static_cast<const unsigned char *>(a.img);
    const int I = px<T>(img, a.pitch, x, y);
    int d = I;
    if (a.hp > 0) {
        int S = 0;
        for (int dy = -a.hp; dy <= a.hp; ++dy) S += R[(long long)min(max(y + dy, 0), a.H - 1) * a.W + x];
        const int n = (2 * a.hp + 1) * (2 * a.hp + 1);
        d = max(n * I - S, 0);
    }
    D[(long long)y * a.W + x] = d;
}

__device__ __forceinline__ int bin_of(int d, long long den)
{
    const long long b = (long long)d * NBINS / den;
    return b > NBINS - 1 ? NBINS - 1 : (int)b;
}

// One CTA of MAP_THREADS per tile: histogram, clip, spread, cumulative map.
// Background-dominated particle images put most pixels of a tile in a few
// bins, so lanes of a warp that hold the same bin add their count with one
// shared-memory atomic (the lane with the lowest index of the group).  The
// cumulative counts are an exact integer scan over the 256 bins (warp scans,
// then the warps' totals); each bin's map value is then formed on its own.
constexpr int MAP_THREADS = 1024;

__global__ void __launch_bounds__(MAP_THREADS) clahe_maps(const PreArgs a, const int *D, float *maps)
{
    __shared__ int h[NBINS];
    __shared__ int excess;
    __shared__ int wtot[NBINS / 32];
    const int ti = blockIdx.x, tj = blockIdx.y, tid = threadIdx.x, lane = tid & 31;
    const int tw = (a.W + a.tx - 1) / a.tx, th = (a.H + a.ty - 1) / a.ty;
    const int x0 = ti * tw, x1 = min(a.W, x0 + tw), y0 = tj * th, y1 = min(a.H, y0 + th);
    const long long den = (long long)a.n * (a.vmax + 1);
    if (tid < NBINS) h[tid] = 0;
    if (tid == 0) excess = 0;
    __syncthreads();
    const int cw = max(x1 - x0, 0), N = cw * max(y1 - y0, 0);
    // warp-uniform trip count, so that every lane takes part in the match
    for (int base = tid - lane; base < N; base += blockDim.x) {
        const int e = base + lane;
        const int bin = e < N ? bin_of(D[(long long)(y0 + e / cw) * a.W + x0 + e % cw], den) : -1;
        const unsigned grp = __match_any_sync(0xffffffffu, bin);
        if (bin >= 0 && lane == __ffs(grp) - 1) atomicAdd(&h[bin], __popc(grp));
    }
    __syncthreads();
    int L = (int)((long long)a.clip_pct * N / (100LL * NBINS));
    if (L < 1) L = 1;
    if (tid < NBINS) {
        const int over = h[tid] > L ? h[tid] - L : 0;
        if (over) atomicAdd(&excess, over);
    }
    __syncthreads();
    int c = 0;
    if (tid < NBINS) {
        const int E = excess;
        c = min(h[tid], L) + E / NBINS + (tid < E % NBINS ? 1 : 0);
        // inclusive scan within the warp, then the totals of the warps before
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, c, o);
            if (lane >= o) c += t;
        }
        if (lane == 31) wtot[tid >> 5] = c;
    }
    __syncthreads();
    if (tid < NBINS) {
        for (int k = 0; k < (tid >> 5); ++k) c += wtot[k];
        float *m = maps + ((long long)tj * a.tx + ti) * NBINS;
        m[tid] = N > 0 ? (float)((double)c * a.vmax / (double)N) : 0.f;
    }
}

// tile pair and weight along one axis: centres at t * ts + (width_t - 1) / 2,
// clamped to the outer centres
__device__ __forceinline__ void tile_pair(int p, int ext, int ts, int nt, int &t0, int &t1, float &w)
{
    const float c0 = 0.5f * (float)(ts - 1);
    const int tl = nt - 1;
    const float cl = (float)(tl * ts) + 0.5f * (float)(ext - tl * ts - 1);
    if (nt == 1 || (float)p <= c0) {
        t0 = t1 = 0;
        w = 0.f;
    } else if ((float)p >= cl) {
        t0 = t1 = tl;
        w = 0.f;
    } else {
        int t = (int)floorf(((float)p - c0) / (float)ts);
        if (t > nt - 2) t = nt - 2;
        t0 = t;
        t1 = t + 1;
        const float a0 = (float)(t0 * ts) + 0.5f * (float)(ts - 1);
        const float a1 = (t1 == tl) ? cl : (float)(t1 * ts) + 0.5f * (float)(ts - 1);
        w = ((float)p - a0) / (a1 - a0);
    }
}

__global__ void clahe_apply(const PreArgs a, const int *D, const float *maps, float *out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= a.W) return;
    const int d = D[(long long)y * a.W + x];
    float v;
    if (a.clip_pct <= 0) {
        v = (float)d / (float)a.n;
    } else {
        const int tw = (a.W + a.tx - 1) / a.tx, th = (a.H + a.ty - 1) / a.ty;
        int i0, i1, j0, j1;
        float wx, wy;
        tile_pair(x, a.W, tw, a.tx, i0, i1, wx);
        tile_pair(y, a.H, th, a.ty, j0, j1, wy);
        const int b = bin_of(d, (long long)a.n * (a.vmax + 1));
        const float m00 = maps[((long long)j0 * a.tx + i0) * NBINS + b], m01 = maps[((long long)j0 * a.tx + i1) * NBINS + b];
        const float m10 = maps[((long long)j1 * a.tx + i0) * NBINS + b], m11 = maps[((long long)j1 * a.tx + i1) * NBINS + b];
        v = (1.f - wy) * ((1.f - wx) * m00 + wx * m01) + wy * ((1.f - wx) * m10 + wx * m11);
    }
    out[(long long)y * a.out_pitch + x] = v;
}

}  // namespace

size_t preprocess_scratch_bytes(int W, int H, int tx, int ty)
{
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    return 2 * up((size_t)W * H * 4) + up((size_t)tx * ty * NBINS * 4);
}

cudaError_t launch_preprocess(const PreArgs &a, void *scratch, cudaStream_t st)
{
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    char *s = static_cast<char *>(scratch);
    int *R = reinterpret_cast<int *>(s);
    int *D = reinterpret_cast<int *>(s + up((size_t)a.W * a.H * 4));
    float *maps = reinterpret_cast<float *>(s + 2 * up((size_t)a.W * a.H * 4));
    const dim3 grid((a.W + 255) / 256, a.H);
    if (a.hp > 0) {
        if (a.fmt == PIX_U8) hp_rows<uint8_t><<<grid, 256, 0, st>>>(a, R);
        else hp_rows<uint16_t><<<grid, 256, 0, st>>>(a, R);
    }
    if (a.fmt == PIX_U8) hp_cols<uint8_t><<<grid, 256, 0, st>>>(a, R, D);
    else hp_cols<uint16_t><<<grid, 256, 0, st>>>(a, R, D);
    if (a.clip_pct > 0) clahe_maps<<<dim3(a.tx, a.ty), MAP_THREADS, 0, st>>>(a, D, maps);
    clahe_apply<<<grid, 256, 0, st>>>(a, D, maps, a.out);
    return cudaGetLastError();
}

}  // namespace rpiv
