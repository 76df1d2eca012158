// Correlation pass with the planes on the fifth-generation tensor cores
// (tcgen05, accumulators in tensor memory), for 50 % overlap (w = 2s, s a
// multiple of 8) at r = 4 (paper Sec. 2: correlation coefficients of the
// warped pair; here BF16 or FP16 products with FP32 accumulation choose the
// integer peak, and the five-point stencil of the Gaussian fit is refitted in
// FP32 from the FP32 frames).
//
// The contraction.  For one window, a group of TC_ROWS consecutive rows r of
// B' and the A rows that meet them (a zero-banded slab, so that rows outside
// the window contribute nothing), one MMA of M = 128, N = 16, K = 16 computes
//     D[(c, i)][n] = sum_k B'(r0 + i, x0 + k + c - R) (A(a0 + n, x0 + k) - m)
// with M = (shift slot c, row i): 32 slots of TC_ROWS rows, the slots c <= 2R
// being shifted copies of B' (sx = c - R), N = 16 A rows, K = 16 columns of
// the window.  Since sy = r0 + i - (a0 + n) = i + R - n for every group, the
// groups of a window accumulate into one TMEM block of 16 columns, and
//     P_w(sy, sx) = sum_i D[(sx + R, i)][i + R - sy]
// is a four-term diagonal sum in the epilogue.  m is a per-tile offset
// subtracted from both frames before rounding to 16 bits (it is restored
// exactly in FP32 from the window and box sums), which keeps the rounded
// operands small.
//
// Layouts (canonical K-major, no swizzle: 8 rows of 16 bytes per core matrix):
//   copies  per chunk q of 8 columns: slots c = 0..7, each TC_ROWS rows of 16 B
//           (slot c holds B' shifted by c - R); the M index m = TC_ROWS c + i
//           is linear at 16 B (SBO = 128) and the chunk stride (LBO) is 8
//           slots, so slot c >= 8 of chunk q is slot c - 8 of chunk q + 1,
//           which holds B' shifted by c - R as well: eight copies serve all
//           2R + 1 <= 16 shifts.  A group keeps one chunk past the tile's
//           columns for them; the slots beyond 2R read further on (their D rows
//           are never read).
//   slab    per chunk q: the window row's A rows from 2R above the window to
//           16 - TC_ROWS below it, rows of 16 B (SBO = 128), chunk stride LBO
// Warp roles in the tensor-core phase (no CTA barrier inside it): producer
// warps build each window row's slab (double-buffered) and its groups' copies
// into a ring of slots; one issuer thread waits for a slot to fill, runs its
// MMAs for every window of the row into the row's TMEM block (double-buffered
// by row) and commits, which frees the slot; a commit after a row's last
// group releases its slab and hands its accumulators to the epilogue warps,
// which free the TMEM block when they have read it.  All waits are bounded and
// share an abort flag, so that one timeout ends every role.
//
// The five-point refit is exact FP32: block planes over the shifts |s| <= 2
// around the predictor (FP32 FMAs on the CUDA cores, before the tensor-core
// phase) supply the stencil of every peak within one pixel of the predictor;
// the rare others are summed directly.
#pragma once

#include "pass_impl.cuh"

namespace rpiv {

constexpr int TC_ROWS = 4;    // B' rows per MMA group
constexpr int TC_M = 128;     // 32 shift slots x TC_ROWS rows
constexpr int TC_N = 16;      // A rows of a group
constexpr int TC_R = 4;       // the radius these kernels are built for
constexpr int TC_EB_PITCH = 20;  // floats per lane in the epilogue buffer (conflict-free 128-bit stores)
constexpr int TC_RN = 2;         // radius of the FP32 block planes of the refit

static_assert(TC_ROWS + 2 * TC_R <= TC_N, "a group's A rows must fit N");

// ------------------------------------------------ tcgen05 building blocks --

// Shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets, each >> 4 in 14 bits; bit 46 = descriptor version of this family;
// no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, A and B both BF16 (or
// both F16), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
template <int PREC>
__device__ __forceinline__ uint32_t tc_idesc()
{
    constexpr uint32_t f = PREC == PREC_BF16 ? 1u : 0u;
    return (1u << 4) | (f << 7) | (f << 10) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// arrive on bar once every MMA this thread issued so far has completed
__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 lanes x 16 columns of FP32 from tensor memory (the warp's lane quarter)
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// whole warp: allocate cols columns (power of two >= 32); the address lands in *slot
__device__ __forceinline__ void tc_alloc(uint32_t *slot, int cols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_dealloc(uint32_t taddr, int cols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}

// Bounded wait of one warp on phase `parity` of bar: lane 0 polls, giving up
// after the limit (error word and abort flag set) or as soon as any role has
// aborted (even if the phase completed); every lane returns the verdict.
static __device__ __forceinline__ bool warp_wait(const PassArgs &a, uint64_t *bar, uint32_t parity,
                                                 volatile int *abort)
{
    int ok = 0;
    if ((threadIdx.x & 31) == 0) {
        const int lim = a.spin > 0 ? a.spin : MBAR_SPIN_LIMIT;
        for (int it = 0; it < lim && !*abort; ++it) {
            if (mbar_try_wait(bar, parity)) {
                ok = 1;
                break;
            }
        }
        if (!ok) {
            if (!*abort && a.err) atomicOr(a.err, 1);
            *abort = 1;
        }
    }
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// ------------------------------------------------------ operand staging --

template <int PREC>
__device__ __forceinline__ uint4 pack8(float4 lo, float4 hi, float m)
{
    uint4 r;
    r.x = pack2<PREC>(lo.x - m, lo.y - m);
    r.y = pack2<PREC>(lo.z - m, lo.w - m);
    r.z = pack2<PREC>(hi.x - m, hi.y - m);
    r.w = pack2<PREC>(hi.z - m, hi.w - m);
    return r;
}

// Slab of window row wy by threads t = 0 .. nt - 1 of the producer warps:
// slab row j holds A row wy s - 2R + j (tile rows), minus m, where it lies in
// the window; zero elsewhere.
template <int PREC>
static __device__ __forceinline__ void tc_slab(const PassPlan &P, const TileGeom &g, const float *As,
                                               unsigned char *slab, int wy, float m, int t, int nt)
{
    const int rows = P.slab_rows, nch = g.aw >> 3;
    for (int it = t; it < rows * nch; it += nt) {
        const int q = it / rows, j = it - q * rows;
        const int r = j - 2 * TC_R;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (r >= 0 && r < g.w) {
            const float *src = As + (wy * g.s + r) * P.a_pitch + 8 * q;
            v = pack8<PREC>(*reinterpret_cast<const float4 *>(src), *reinterpret_cast<const float4 *>(src + 4), m);
        }
        *reinterpret_cast<uint4 *>(slab + q * P.slab_lbo + j * 16) = v;
    }
}

// Copies of group gi of window row wy into a ring slot, by the lanes of one
// warp: B' rows y = wy s - R + TC_ROWS gi + i (tile rows); slot c of chunk q,
// row i holds B'(y, 8q + t + c - R) - m.  A lane takes one (row, chunk), rows
// fastest (so that a store instruction covers consecutive 16-byte rows): 16
// floats, the even and odd column pairs converted once, eight 16-byte stores.
template <int PREC>
static __device__ __forceinline__ void tc_group(const PassPlan &P, const TileGeom &g, const float *Bs,
                                                unsigned char *dst0, int wy, int gi, float m, int t, int nt)
{
    constexpr int R = TC_R;
    const int nq = (g.aw >> 3) + 1;
    for (int it = t; it < TC_ROWS * nq; it += nt) {
        const int q = it / TC_ROWS, i = it - q * TC_ROWS;
        const int y = wy * g.s - R + TC_ROWS * gi + i;
        const float *src = Bs + (y + R + 1) * P.b_pitch + P.padl + 8 * q - R;
        float v[16];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float4 f = *reinterpret_cast<const float4 *>(src + 4 * j);
            v[4 * j] = f.x - m;
            v[4 * j + 1] = f.y - m;
            v[4 * j + 2] = f.z - m;
            v[4 * j + 3] = f.w - m;
        }
        uint32_t ev[8], od[7];
#pragma unroll
        for (int j = 0; j < 8; ++j) ev[j] = pack2<PREC>(v[2 * j], v[2 * j + 1]);
#pragma unroll
        for (int j = 0; j < 7; ++j) od[j] = pack2<PREC>(v[2 * j + 1], v[2 * j + 2]);
        unsigned char *dst = dst0 + q * P.cp_lbo + i * 16;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            uint4 wv;
            if ((c & 1) == 0)
                wv = make_uint4(ev[c / 2], ev[c / 2 + 1], ev[c / 2 + 2], ev[c / 2 + 3]);
            else
                wv = make_uint4(od[c / 2], od[c / 2 + 1], od[c / 2 + 2], od[c / 2 + 3]);
            *reinterpret_cast<uint4 *>(dst + c * (TC_ROWS * 16)) = wv;
        }
    }
}

// ------------------------------------------------------------- epilogue --

// Window wx of a row whose accumulators start at TMEM column col0: a warp of
// lane quarter 0 forms the planes of slots 0..7, one of quarter 1 those of
// slot 8: the 16 columns of its lanes staged in eb, then the diagonal sums
// P_w(sy, sx) = sum_i D[(sx + R, i)][i + R - sy] into the window's plane.
static __device__ __forceinline__ void tc_epilogue_window(uint32_t tmem, int quarter, uint32_t col, float *eb,
                                                          float *pw)
{
    constexpr int R = TC_R, ND = 2 * R + 1;
    const int lane = threadIdx.x & 31;
    float r[16];
    tc_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + col, r);
    float4 *d4 = reinterpret_cast<float4 *>(eb + lane * TC_EB_PITCH);
    d4[0] = make_float4(r[0], r[1], r[2], r[3]);
    d4[1] = make_float4(r[4], r[5], r[6], r[7]);
    d4[2] = make_float4(r[8], r[9], r[10], r[11]);
    d4[3] = make_float4(r[12], r[13], r[14], r[15]);
    __syncwarp();
    const int nout = quarter == 0 ? 8 * ND : ND;  // slots 0..7, or slot 8
    for (int o = lane; o < nout; o += 32) {
        const int cl = o / ND, syi = o - cl * ND;  // slot 8 quarter + cl, sy = syi - R
        // lane 4 cl + i holds row i of the slot; its column for sy is i + R - sy
        const float *e = eb + (TC_ROWS * cl) * TC_EB_PITCH + (2 * R - syi);
        float s = e[0];
        s += e[TC_EB_PITCH + 1];
        s += e[2 * TC_EB_PITCH + 2];
        s += e[3 * TC_EB_PITCH + 3];
        pw[syi * ND + 8 * quarter + cl] = s;
    }
    __syncwarp();
}

// ------------------------------------------------- the tensor-core phase --

// Barriers of the phase (after the region load's barrier):
//   full[NS]      a producer warp filled a ring slot (group k is built by
//                 producer warp k mod TC_PRODUCERS, whole)
//   empty[NS]     the MMAs that read a slot completed (commit)
//   slab_full[2]  producer warps built a row's slab
//   row_done[2]   a row's MMAs completed (commit): its slab is free, its TMEM
//                 block ready for the epilogue
//   tmem_free[2]  the epilogue warps read a row's TMEM block (one arrival each)
constexpr int TC_PRODUCERS = 4;  // producer warps: 2, 5, 6, 7
constexpr int TC_EPI_WARPS = 3;  // epilogue warps: 0, 4 (lane quarter 0), 1 (quarter 1)
constexpr int TC_ISSUER = 3;     // warp of the MMA-issuing thread

__device__ __forceinline__ int tc_producer_index(int warp)
{
    return warp == 2 ? 0 : (warp >= 5 ? warp - 4 : -1);
}

template <int PREC, int GC>
static __device__ __forceinline__ void tc_phase(const PassArgs &a, const TileGeom &g, const float *As,
                                                const float *Bs, float *Ps, unsigned char *smem, uint32_t tmem,
                                                uint64_t *bars, float m, volatile int *abort)
{
    constexpr int R = TC_R, W = 2 * GC, NG = (W + 2 * R) / TC_ROWS, KS = W / 16, CPW = GC / 8;
    constexpr int NP = (2 * R + 1) * (2 * R + 1);
    static_assert((W + 2 * R) % TC_ROWS == 0 && GC % 8 == 0, "shape");
    const PassPlan &P = a.plan;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NS = P.tc_nbuf;
    uint64_t *full = bars, *empty = bars + NS, *slab_full = bars + 2 * NS, *row_done = slab_full + 2,
             *tmem_free = row_done + 2;
    unsigned char *slab = smem + P.off_slab;  // two slabs, slab_bytes apart
    unsigned char *ring = smem + P.off_cp;
    const int slab_bytes = P.slab_lbo * (g.aw >> 3);
    const int tcols = 16 * P.TX;  // columns of one row's TMEM block
    const int pidx = tc_producer_index(warp);

    if (pidx >= 0) {
        // ---------------------------------------------------------- producers
        const int t = pidx * 32 + lane, nt = TC_PRODUCERS * 32;
        for (int wy = 0; wy < g.nwy; ++wy) {
            const int sb = wy & 1;
            if (wy >= 2 && !warp_wait(a, row_done + sb, ((wy >> 1) - 1) & 1, abort)) return;
            tc_slab<PREC>(P, g, As, slab + sb * slab_bytes, wy, m, t, nt);
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(slab_full + sb);
            for (int gi = 0; gi < NG; ++gi) {
                const int k = wy * NG + gi, slot = k % NS;
                if (k % TC_PRODUCERS != pidx) continue;
                if (k >= NS && !warp_wait(a, empty + slot, ((k / NS) - 1) & 1, abort)) return;
                tc_group<PREC>(P, g, Bs, ring + slot * P.cp_group, wy, gi, m, lane, 32);
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) mbar_arrive(full + slot);
            }
        }
    } else if (warp == TC_ISSUER) {
        // ------------------------------------------------------------- issuer
        const uint32_t idesc = tc_idesc<PREC>();
        const uint32_t slab_s = smem_addr(slab), ring_s = smem_addr(ring);
        uint64_t *last = nullptr;  // the barrier of the last commit, and its phase
        uint32_t last_par = 0;
        bool ok = true;
        for (int wy = 0; wy < g.nwy && ok; ++wy) {
            const int tb = wy & 1;
            if (wy >= 2 && !warp_wait(a, tmem_free + tb, ((wy >> 1) - 1) & 1, abort)) {
                ok = false;
                break;
            }
            if (!warp_wait(a, slab_full + tb, (wy >> 1) & 1, abort)) {
                ok = false;
                break;
            }
            for (int gi = 0; gi < NG; ++gi) {
                const int k = wy * NG + gi, slot = k % NS;
                if (!warp_wait(a, full + slot, (k / NS) & 1, abort)) {
                    ok = false;
                    break;
                }
                if (lane == 0) {
                    tc_fence_after();
                    // the start-address field is the low 14 bits, in units of 16 bytes
                    const uint64_t da0 = tc_desc(ring_s + slot * P.cp_group, P.cp_lbo, 128);
                    const uint64_t db0 = tc_desc(slab_s + tb * slab_bytes + TC_ROWS * gi * 16, P.slab_lbo, 128);
                    for (int wx = 0; wx < g.nwx; ++wx) {
#pragma unroll
                        for (int kk = 0; kk < KS; ++kk) {
                            const int chunk = wx * CPW + 2 * kk;
                            tc_mma(tmem + (uint32_t)(tb * tcols + 16 * wx), da0 + (uint64_t)((chunk * P.cp_lbo) >> 4),
                                   db0 + (uint64_t)((chunk * P.slab_lbo) >> 4), idesc, (gi | kk) != 0 ? 1u : 0u);
                        }
                    }
                    tc_commit(empty + slot);
                }
                last = empty + slot;
                last_par = (k / NS) & 1;
            }
            if (!ok) break;
            if (lane == 0) tc_commit(row_done + tb);
            last = row_done + tb;
            last_par = (wy >> 1) & 1;
        }
        if (!ok && last && lane == 0) {
            // drain: a bounded chance for the MMAs in flight before TMEM is freed
            const int lim = a.spin > 0 ? a.spin : MBAR_SPIN_LIMIT;
            for (int it = 0; it < lim; ++it)
                if (mbar_try_wait(last, last_par)) break;
        }
        __syncwarp();
    } else if (warp == 0 || warp == 1 || warp == 4) {
        // ----------------------------------------------------------- epilogue
        const int quarter = warp & 3;
        float *eb = reinterpret_cast<float *>(smem + P.off_ebuf) + (warp == 4 ? 2 : quarter) * 32 * TC_EB_PITCH;
        for (int wy = 0; wy < g.nwy; ++wy) {
            const int tb = wy & 1;
            if (!warp_wait(a, row_done + tb, (wy >> 1) & 1, abort)) return;
            tc_fence_after();
            // quarter 0: warps 0 and 4 take alternate windows; quarter 1: warp 1 all
            const int wx0 = warp == 4 ? 1 : 0, dwx = quarter == 0 ? 2 : 1;
            for (int wx = wx0; wx < g.nwx; wx += dwx)
                tc_epilogue_window(tmem, quarter, (uint32_t)(tb * tcols + 16 * wx), eb,
                                   Ps + (wy * g.nwx + wx) * NP);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tmem_free + tb);
        }
    }
}

// ------------------------------------------------- FP32 refit planes --

// Block planes of the FP32 refit: Q_b(s) = sum over block b of A(x) B'(x + s)
// for |sy|, |sx| <= TC_RN (the stencil of every peak within one pixel of the
// predictor), from the FP32 regions staged for radius R.  Each thread owns one
// (block, sy, row group) and keeps the 2 TC_RN + 1 sx accumulators in
// registers (as block_planes_fp32), RG row groups summed by shuffles.
static __device__ __forceinline__ void tc_refit_planes(const PassArgs &a, const TileGeom &g, const float *As,
                                                       const float *Bs, float *Qs)
{
    constexpr int RN = TC_RN, ND = 2 * RN + 1;
    constexpr int MIS = ((-RN) % 4 + 4) % 4;
    constexpr int NQ = (4 + 2 * RN + MIS + 3) / 4;
    const PassPlan &P = a.plan;
    const int G = g.G, RG = P.RGx, rows = G / RG, lrg = __ffs(RG) - 1;
    const int units = g.nb * ND;  // (block, sy)
    const int lane = threadIdx.x & 31, gi = lane >> (5 - lrg), ul = lane & ((32 >> lrg) - 1);
    // B' row of A row y at shift sy: smem row y + sy + R + 1, with sy = syi - RN
    const int row_off = g.R + 1 - RN;
    for (int base = (threadIdx.x - lane) >> lrg; base < units; base += blockDim.x >> lrg) {
        const int u = min(base + ul, units - 1);
        const int b = u / ND, syi = u - b * ND;
        const int byi = b / g.nbx, bxi = b - byi * g.nbx;
        const int c0 = bxi * G, r0 = byi * G + gi * rows;
        float acc[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) acc[d] = 0.f;
        for (int y = r0; y < r0 + rows; ++y) {
            const float *arow = As + y * P.a_pitch;
            const float *brow = Bs + (y + syi + row_off) * P.b_pitch + P.padl - RN - MIS;
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
        sum_row_groups<ND>(acc, lrg);
        if (base + ul < units && gi == 0) {
            float *out = Qs + b * ND * ND + syi * ND;
#pragma unroll
            for (int d = 0; d < ND; ++d) out[d] = acc[d];
        }
    }
}

// One warp per window: the scaled coefficient from the window's tensor-core
// plane in offset form, (P - (mu_A - m)(S1 - n m)) / sqrt(E_B), which equals
// the numerator sum (A - mu_A) B' of the definition; argmax with ties to the
// smallest row-major index.  A peak within one pixel of the predictor takes
// its five stencil values from the FP32 refit planes (the window's four
// blocks); the others go to the direct FP32 sums.
static __device__ __forceinline__ void tc_plane_and_peak(const PassArgs &a, const TileGeom &g, const float *Ps,
                                                         const float *Qs, const float *Vs, const float *stats,
                                                         float m, const WinShared &ws)
{
    constexpr int R = TC_R, ND = 2 * R + 1, NP = ND * ND, NQ = (NP + 31) / 32;
    constexpr int RN = TC_RN, NDN = 2 * RN + 1;
    constexpr uint32_t NONE = 0xffffffffu;
    const PassPlan &P = a.plan;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const float n = (float)(g.w * g.w), tau = TAU_PER_PIXEL * n, nm = n * m;
    const int cp = P.v_pitch;
    const float2 *VV = reinterpret_cast<const float2 *>(Vs);
    int qv[NQ], vv[NQ];
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
        const int q = min(lane + 32 * j, NP - 1);
        const int qy = q / ND, qx = q - qy * ND;
        qv[j] = q;
        vv[j] = (qy - R) * cp + (qx - R);
    }
    for (int wi = warp; wi < g.nwin; wi += nwarps) {
        const int wyi = wi / g.nwx, wxi = wi - wyi * g.nwx;
        const float muA = stats[2 * wi], EA = stats[2 * wi + 1];
        if (!(EA > tau)) {
            if (lane == 0) {
                ws.peaks[wi] = NP / 2;
                ws.need[wi] = 0;
            }
            continue;
        }
        const float dmu = muA - m;
        const float *pw = Ps + wi * NP;
        const float2 *vb = VV + (wyi * g.s + R + 1) * cp + wxi * g.s + R + 1;
        float best = 0.f;
        uint32_t bq = NONE;
#pragma unroll
        for (int j = 0; j < NQ; ++j) {
            if (j < NQ - 1 || lane + 32 * j < NP) {
                const float2 bx = vb[vv[j]];
                const float c = (pw[qv[j]] - dmu * (bx.x - nm)) * bx.y + 0.f;
                // ascending q: the first of equal values stays; NaN never wins
                if (c > best || (bq == NONE && c == c)) {
                    best = c;
                    bq = (uint32_t)qv[j];
                }
            }
        }
        const uint32_t key = bq == NONE ? 0u : ord_key(best);
        const uint32_t kmax = __reduce_max_sync(0xffffffffu, key);
        const uint32_t qmin = __reduce_min_sync(0xffffffffu, (key == kmax && bq != NONE) ? bq : NONE);
        const int bidx = qmin < (uint32_t)NP ? (int)qmin : NP / 2;  // no finite value: zero shift
        const int ky = bidx / ND - R, kx = bidx % ND - R;
        const bool near = ky >= 1 - RN && ky <= RN - 1 && kx >= 1 - RN && kx <= RN - 1;
        if (near && lane < 5) {
            int sy, sx;
            stencil_shift(lane, ky, kx, sy, sx);
            // blocks (wyi + yy, wxi + xx) of the window (50 % overlap: 2 x 2 blocks)
            const float *q0 = Qs + (wyi * g.nbx + wxi) * NDN * NDN + (sy + RN) * NDN + (sx + RN);
            const int rs = g.nbx * NDN * NDN;
            float num = q0[0];
            num += q0[NDN * NDN];
            num += q0[rs];
            num += q0[rs + NDN * NDN];
            const int vo = sy * cp + sx;
            ws.c5[wi * 5 + lane] = scaled_zncc(num, muA, vb[vo].x, vb[vo].y);
        }
        if (lane == 0) {
            ws.peaks[wi] = bidx;
            ws.need[wi] = near ? 0 : 0x1f;
        }
    }
}

// ------------------------------------------------------------- the kernel --

// Tiles of TX x TY windows of 50 % overlap (w = 2 GC, s = GC), r = 4: regions,
// FP32 statistics and box sums as in pass_kernel, the FP32 refit planes, the
// tensor-core phase, argmax on the planes, the refit, the Gaussian fit.
template <int PREC, int GC>
__global__ void __launch_bounds__(PASS_THREADS, 2) tc_pass_kernel(const __grid_constant__ PassArgs a)
{
    constexpr int R = TC_R;
    extern __shared__ __align__(16) unsigned char smem[];
    const PassPlan &P = a.plan;
    TileGeom g;
    g.R = R;
    g.ND = 2 * R + 1;
    g.NP = g.ND * g.ND;
    g.G = GC;
    g.w = 2 * GC;
    g.s = GC;
    g.kb = 2;
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
    g.BC = g.aw + 2 * (R + 1);
    g.BR = g.ah + 2 * (R + 1);
    g.OFFB = P.padl - (R + 1);
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
    float *Qs = reinterpret_cast<float *>(smem + P.off_refit);  // FP32 refit planes
    float *stats = reinterpret_cast<float *>(smem + P.off_stats);
    float2 *bst = reinterpret_cast<float2 *>(smem + P.off_gst);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + P.off_red);  // [0]: regions, then the phase's
    const int nbars = 2 * P.tc_nbuf + 6;
    // after the barriers: the TMEM address, the tile offset and the abort flag
    // (no static shared memory, so that the full dynamic carve-out can be granted)
    uint32_t &tmem_slot = *reinterpret_cast<uint32_t *>(bar + 1 + nbars);
    float &tile_off = *(reinterpret_cast<float *>(bar + 1 + nbars) + 1);
    volatile int *abort = reinterpret_cast<volatile int *>(bar + 2 + nbars);
    WinShared ws;
    ws.c5 = reinterpret_cast<float *>(smem + P.off_c5);
    ws.peaks = reinterpret_cast<int *>(smem + P.off_peaks);
    ws.need = reinterpret_cast<int *>(smem + P.off_need);
    ws.dpart = reinterpret_cast<float *>(smem + P.off_dpart);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // 1: A and B' regions
    const bool loaded = load_regions(a, g, pair, As, Bs, bar);
    if (__syncthreads_or(!loaded)) {
        invalid_tile(a, g, pair);
        return;
    }
    if (warp == 0) tc_alloc(&tmem_slot, P.tmem_cols);
    if (threadIdx.x == 32) {
        const int NS = P.tc_nbuf;
        for (int b = 0; b < NS; ++b) {
            mbar_init(bar + 1 + b, 1);              // full (one producer warp)
            mbar_init(bar + 1 + NS + b, 1);         // empty (commit)
        }
        mbar_init(bar + 1 + 2 * NS, TC_PRODUCERS);  // slab_full
        mbar_init(bar + 2 + 2 * NS, TC_PRODUCERS);
        mbar_init(bar + 3 + 2 * NS, 1);             // row_done (commit)
        mbar_init(bar + 4 + 2 * NS, 1);
        mbar_init(bar + 5 + 2 * NS, TC_EPI_WARPS);  // tmem_free
        mbar_init(bar + 6 + 2 * NS, TC_EPI_WARPS);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }

    // 2: A window statistics, box sums of B' for every window and shift
    block_stats(a, g, As, bst);
    box_sums(a, g, Bs, Cs, Vs);  // contains a barrier between its two passes
    __syncthreads();
    window_stats(a, g, bst, stats);
    if (warp == 0) {
        // tile offset: the mean of the A region, from the block sums in a fixed order
        float sum = 0.f;
        for (int b = lane; b < g.nb; b += 32) sum += bst[b].x;
        sum = warp_sum(sum);
        if (lane == 0) tile_off = sum / (float)(g.aw * g.ah);
    }
    // 3: FP32 refit planes (their buffer is not reused by the tensor-core phase)
    tc_refit_planes(a, g, As, Bs, Qs);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const float m = tile_off;

    // 4: tensor-core planes (operand buffers over the dead column box sums)
    if (a.dbg_stall == 2 && warp == TC_ISSUER) {
        // test hook: wait on a phase of the first slot's barrier that nothing
        // completes, before any MMA is issued
        warp_wait(a, bar + 1 + P.tc_nbuf, 0u, abort);
    }
    tc_phase<PREC, GC>(a, g, As, Bs, Ps, smem, tmem, bar + 1, m, abort);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tc_dealloc(tmem, P.tmem_cols);
    if (*abort) {
        invalid_tile(a, g, pair);
        return;
    }

    // 5: argmax on the planes, FP32 five-point refit, Gaussian fit, outputs
    tc_plane_and_peak(a, g, Ps, Qs, Vs, stats, m, ws);
    __syncthreads();
    stencil_direct(a, g, As, Bs, ws);
    __syncthreads();
    finalize(a, g, Vs, stats, ws, pair);
}

}  // namespace rpiv
