/*
 * Seeded synthetic PIV image-pair generator.
 *
 * This module only manufactures inputs: tracer-particle images and the
 * analytic displacement fields that move the particles between the two
 * exposures.  It holds none of the correlation method's arithmetic and is
 * shared, as an input source only, by the FP64 oracle tests and by the CUDA
 * path's tests and benchmark.
 *
 * Image model (stands in for the laboratory particle images of the paper's
 * Sec. 3 experiments, plate 0.01-0.02 particles/pixel, cylinder 0.002 ppp):
 *   - particle centres p uniform over the image grown by a margin on every side,
 *     count = ppp * (W + 2m) * (H + 2m);
 *   - frame A holds each particle at p - d(p)/2, frame B at p + d(p)/2, so the
 *     true displacement at the pair's mid-time position p is d(p);
 *   - profile I0 * exp(-8 rho^2 / dp^2) (dp = e^-2 diameter), integrated over
 *     each pixel's unit square with erf (separable in x and y);
 *   - optional out-of-plane loss: a fraction of the particles of A is absent
 *     from B and the same number of fresh particles appear only in B;
 *   - additive Gaussian noise of standard deviation noise_frac * full scale,
 *     then round-to-nearest and clip to [0, full scale].
 *
 * Random numbers: xoshiro256** seeded through splitmix64 (both from their
 * published definitions).  Independent streams (particle positions, particle
 * attributes, loss selection, noise) are derived by seeding separate
 * generators from splitmix64(seed ^ stream_tag); the noise of image row y uses
 * its own generator seeded from (seed, frame, y), so the result does not
 * depend on the number of threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- RNG --- */

static uint64_t splitmix64_next(uint64_t *x)
{
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s[4]; } xo256;

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static void xo_seed(xo256 *r, uint64_t seed)
{
    uint64_t x = seed;
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64_next(&x);
}

static uint64_t xo_next(xo256 *r)
{
    uint64_t *s = r->s;
    const uint64_t result = rotl64(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

/* uniform in [0, 1) with 53 random bits */
static double xo_unif(xo256 *r) { return (double)(xo_next(r) >> 11) * 0x1.0p-53; }

/* standard normal by the Box-Muller transform (one draw per call) */
static double xo_normal(xo256 *r)
{
    double u1 = xo_unif(r), u2 = xo_unif(r);
    if (u1 < 1e-300) u1 = 1e-300;
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925 * u2);
}

static uint64_t stream_seed(uint64_t seed, uint64_t tag, uint64_t sub)
{
    uint64_t x = seed ^ (tag * 0xD1B54A32D192ED03ULL) ^ (sub * 0x8CB92BA72F3D8DD7ULL);
    return splitmix64_next(&x);
}

/* --------------------------------------------------------------- flow --- */

#define SYNTH_MAX_VORTEX 8
#define SYNTH_MAX_MODES 16

typedef struct {
    double U, V;                      /* uniform displacement, px/frame        */
    int n_vortex;                     /* Lamb-Oseen vortices                   */
    double vx[SYNTH_MAX_VORTEX], vy[SYNTH_MAX_VORTEX];
    double gamma[SYNTH_MAX_VORTEX];   /* circulation, px^2/frame               */
    double rc[SYNTH_MAX_VORTEX];      /* core radius, px                       */
    double shear_dU;                  /* u += dU/2 * tanh((y - y0)/delta)      */
    double shear_y0, shear_delta;
    int n_modes;                      /* streamfunction Fourier modes          */
    double kx[SYNTH_MAX_MODES], ky[SYNTH_MAX_MODES];
    double amp[SYNTH_MAX_MODES], phase[SYNTH_MAX_MODES];
    double Lx, Ly;                    /* periods of the modes, px              */
} synth_flow;

/*
 * Displacement at image position (x, y): x = column, y = row (down).
 * Lamb-Oseen: u_theta(r) = Gamma/(2 pi r) (1 - exp(-r^2/rc^2)), with
 * (u, v) = u_theta * (-(y-yc), (x-xc)) / r, whose vorticity dv/dx - du/dy is
 * Gamma/(pi rc^2) exp(-r^2/rc^2).
 * Modes: psi = sum a sin(2 pi (kx x/Lx + ky y/Ly) + phase), u = dpsi/dy,
 * v = -dpsi/dx (divergence free).
 */
void synth_flow_eval(const synth_flow *f, long n, const double *x, const double *y,
                     double *u, double *v)
{
    const double two_pi = 6.283185307179586476925;
    for (long i = 0; i < n; ++i) {
        double uu = f->U, vv = f->V;
        for (int k = 0; k < f->n_vortex; ++k) {
            double dx = x[i] - f->vx[k], dy = y[i] - f->vy[k];
            double r2 = dx * dx + dy * dy;
            double q;
            if (r2 < 1e-24) {
                q = 0.0;
            } else {
                /* u_theta / r = Gamma (1 - e^{-r^2/rc^2}) / (2 pi r^2) */
                q = f->gamma[k] * (-expm1(-r2 / (f->rc[k] * f->rc[k]))) / (two_pi * r2);
            }
            uu += -q * dy;
            vv += q * dx;
        }
        if (f->shear_dU != 0.0) uu += 0.5 * f->shear_dU * tanh((y[i] - f->shear_y0) / f->shear_delta);
        for (int m = 0; m < f->n_modes; ++m) {
            double ph = two_pi * (f->kx[m] * x[i] / f->Lx + f->ky[m] * y[i] / f->Ly) + f->phase[m];
            double c = f->amp[m] * cos(ph);
            uu += c * two_pi * f->ky[m] / f->Ly;
            vv -= c * two_pi * f->kx[m] / f->Lx;
        }
        u[i] = uu;
        v[i] = vv;
    }
}

/* ------------------------------------------------------------- images --- */

typedef struct {
    int W, H;
    int bit_depth;       /* 8, 12 or 16 */
    double ppp;          /* particles per pixel */
    double dp_min, dp_max;  /* e^-2 diameter range, px (uniform) */
    double i0_min, i0_max;  /* peak intensity range in 8-bit units; scaled by (2^bits - 1)/255 */
    double noise_frac;   /* noise sigma as a fraction of full scale */
    double loss_frac;    /* fraction of particles replaced between frames */
    double margin;       /* border added around the image for particle centres, px */
    uint64_t seed;
} synth_params;

typedef struct { double x, y, dp, i0; } particle;

static void splat(double *img, int W, int H, double xc, double yc, double dp, double i0)
{
    /* pixel-integrated separable Gaussian: sigma = dp/4, erf argument scale 2*sqrt(2)/dp */
    const double k = 2.0 * 1.4142135623730951 / dp;
    const double norm = (dp / 4.0) * 1.2533141373155003; /* sigma * sqrt(pi/2) */
    int rad = (int)ceil(1.5 * dp) + 1;
    int x0 = (int)floor(xc) - rad, x1 = (int)floor(xc) + rad;
    int y0 = (int)floor(yc) - rad, y1 = (int)floor(yc) + rad;
    if (x1 < 0 || y1 < 0 || x0 > W - 1 || y0 > H - 1) return;
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    if (x1 > W - 1) x1 = W - 1;
    if (y1 > H - 1) y1 = H - 1;
    double ix[64], iy[64];
    int nxp = x1 - x0 + 1, nyp = y1 - y0 + 1;
    if (nxp > 64 || nyp > 64) return;
    for (int i = 0; i < nxp; ++i) {
        double a = (x0 + i - 0.5 - xc) * k, b = (x0 + i + 0.5 - xc) * k;
        ix[i] = norm * (erf(b) - erf(a));
    }
    for (int j = 0; j < nyp; ++j) {
        double a = (y0 + j - 0.5 - yc) * k, b = (y0 + j + 0.5 - yc) * k;
        iy[j] = norm * (erf(b) - erf(a));
    }
    for (int j = 0; j < nyp; ++j) {
        double *row = img + (size_t)(y0 + j) * W + x0;
        double s = i0 * iy[j];
        for (int i = 0; i < nxp; ++i) row[i] += s * ix[i];
    }
}

static void finish_frame(const synth_params *P, const double *acc, void *out, int frame)
{
    const double fs = (double)((1 << P->bit_depth) - 1);
    const double sigma = P->noise_frac * fs;
    const int W = P->W, H = P->H;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y) {
        xo256 r;
        xo_seed(&r, stream_seed(P->seed, 0x4E4F495345ULL + (uint64_t)frame, (uint64_t)y));
        for (int x = 0; x < W; ++x) {
            double val = acc[(size_t)y * W + x];
            if (sigma > 0.0) val += sigma * xo_normal(&r);
            double q = floor(val + 0.5);
            if (q < 0.0) q = 0.0;
            if (q > fs) q = fs;
            if (P->bit_depth <= 8)
                ((uint8_t *)out)[(size_t)y * W + x] = (uint8_t)q;
            else
                ((uint16_t *)out)[(size_t)y * W + x] = (uint16_t)q;
        }
    }
}

/*
 * Render one image pair.  img_a / img_b are W*H arrays of uint8 (bit_depth 8)
 * or uint16 (bit_depth 12 or 16), row-major without padding.
 * Returns the number of particles placed, or -1 on bad arguments.
 */
long synth_render_pair(const synth_params *P, const synth_flow *F, void *img_a, void *img_b)
{
    if (P->W < 1 || P->H < 1 || !(P->bit_depth == 8 || P->bit_depth == 12 || P->bit_depth == 16))
        return -1;
    const int W = P->W, H = P->H;
    const double m = P->margin;
    const double scale = (double)((1 << P->bit_depth) - 1) / 255.0;
    long n = (long)floor(P->ppp * (W + 2.0 * m) * (H + 2.0 * m) + 0.5);
    particle *pa = (particle *)malloc(sizeof(particle) * (size_t)(n > 0 ? n : 1));
    particle *pb = (particle *)malloc(sizeof(particle) * (size_t)(n > 0 ? n : 1));
    double *acc_a = (double *)calloc((size_t)W * H, sizeof(double));
    double *acc_b = (double *)calloc((size_t)W * H, sizeof(double));
    if (!pa || !pb || !acc_a || !acc_b) {
        free(pa); free(pb); free(acc_a); free(acc_b);
        return -1;
    }
    xo256 rpos, ratt, rloss;
    xo_seed(&rpos, stream_seed(P->seed, 0x504F53ULL, 0));
    xo_seed(&ratt, stream_seed(P->seed, 0x415454ULL, 0));
    xo_seed(&rloss, stream_seed(P->seed, 0x4C4F5353ULL, 0));
    for (long i = 0; i < n; ++i) {
        double px = -m + (W + 2.0 * m) * xo_unif(&rpos);
        double py = -m + (H + 2.0 * m) * xo_unif(&rpos);
        double dp = P->dp_min + (P->dp_max - P->dp_min) * xo_unif(&ratt);
        double i0 = (P->i0_min + (P->i0_max - P->i0_min) * xo_unif(&ratt)) * scale;
        double u, v;
        synth_flow_eval(F, 1, &px, &py, &u, &v);
        pa[i].x = px - 0.5 * u; pa[i].y = py - 0.5 * v; pa[i].dp = dp; pa[i].i0 = i0;
        pb[i].x = px + 0.5 * u; pb[i].y = py + 0.5 * v; pb[i].dp = dp; pb[i].i0 = i0;
    }
    /* out-of-plane loss: replace a fraction of B's particles by fresh ones */
    if (P->loss_frac > 0.0) {
        for (long i = 0; i < n; ++i) {
            if (xo_unif(&rloss) < P->loss_frac) {
                pb[i].x = -m + (W + 2.0 * m) * xo_unif(&rloss);
                pb[i].y = -m + (H + 2.0 * m) * xo_unif(&rloss);
                pb[i].dp = P->dp_min + (P->dp_max - P->dp_min) * xo_unif(&rloss);
                pb[i].i0 = (P->i0_min + (P->i0_max - P->i0_min) * xo_unif(&rloss)) * scale;
            }
        }
    }
    for (long i = 0; i < n; ++i) splat(acc_a, W, H, pa[i].x, pa[i].y, pa[i].dp, pa[i].i0);
    for (long i = 0; i < n; ++i) splat(acc_b, W, H, pb[i].x, pb[i].y, pb[i].dp, pb[i].i0);
    finish_frame(P, acc_a, img_a, 0);
    finish_frame(P, acc_b, img_b, 1);
    free(pa); free(pb); free(acc_a); free(acc_b);
    return n;
}

/* Uniform doubles from the generator, for seeded choices made on the host
 * (e.g. sample positions of a finite-difference check). */
void synth_uniform(uint64_t seed, long n, double *out)
{
    xo256 r;
    xo_seed(&r, stream_seed(seed, 0x554E4946ULL, 0));
    for (long i = 0; i < n; ++i) out[i] = xo_unif(&r);
}

/* Reference values for the generator's own tests: the first outputs of
 * splitmix64 and xoshiro256** from a given seed. */
void synth_rng_probe(uint64_t seed, int n, uint64_t *sm_out, uint64_t *xo_out)
{
    uint64_t x = seed;
    for (int i = 0; i < n; ++i) sm_out[i] = splitmix64_next(&x);
    xo256 r;
    xo_seed(&r, seed);
    for (int i = 0; i < n; ++i) xo_out[i] = xo_next(&r);
}
