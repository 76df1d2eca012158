/*
 * FP64 CPU oracle of the PIV correction path (RapidPIV, arXiv 2504.17987).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously-correct loops in double
 * precision.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline may load it; the product path never does.  It shares no code,
 * header, table or constant with the CUDA implementation.
 *
 * Each stage follows the method's description (Sec. 2 of the paper, "RapidPIV"):
 * the image pair is warped by the current displacement estimate, a
 * correlation-coefficient stencil is evaluated around the chosen peak, a
 * three-point Gaussian fit gives the sub-pixel correction, the universal
 * outlier detector (normalised median test, threshold 2, regulariser 0.1 px,
 * Sec. 3.1) flags and replaces outliers by the median of their valid
 * neighbours, and vorticity is derived from the final field.  Readings of
 * points the paper leaves open (search range, deformation form, borders,
 * tie-breaks, degenerate windows, pyramid) are stated beside each function.
 *
 * Conventions: images are row-major double arrays I[y*W + x]; pixel centres at
 * integer (x, y); x = column, y = row (downwards).  A vector grid of window w
 * and step s has nx = floor((W - w)/s) + 1 nodes per row, node i at
 * x = i*s + (w-1)/2, window i covering columns [i*s, i*s + w).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* degenerate-energy threshold, per pixel of the window (intensity units^2) */
#define ORC_TAU_PER_PIXEL 1e-6

int orc_grid_n(int extent, int w, int s)
{
    if (w < 1 || s < 1 || extent < w) return 0;
    return (extent - w) / s + 1;
}

/* ------------------------------------------------------------ sampling --- */

static double pix_clamped(const double *I, int W, int H, long x, long y)
{
    if (x < 0) x = 0;
    if (x > W - 1) x = W - 1;
    if (y < 0) y = 0;
    if (y > H - 1) y = H - 1;
    return I[(size_t)y * W + x];
}

/* Bilinear interpolation of image I at real position (X, Y), clamp-to-edge. */
double orc_bilinear(const double *I, int W, int H, double X, double Y)
{
    double fx = floor(X), fy = floor(Y);
    long x0 = (long)fx, y0 = (long)fy;
    double tx = X - fx, ty = Y - fy;
    double i00 = pix_clamped(I, W, H, x0, y0);
    double i10 = pix_clamped(I, W, H, x0 + 1, y0);
    double i01 = pix_clamped(I, W, H, x0, y0 + 1);
    double i11 = pix_clamped(I, W, H, x0 + 1, y0 + 1);
    return (1 - tx) * (1 - ty) * i00 + tx * (1 - ty) * i10 + (1 - tx) * ty * i01 + tx * ty * i11;
}

/* Gradient (d/dX, d/dY) of the bilinear interpolant inside the cell chosen by
 * floor(X), floor(Y) (clamp-to-edge: a clamped direction has zero slope). */
static void bilinear_grad(const double *I, int W, int H, double X, double Y, double *gx, double *gy)
{
    double fx = floor(X), fy = floor(Y);
    long x0 = (long)fx, y0 = (long)fy;
    double tx = X - fx, ty = Y - fy;
    double i00 = pix_clamped(I, W, H, x0, y0);
    double i10 = pix_clamped(I, W, H, x0 + 1, y0);
    double i01 = pix_clamped(I, W, H, x0, y0 + 1);
    double i11 = pix_clamped(I, W, H, x0 + 1, y0 + 1);
    *gx = (1 - ty) * (i10 - i00) + ty * (i11 - i01);
    *gy = (1 - tx) * (i01 - i00) + tx * (i11 - i10);
}

/*
 * Position of a point along one grid axis: node index i0, the next node i1 and
 * weight t of i1, so that value = (1-t) g[i0] + t g[i1].  Outside the node
 * hull the field is extended by the border value (reading: constant
 * extrapolation; the paper does not say).
 */
static void axis_weights(double pos, int n, int w, int s, int *i0, int *i1, double *t)
{
    double f = (pos - 0.5 * (w - 1)) / s;
    if (n <= 1) { *i0 = 0; *i1 = 0; *t = 0.0; return; }
    if (f < 0) f = 0;
    if (f > n - 1) f = n - 1;
    int a = (int)floor(f);
    if (a > n - 2) a = n - 2;
    *i0 = a;
    *i1 = a + 1;
    *t = f - a;
}

/* Bilinear value of the grid field (gu, gv) at image position (x, y). */
void orc_field_at(const double *gu, const double *gv, int nx, int ny, int w, int s,
                  double x, double y, double *du, double *dv)
{
    int i0, i1, j0, j1;
    double tx, ty;
    axis_weights(x, nx, w, s, &i0, &i1, &tx);
    axis_weights(y, ny, w, s, &j0, &j1, &ty);
    double w00 = (1 - tx) * (1 - ty), w10 = tx * (1 - ty), w01 = (1 - tx) * ty, w11 = tx * ty;
    *du = w00 * gu[j0 * nx + i0] + w10 * gu[j0 * nx + i1] + w01 * gu[j1 * nx + i0] + w11 * gu[j1 * nx + i1];
    *dv = w00 * gv[j0 * nx + i0] + w10 * gv[j0 * nx + i1] + w01 * gv[j1 * nx + i0] + w11 * gv[j1 * nx + i1];
}

/*
 * Deformed image over the image grown by M pixels on every side:
 * out[(y+M)*(W+2M) + (x+M)] for x in [-M, W+M), y in [-M, H+M).
 *   mode 0 (frame B only):  out = B(x + d(x))
 *   mode 1 (central):       out = B(x + d(x)/2)   (frame A is warped by -d/2
 *                                                   with orc_deform_ext too)
 * sign = +1 or -1 selects the direction; scale multiplies d.
 */
void orc_deform_ext(const double *img, int W, int H, const double *gu, const double *gv,
                    int nx, int ny, int w, int s, int M, double scale, double *out)
{
    const int WE = W + 2 * M, HE = H + 2 * M;
    for (int yy = 0; yy < HE; ++yy) {
        for (int xx = 0; xx < WE; ++xx) {
            double x = xx - M, y = yy - M, du, dv;
            orc_field_at(gu, gv, nx, ny, w, s, x, y, &du, &dv);
            out[(size_t)yy * WE + xx] = orc_bilinear(img, W, H, x + scale * du, y + scale * dv);
        }
    }
}

/* Same growth by M pixels for an undeformed image (edge-clamped copy). */
void orc_pad_ext(const double *img, int W, int H, int M, double *out)
{
    const int WE = W + 2 * M, HE = H + 2 * M;
    for (int yy = 0; yy < HE; ++yy)
        for (int xx = 0; xx < WE; ++xx)
            out[(size_t)yy * WE + xx] = pix_clamped(img, W, H, xx - M, yy - M);
}

/* --------------------------------------------------------- correlation --- */

/*
 * Zero-normalised correlation coefficient between the window of A at
 * (x0, y0) and the window of B' displaced by (sx, sy):
 *     C = sum a~ b~ / sqrt(E_A E_B),  a~ = A - mean, b~ = B' - mean (per shift).
 * Windows whose energy E_A or E_B is at most tau = 1e-6 * w^2 are degenerate:
 * C = 0 (reading: the paper gives no rule).  Images are the grown arrays of
 * orc_deform_ext / orc_pad_ext with margin M.  *num_out (nullable) receives
 * the raw numerator sum a~ * B' (equal to sum a~ b~ since a~ sums to zero).
 */
double orc_zncc(const double *Aext, const double *Bext, int W, int M, int x0, int y0, int w,
                int sx, int sy, double *num_out)
{
    const int WE = W + 2 * M;
    const double n = (double)w * w;
    double sa = 0, sb = 0;
    for (int y = 0; y < w; ++y)
        for (int x = 0; x < w; ++x) {
            sa += Aext[(size_t)(y0 + y + M) * WE + (x0 + x + M)];
            sb += Bext[(size_t)(y0 + y + sy + M) * WE + (x0 + x + sx + M)];
        }
    double ma = sa / n, mb = sb / n;
    double ea = 0, eb = 0, num = 0, raw = 0;
    for (int y = 0; y < w; ++y)
        for (int x = 0; x < w; ++x) {
            double a = Aext[(size_t)(y0 + y + M) * WE + (x0 + x + M)] - ma;
            double bv = Bext[(size_t)(y0 + y + sy + M) * WE + (x0 + x + sx + M)];
            double b = bv - mb;
            ea += a * a;
            eb += b * b;
            num += a * b;
            raw += a * bv;
        }
    if (num_out) *num_out = raw;
    const double tau = ORC_TAU_PER_PIXEL * n;
    if (ea <= tau || eb <= tau) return 0.0;
    return num / sqrt(ea * eb);
}

/* Energy of the A window (sum of squared deviations from its mean). */
static double window_energy(const double *Aext, int W, int M, int x0, int y0, int w)
{
    const int WE = W + 2 * M;
    double s = 0;
    for (int y = 0; y < w; ++y)
        for (int x = 0; x < w; ++x) s += Aext[(size_t)(y0 + y + M) * WE + (x0 + x + M)];
    double m = s / ((double)w * w), e = 0;
    for (int y = 0; y < w; ++y)
        for (int x = 0; x < w; ++x) {
            double a = Aext[(size_t)(y0 + y + M) * WE + (x0 + x + M)] - m;
            e += a * a;
        }
    return e;
}

/*
 * Three-point Gaussian sub-pixel estimator through (c_minus, c0, c_plus) at
 * offsets -1, 0, +1 (Sec. 2: "Gaussian sub-pixel interpolation"):
 *     delta = (ln c- - ln c+) / (2 ln c- - 4 ln c0 + 2 ln c+).
 * Reading for undefined cases: if a value is not positive or the log
 * curvature is not negative, use the three-point parabola
 * (c- - c+)/(2c- - 4c0 + 2c+); if that curvature is not negative either,
 * delta = 0.  |delta| is clamped to 1.
 */
double orc_gauss3(double cm, double c0, double cp)
{
    double d;
    if (cm > 0 && c0 > 0 && cp > 0) {
        double lm = log(cm), l0 = log(c0), lp = log(cp);
        double den = 2 * lm - 4 * l0 + 2 * lp;
        if (den < 0) {
            d = (lm - lp) / den;
            goto clamp;
        }
    }
    {
        double den = 2 * cm - 4 * c0 + 2 * cp;
        if (den < 0) {
            d = (cm - cp) / den;
            goto clamp;
        }
    }
    return 0.0;
clamp:
    if (d > 1) d = 1;
    if (d < -1) d = -1;
    return d;
}

/*
 * One correlation pass over every window of a grid.
 *   Aext, Bext : grown (margin M >= r + 1) frame A (or A') and deformed B'.
 *   pu, pv     : predictor at the nodes of this grid (the deformation field).
 *   r          : search radius; the plane covers shifts [-r, r]^2 (r = 0 is the
 *                paper's fixed stencil centred at zero shift).
 *   force_peaks: nullable (2 ints per window: ky, kx); if given, the integer
 *                peak is taken from it instead of the argmax.
 * Per window outputs: u, v, integer peak (ky, kx), sub-pixel (dy, dx), the
 * five stencil values c5 = {C(k), C(k - ex), C(k + ex), C(k - ey), C(k + ey)},
 * valid (0 if the A window is degenerate; then u, v = predictor), and, when
 * plane is non-null, the (2r+1)^2 plane in row-major (sy, sx) order.
 * Argmax reading: strict '>' scanning sy then sx from -r, so ties keep the
 * smallest row-major index.
 */
void orc_pass(const double *Aext, const double *Bext, int W, int H, int M, int w, int s, int r,
              const double *pu, const double *pv, const int *force_peaks, const unsigned char *only,
              double *u, double *v, int *peaks, double *sub, double *c5, int *valid, double *plane)
{
    const int nx = orc_grid_n(W, w, s), ny = orc_grid_n(H, w, s);
    const int np = 2 * r + 1;
    const double tau = ORC_TAU_PER_PIXEL * (double)w * w;
    double *pl = (double *)malloc(sizeof(double) * np * np);
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            const int k = j * nx + i;
            const int x0 = i * s, y0 = j * s;
            if (only && !only[k]) {
                /* window not requested (sampled evaluation of large grids) */
                u[k] = v[k] = NAN;
                valid[k] = -1;
                continue;
            }
            for (int sy = -r; sy <= r; ++sy)
                for (int sx = -r; sx <= r; ++sx)
                    pl[(sy + r) * np + (sx + r)] = orc_zncc(Aext, Bext, W, M, x0, y0, w, sx, sy, NULL);
            if (plane) memcpy(plane + (size_t)k * np * np, pl, sizeof(double) * np * np);
            double ea = window_energy(Aext, W, M, x0, y0, w);
            if (!(ea > tau)) {
                u[k] = pu[k];
                v[k] = pv[k];
                peaks[2 * k] = 0;
                peaks[2 * k + 1] = 0;
                sub[2 * k] = 0;
                sub[2 * k + 1] = 0;
                for (int q = 0; q < 5; ++q) c5[5 * k + q] = 0;
                valid[k] = 0;
                continue;
            }
            int ky, kx;
            if (force_peaks) {
                ky = force_peaks[2 * k];
                kx = force_peaks[2 * k + 1];
            } else {
                int best = 0;
                for (int q = 1; q < np * np; ++q)
                    if (pl[q] > pl[best]) best = q;
                ky = best / np - r;
                kx = best % np - r;
            }
            double c0 = orc_zncc(Aext, Bext, W, M, x0, y0, w, kx, ky, NULL);
            double cxm = orc_zncc(Aext, Bext, W, M, x0, y0, w, kx - 1, ky, NULL);
            double cxp = orc_zncc(Aext, Bext, W, M, x0, y0, w, kx + 1, ky, NULL);
            double cym = orc_zncc(Aext, Bext, W, M, x0, y0, w, kx, ky - 1, NULL);
            double cyp = orc_zncc(Aext, Bext, W, M, x0, y0, w, kx, ky + 1, NULL);
            double dx = orc_gauss3(cxm, c0, cxp);
            double dy = orc_gauss3(cym, c0, cyp);
            peaks[2 * k] = ky;
            peaks[2 * k + 1] = kx;
            sub[2 * k] = dy;
            sub[2 * k + 1] = dx;
            c5[5 * k + 0] = c0;
            c5[5 * k + 1] = cxm;
            c5[5 * k + 2] = cxp;
            c5[5 * k + 3] = cym;
            c5[5 * k + 4] = cyp;
            u[k] = pu[k] + kx + dx;
            v[k] = pv[k] + ky + dy;
            valid[k] = 1;
        }
    }
    free(pl);
}

/* ---------------------------------------------------------- validation --- */

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Median of n values (n >= 1); even n gives the mean of the two middle ones. */
double orc_median(const double *vals, int n)
{
    double tmp[16];
    memcpy(tmp, vals, sizeof(double) * n);
    qsort(tmp, n, sizeof(double), cmp_double);
    if (n % 2) return tmp[n / 2];
    return 0.5 * (tmp[n / 2 - 1] + tmp[n / 2]);
}

/*
 * Universal outlier detector (normalised median test, Westerweel & Scarano
 * 2005, as used in Sec. 2 with threshold 2 and regulariser 0.1 px, Sec. 3.1).
 * For each node and each component, over the existing 3x3 neighbours
 * (excluding the node; 8 inside, 5 on edges, 3 in corners):
 *     um = median(neighbours), rm = median(|u_i - um|),
 *     r0 = |u0 - um| / (rm + eps);
 * the vector is an outlier if r0 > thr for either component, or if its window
 * was invalid.  Outliers are replaced by the component-wise median of their
 * non-outlier neighbours (one iteration; detection uses all neighbours); with
 * no such neighbour the value is kept.  mask = 1 passed, 0 flagged.
 * replace = 0 only flags.
 */
void orc_uod(const double *u, const double *v, const int *valid, int nx, int ny, double thr,
             double eps, int replace, double *uo, double *vo, unsigned char *mask)
{
    const int N = nx * ny;
    unsigned char *out = (unsigned char *)malloc((size_t)(N > 0 ? N : 1));
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const int k = j * nx + i;
            double nu[8], nv[8];
            int c = 0;
            for (int dj = -1; dj <= 1; ++dj)
                for (int di = -1; di <= 1; ++di) {
                    if (!di && !dj) continue;
                    int ii = i + di, jj = j + dj;
                    if (ii < 0 || jj < 0 || ii >= nx || jj >= ny) continue;
                    nu[c] = u[jj * nx + ii];
                    nv[c] = v[jj * nx + ii];
                    ++c;
                }
            int bad = valid ? !valid[k] : 0;
            if (c > 0) {
                double res[8];
                double um = orc_median(nu, c);
                for (int q = 0; q < c; ++q) res[q] = fabs(nu[q] - um);
                double rmu = orc_median(res, c);
                double vm = orc_median(nv, c);
                for (int q = 0; q < c; ++q) res[q] = fabs(nv[q] - vm);
                double rmv = orc_median(res, c);
                double r0u = fabs(u[k] - um) / (rmu + eps);
                double r0v = fabs(v[k] - vm) / (rmv + eps);
                if (r0u > thr || r0v > thr) bad = 1;
            }
            out[k] = (unsigned char)bad;
        }
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const int k = j * nx + i;
            uo[k] = u[k];
            vo[k] = v[k];
            mask[k] = out[k] ? 0 : 1;
            if (!out[k] || !replace) continue;
            double nu[8], nv[8];
            int c = 0;
            for (int dj = -1; dj <= 1; ++dj)
                for (int di = -1; di <= 1; ++di) {
                    if (!di && !dj) continue;
                    int ii = i + di, jj = j + dj;
                    if (ii < 0 || jj < 0 || ii >= nx || jj >= ny) continue;
                    if (out[jj * nx + ii]) continue;
                    nu[c] = u[jj * nx + ii];
                    nv[c] = v[jj * nx + ii];
                    ++c;
                }
            if (c > 0) {
                uo[k] = orc_median(nu, c);
                vo[k] = orc_median(nv, c);
            }
        }
    free(out);
}

/* ---------------------------------------------------- grid-to-grid map --- */

/*
 * Bilinear interpolation of a source grid field onto the nodes of a
 * destination grid (pass-to-pass predictor, and the pyramid's upsampling).
 * The source lives levels_up pyramid levels above the destination (0 = same
 * image); a destination position X maps to (X + 0.5)/2^L - 0.5 on the source
 * image (pixel k of a level covers pixels 2k, 2k+1 of the level below) and
 * the value is multiplied by 2^L.
 */
void orc_interp_grid(const double *su, const double *sv, int snx, int sny, int sw, int ss,
                     int dnx, int dny, int dw, int ds, int levels_up, double *du, double *dv)
{
    const double f = ldexp(1.0, levels_up);
    for (int j = 0; j < dny; ++j)
        for (int i = 0; i < dnx; ++i) {
            double X = i * ds + 0.5 * (dw - 1), Y = j * ds + 0.5 * (dw - 1);
            double xs = (X + 0.5) / f - 0.5, ys = (Y + 0.5) / f - 0.5;
            double a, b;
            orc_field_at(su, sv, snx, sny, sw, ss, xs, ys, &a, &b);
            du[j * dnx + i] = f * a;
            dv[j * dnx + i] = f * b;
        }
}

/* -------------------------------------------------------------- pyramid --- */

/* 2x2 box average: dst is floor(W/2) x floor(H/2); an odd last row/column is dropped. */
void orc_downsample(const double *src, int W, int H, double *dst)
{
    const int W2 = W / 2, H2 = H / 2;
    for (int y = 0; y < H2; ++y)
        for (int x = 0; x < W2; ++x)
            dst[(size_t)y * W2 + x] = 0.25 * (src[(size_t)(2 * y) * W + 2 * x] + src[(size_t)(2 * y) * W + 2 * x + 1] +
                                              src[(size_t)(2 * y + 1) * W + 2 * x] +
                                              src[(size_t)(2 * y + 1) * W + 2 * x + 1]);
}

/* ------------------------------------------------------------ vorticity --- */

/*
 * omega = dv/dx - du/dy on the grid (image axes, x = column, y = row down),
 * 1/frame: central differences over 2s inside, one-sided over s on the
 * border rows/columns, zero along an axis with a single node.
 */
void orc_vorticity(const double *u, const double *v, int nx, int ny, int s, double *w)
{
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double dvdx = 0, dudy = 0;
            if (nx > 1) {
                if (i == 0) dvdx = (v[j * nx + 1] - v[j * nx]) / s;
                else if (i == nx - 1) dvdx = (v[j * nx + i] - v[j * nx + i - 1]) / s;
                else dvdx = (v[j * nx + i + 1] - v[j * nx + i - 1]) / (2.0 * s);
            }
            if (ny > 1) {
                if (j == 0) dudy = (u[nx + i] - u[i]) / s;
                else if (j == ny - 1) dudy = (u[j * nx + i] - u[(j - 1) * nx + i]) / s;
                else dudy = (u[(j + 1) * nx + i] - u[(j - 1) * nx + i]) / (2.0 * s);
            }
            w[j * nx + i] = dvdx - dudy;
        }
}

/* ------------------------------------------------- score and its adjoint --- */

/*
 * Score S = sum over windows of the zero-shift correlation coefficient C_w(0)
 * between A and B deformed by the grid field (gu, gv) (frame-B-only
 * deformation), and, when gu_out/gv_out are non-null, dS/d(gu, gv):
 *   dC/dB'(x)  = a~(x)/sqrt(E_A E_B) - C b~(x)/E_B
 *   dB'(x)/dd  = gradient of the bilinear interpolant of B at x + d(x)
 *                (in-cell derivative, cell chosen by floor)
 *   dd(x)/dd_k = bilinear weight of node k at x (constant extrapolation).
 * Degenerate windows contribute 0 to S and to the gradient.
 */
double orc_score_grad(const double *A, const double *B, int W, int H, int w, int s,
                      const double *gu, const double *gv, double *gu_out, double *gv_out)
{
    const int nx = orc_grid_n(W, w, s), ny = orc_grid_n(H, w, s);
    const double n = (double)w * w, tau = ORC_TAU_PER_PIXEL * n;
    double *bp = (double *)malloc(sizeof(double) * w * w);
    double *gxb = (double *)malloc(sizeof(double) * w * w);
    double *gyb = (double *)malloc(sizeof(double) * w * w);
    if (gu_out) memset(gu_out, 0, sizeof(double) * nx * ny);
    if (gv_out) memset(gv_out, 0, sizeof(double) * nx * ny);
    double S = 0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const int x0 = i * s, y0 = j * s;
            double sa = 0, sb = 0;
            for (int y = 0; y < w; ++y)
                for (int x = 0; x < w; ++x) {
                    double px = x0 + x, py = y0 + y, du, dv;
                    orc_field_at(gu, gv, nx, ny, w, s, px, py, &du, &dv);
                    double b = orc_bilinear(B, W, H, px + du, py + dv);
                    bp[y * w + x] = b;
                    if (gu_out || gv_out) bilinear_grad(B, W, H, px + du, py + dv, &gxb[y * w + x], &gyb[y * w + x]);
                    sa += A[(size_t)(y0 + y) * W + x0 + x];
                    sb += b;
                }
            double ma = sa / n, mb = sb / n, ea = 0, eb = 0, num = 0;
            for (int y = 0; y < w; ++y)
                for (int x = 0; x < w; ++x) {
                    double a = A[(size_t)(y0 + y) * W + x0 + x] - ma, b = bp[y * w + x] - mb;
                    ea += a * a;
                    eb += b * b;
                    num += a * b;
                }
            if (ea <= tau || eb <= tau) continue;
            double rs = 1.0 / sqrt(ea * eb);
            double C = num * rs;
            S += C;
            if (!gu_out && !gv_out) continue;
            for (int y = 0; y < w; ++y)
                for (int x = 0; x < w; ++x) {
                    double a = A[(size_t)(y0 + y) * W + x0 + x] - ma, b = bp[y * w + x] - mb;
                    double g = a * rs - C * b / eb;
                    double gx = g * gxb[y * w + x], gy = g * gyb[y * w + x];
                    int i0, i1, j0, j1;
                    double tx, ty;
                    axis_weights(x0 + x, nx, w, s, &i0, &i1, &tx);
                    axis_weights(y0 + y, ny, w, s, &j0, &j1, &ty);
                    double w00 = (1 - tx) * (1 - ty), w10 = tx * (1 - ty), w01 = (1 - tx) * ty, w11 = tx * ty;
                    if (gu_out) {
                        gu_out[j0 * nx + i0] += w00 * gx;
                        gu_out[j0 * nx + i1] += w10 * gx;
                        gu_out[j1 * nx + i0] += w01 * gx;
                        gu_out[j1 * nx + i1] += w11 * gx;
                    }
                    if (gv_out) {
                        gv_out[j0 * nx + i0] += w00 * gy;
                        gv_out[j0 * nx + i1] += w10 * gy;
                        gv_out[j1 * nx + i0] += w01 * gy;
                        gv_out[j1 * nx + i1] += w11 * gy;
                    }
                }
        }
    free(bp);
    free(gxb);
    free(gyb);
    return S;
}

/* ------------------------------------------------------- pre-processing --- */
/*
 * The pre-processing before the flow estimate (Sec. 2): a high-pass filter
 * against the static background, then contrast-limited adaptive histogram
 * equalisation (CLAHE, Zuiderveld 1994).  Readings (the paper gives no
 * parameters):
 *   high-pass   d(x) = max(0, n I(x) - S(x)), S the sum of I over the
 *               (2 hp + 1)^2 box around x with clamp-to-edge, n its pixel
 *               count; the filtered value is d / n (I minus its box mean,
 *               negative values cut at zero).  hp = 0 disables it (d / n = I).
 *   CLAHE       tiles tx x ty of ceil(W / tx) x ceil(H / ty) pixels (the last
 *               row and column of tiles may be smaller); 256 bins over
 *               [0, vmax + 1): bin = floor(d * 256 / (n (vmax + 1)));
 *               per tile of N pixels the histogram is clipped at
 *               L = max(1, floor(clip_pct N / (100 * 256))), the clipped
 *               excess E is spread as E / 256 to every bin plus one to the
 *               first E mod 256 bins; map[b] = cdf[b] * vmax / N.
 *               A pixel takes the bilinear blend of the maps of the four
 *               tiles whose centres surround it (centres at t * tw +
 *               (width_t - 1) / 2; clamped to the outer centres).
 *               clip_pct = 0 disables CLAHE (output d / n).
 * Every integer is computed exactly (64-bit), so the bins are the kernel's.
 */
static long long clamp_ll(long long v, long long lo, long long hi) { return v < lo ? lo : (v > hi ? hi : v); }

void orc_preprocess(const double *I, int W, int H, int vmax, int hp, int tx, int ty, int clip_pct, double *out)
{
    const long long n = (long long)(2 * hp + 1) * (2 * hp + 1);
    long long *d = (long long *)malloc(sizeof(long long) * (size_t)W * H);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            long long S = 0;
            for (int dy = -hp; dy <= hp; ++dy)
                for (int dx = -hp; dx <= hp; ++dx)
                    S += (long long)I[clamp_ll(y + dy, 0, H - 1) * W + clamp_ll(x + dx, 0, W - 1)];
            long long v = hp > 0 ? n * (long long)I[(size_t)y * W + x] - S : (long long)I[(size_t)y * W + x];
            d[(size_t)y * W + x] = v > 0 ? v : 0;
        }
    if (clip_pct <= 0) {
        for (size_t i = 0; i < (size_t)W * H; ++i) out[i] = (double)d[i] / (double)n;
        free(d);
        return;
    }
    const int nb = 256;
    const int tw = (W + tx - 1) / tx, th = (H + ty - 1) / ty;
    double *map = (double *)malloc(sizeof(double) * (size_t)tx * ty * nb);
    const long long den = n * ((long long)vmax + 1);
    for (int j = 0; j < ty; ++j)
        for (int i = 0; i < tx; ++i) {
            long long h[256] = {0};
            const int x0 = i * tw, x1 = (x0 + tw < W) ? x0 + tw : W;
            const int y0 = j * th, y1 = (y0 + th < H) ? y0 + th : H;
            long long N = 0;
            for (int y = y0; y < y1; ++y)
                for (int x = x0; x < x1; ++x) {
                    long long b = d[(size_t)y * W + x] * nb / den;
                    if (b > nb - 1) b = nb - 1;
                    h[b]++;
                    N++;
                }
            long long L = (long long)clip_pct * N / (100LL * nb);
            if (L < 1) L = 1;
            long long E = 0;
            for (int b = 0; b < nb; ++b)
                if (h[b] > L) {
                    E += h[b] - L;
                    h[b] = L;
                }
            long long c = 0;
            for (int b = 0; b < nb; ++b) {
                c += h[b] + E / nb + (b < E % nb ? 1 : 0);
                map[((size_t)j * tx + i) * nb + b] = N > 0 ? (double)c * vmax / (double)N : 0.0;
            }
        }
    for (int y = 0; y < H; ++y) {
        /* vertical tile pair and weight */
        int j0, j1;
        double wy;
        {
            const double cy0 = (th - 1) * 0.5;
            const int jl = ty - 1;
            const double cyl = jl * th + ((H - jl * th) - 1) * 0.5;
            if (ty == 1 || y <= cy0) { j0 = j1 = 0; wy = 0.0; }
            else if (y >= cyl) { j0 = j1 = jl; wy = 0.0; }
            else {
                j0 = (int)floor((y - cy0) / th);
                if (j0 > ty - 2) j0 = ty - 2;
                j1 = j0 + 1;
                const double c0 = j0 * th + (th - 1) * 0.5;
                const double c1 = (j1 == jl) ? cyl : j1 * th + (th - 1) * 0.5;
                wy = (y - c0) / (c1 - c0);
            }
        }
        for (int x = 0; x < W; ++x) {
            int i0, i1;
            double wx;
            const double cx0 = (tw - 1) * 0.5;
            const int il = tx - 1;
            const double cxl = il * tw + ((W - il * tw) - 1) * 0.5;
            if (tx == 1 || x <= cx0) { i0 = i1 = 0; wx = 0.0; }
            else if (x >= cxl) { i0 = i1 = il; wx = 0.0; }
            else {
                i0 = (int)floor((x - cx0) / tw);
                if (i0 > tx - 2) i0 = tx - 2;
                i1 = i0 + 1;
                const double c0 = i0 * tw + (tw - 1) * 0.5;
                const double c1 = (i1 == il) ? cxl : i1 * tw + (tw - 1) * 0.5;
                wx = (x - c0) / (c1 - c0);
            }
            long long b = d[(size_t)y * W + x] * nb / den;
            if (b > nb - 1) b = nb - 1;
            const double m00 = map[((size_t)j0 * tx + i0) * nb + b], m01 = map[((size_t)j0 * tx + i1) * nb + b];
            const double m10 = map[((size_t)j1 * tx + i0) * nb + b], m11 = map[((size_t)j1 * tx + i1) * nb + b];
            out[(size_t)y * W + x] = (1 - wy) * ((1 - wx) * m00 + wx * m01) + wy * ((1 - wx) * m10 + wx * m11);
        }
    }
    free(map);
    free(d);
}
