"""Pins of each oracle stage against facts fixed by mathematics, not by the oracle.

Every expected value below comes from a closed form, an independent library
routine (numpy FFT), a hand computation, or an invariant; none is produced by
re-running the oracle's own formula.
"""
import math

import numpy as np
import pytest

import oracle
from synth import workloads as wl


def _rng(seed):
    return np.random.default_rng(seed)


# --------------------------------------------------------------- sampling ---

def test_bilinear_is_exact_on_affine_images_and_clamps():
    H, W = 20, 30
    y, x = np.mgrid[0:H, 0:W]
    img = 2.5 * x - 1.25 * y + 7.0
    for X, Y in [(3.25, 4.5), (10.0, 11.0), (28.9, 0.1), (0.0, 18.999)]:
        assert oracle.bilinear(img, X, Y) == pytest.approx(2.5 * X - 1.25 * Y + 7.0, abs=1e-12)
    # clamp-to-edge: beyond the border the edge pixel's value continues
    assert oracle.bilinear(img, -3.0, 5.0) == pytest.approx(img[5, 0], abs=1e-12)
    assert oracle.bilinear(img, 40.0, 25.0) == pytest.approx(img[H - 1, W - 1], abs=1e-12)


def test_field_interpolation_affine_inside_constant_outside():
    w, s = 16, 8
    nx, ny = 6, 5
    xn = np.arange(nx) * s + 7.5
    yn = np.arange(ny) * s + 7.5
    Xn, Yn = np.meshgrid(xn, yn)
    gu = 0.1 * Xn + 0.02 * Yn - 1.0
    gv = -0.05 * Xn + 0.3
    for (x, y) in [(10.0, 12.3), (30.7, 20.0), (7.5, 7.5), (47.5, 39.5)]:
        du, dv = oracle.field_at(gu, gv, w, s, x, y)
        assert du == pytest.approx(0.1 * x + 0.02 * y - 1.0, abs=1e-12)
        assert dv == pytest.approx(-0.05 * x + 0.3, abs=1e-12)
    # outside the node hull the border value is extended (x below the first node)
    du, _ = oracle.field_at(gu, gv, w, s, 2.0, 20.0)
    assert du == pytest.approx(0.1 * 7.5 + 0.02 * 20.0 - 1.0, abs=1e-12)
    du, _ = oracle.field_at(gu, gv, w, s, 100.0, 100.0)
    assert du == pytest.approx(0.1 * xn[-1] + 0.02 * yn[-1] - 1.0, abs=1e-12)


def test_deform_integer_shift_is_exact_translation():
    img = _rng(1).uniform(0, 255, (40, 50))
    w, s = 16, 8
    nx, ny = oracle.grid_n(50, w, s), oracle.grid_n(40, w, s)
    gu = np.full((ny, nx), 3.0)
    gv = np.full((ny, nx), -2.0)
    M = 5
    out = oracle.deform_ext(img, gu, gv, w, s, M)
    # B'(x, y) = B(x + 3, y - 2) wherever the sample lies inside the image
    for (x, y) in [(0, 2), (10, 20), (46, 39), (20, 5)]:
        assert out[y + M, x + M] == img[y - 2, x + 3]


def test_deform_affine_image_affine_field_closed_form():
    H, W = 48, 64
    yy, xx = np.mgrid[0:H, 0:W]
    alpha, beta, gamma = 1.5, -0.75, 40.0
    img = alpha * xx + beta * yy + gamma
    w, s = 16, 8
    nx, ny = oracle.grid_n(W, w, s), oracle.grid_n(H, w, s)
    Xn, Yn = np.meshgrid(np.arange(nx) * s + 7.5, np.arange(ny) * s + 7.5)
    gu = 0.05 * Xn - 0.02 * Yn + 0.3
    gv = 0.01 * Xn + 0.04 * Yn - 0.7
    M = 2
    out = oracle.deform_ext(img, gu, gv, w, s, M)
    # inside the node hull, d is affine; the sample stays inside the image
    for (x, y) in [(10, 10), (30, 25), (50, 35), (8, 38)]:
        du = 0.05 * x - 0.02 * y + 0.3
        dv = 0.01 * x + 0.04 * y - 0.7
        assert out[y + M, x + M] == pytest.approx(alpha * (x + du) + beta * (y + dv) + gamma, abs=1e-10)


# ------------------------------------------------------------ correlation ---

def test_self_correlation_is_one_at_zero_shift_and_peaks_there():
    A = _rng(2).uniform(0, 255, (64, 64))
    M = 6
    Ae = oracle.pad_ext(A, M)
    c, _ = oracle.zncc(Ae, Ae, 64, M, 16, 16, 16, 0, 0)
    assert c == pytest.approx(1.0, abs=1e-12)
    z = np.zeros((oracle.grid_n(64, 16, 8),) * 2)
    res = oracle.correlate_pass(A, A, 16, 8, 4, z, z, want_plane=True)
    assert np.all(res.peaks == 0)
    assert np.all(np.abs(res.plane) <= 1.0 + 1e-12)


def test_anti_correlation_and_affine_invariance():
    A = _rng(3).uniform(0, 255, (40, 40))
    B = _rng(4).uniform(0, 255, (40, 40))
    M = 4
    Ae, Be = oracle.pad_ext(A, M), oracle.pad_ext(B, M)
    c, _ = oracle.zncc(Ae, oracle.pad_ext(-A, M), 40, M, 8, 8, 16, 0, 0)
    assert c == pytest.approx(-1.0, abs=1e-12)
    c1, _ = oracle.zncc(Ae, Be, 40, M, 8, 8, 16, 2, -1)
    c2, _ = oracle.zncc(Ae, oracle.pad_ext(2.5 * B + 7.0, M), 40, M, 8, 8, 16, 2, -1)
    assert c1 == pytest.approx(c2, abs=1e-12)
    assert abs(c1) <= 1.0


def test_numerator_equals_fft_linear_cross_correlation():
    # brute-force numerator sum a~(x) B(x + s) against a zero-padded FFT correlation
    rng = _rng(5)
    w, r = 8, 3
    A = rng.uniform(0, 100, (30, 30))
    B = rng.uniform(0, 100, (30, 30))
    M = r + 2
    Ae, Be = oracle.pad_ext(A, M), oracle.pad_ext(B, M)
    x0 = y0 = 10
    a = A[y0:y0 + w, x0:x0 + w]
    at = a - a.mean()
    region = B[y0 - r:y0 + w + r, x0 - r:x0 + w + r]
    # corr[s] = sum_x at[x] region[x + s + r]  ==  IFFT(conj(FFT(at)) * FFT(region))
    n = w + 2 * r + w
    Fa = np.fft.fft2(at, (n, n))
    Fb = np.fft.fft2(region, (n, n))
    full = np.real(np.fft.ifft2(np.conj(Fa) * Fb))
    for sy in range(-r, r + 1):
        for sx in range(-r, r + 1):
            _, num = oracle.zncc(Ae, Be, 30, M, x0, y0, w, sx, sy)
            assert num == pytest.approx(full[sy + r, sx + r], rel=1e-9, abs=1e-7)


def test_integer_circular_shift_found_exactly():
    A = _rng(6).uniform(0, 255, (96, 96))
    for dy, dx in [(3, -2), (-4, 4), (0, 1)]:
        B = np.roll(A, (dy, dx), axis=(0, 1))
        z = np.zeros((oracle.grid_n(96, 32, 16),) * 2)
        res = oracle.correlate_pass(A, B, 32, 16, 4, z, z)
        inner = (slice(1, -1), slice(1, -1))
        assert np.all(res.peaks[inner][..., 0] == dy) and np.all(res.peaks[inner][..., 1] == dx)
        assert np.allclose(res.c5[inner][..., 0], 1.0, atol=1e-12)


def test_argmax_tie_keeps_smallest_row_major_shift():
    # A window correlated with a B that repeats with period 2 along x: shifts
    # sx = -2, 0, 2 give identical planes; the first in row-major order wins.
    rng = _rng(7)
    base = rng.uniform(0, 255, (40, 2))
    A = np.tile(base, (1, 20))
    z = np.zeros((oracle.grid_n(40, 16, 8), oracle.grid_n(40, 16, 8)))
    res = oracle.correlate_pass(A, A, 16, 8, 2, z, z, want_plane=True)
    # windows of the first column see edge-clamped samples at sx = -2: no exact tie there
    inner = res.peaks[:, 1:]
    assert np.all(inner[..., 0] == 0)
    assert np.all(inner[..., 1] == -2)
    pl = res.plane[:, 1:]
    assert np.all(pl[..., 2, 0] == pl[..., 2, 2])  # the exact tie the rule decides


def test_degenerate_window_is_invalid_and_keeps_predictor():
    A = np.full((48, 48), 17.0)
    B = _rng(8).uniform(0, 255, (48, 48))
    n = oracle.grid_n(48, 16, 8)
    pu = np.full((n, n), 0.5)
    pv = np.full((n, n), -0.25)
    res = oracle.correlate_pass(A, B, 16, 8, 2, pu, pv)
    assert np.all(res.valid == 0)
    assert np.all(res.u == 0.5) and np.all(res.v == -0.25)


# --------------------------------------------------------------- sub-pixel ---

@pytest.mark.parametrize("sigma", [0.6, 1.0, 2.0])
@pytest.mark.parametrize("delta", [-0.45, -0.2, 0.0, 0.13, 0.37, 0.49])
def test_gauss3_recovers_sampled_gaussian_exactly(sigma, delta):
    c = [math.exp(-((k - delta) ** 2) / (2 * sigma * sigma)) * 0.83 for k in (-1, 0, 1)]
    assert oracle.gauss3(*c) == pytest.approx(delta, abs=1e-12)


def test_gauss3_parabola_fallback_and_clamp():
    # a value <= 0 forces the parabola, which is exact on a quadratic
    a, b, d = 0.5, 1.0, 0.3
    c = [a - b * (k - d) ** 2 for k in (-1, 0, 1)]
    assert c[0] <= 0
    assert oracle.gauss3(*c) == pytest.approx(d, abs=1e-12)
    # flat: no curvature, delta = 0
    assert oracle.gauss3(0.5, 0.5, 0.5) == 0.0
    # a Gaussian sampled 1.5 away from the centre sample is clamped to 1
    c = [math.exp(-((k - 1.5) ** 2) / 2.0) for k in (-1, 0, 1)]
    assert oracle.gauss3(*c) == 1.0


# ------------------------------------------------------------- validation ---

def test_median_even_and_odd():
    assert oracle.median([3.0, 1.0, 2.0]) == 2.0
    assert oracle.median([4.0, 1.0, 3.0, 2.0]) == 2.5


def test_uod_detects_and_replaces_a_spike_by_hand_median():
    i, j = np.meshgrid(np.arange(5), np.arange(5))
    u = 0.1 * i + 0.2 * j
    v = -0.05 * i
    u[2, 2] = 10.0
    uo, vo, mask = oracle.uod(u, v, thr=2.0, eps=0.1)
    expected_mask = np.ones((5, 5), np.uint8)
    expected_mask[2, 2] = 0
    assert np.array_equal(mask, expected_mask)
    # neighbours of (2,2) in u: 0.3 0.4 0.5 / 0.5 . 0.7 / 0.7 0.8 0.9 -> median (0.5+0.7)/2 = 0.6
    assert uo[2, 2] == pytest.approx(0.6, abs=1e-12)
    # v neighbours: -0.05,-0.10,-0.15 (x3 rows, minus centre) -> median -0.10
    assert vo[2, 2] == pytest.approx(-0.10, abs=1e-12)
    # everything else untouched
    keep = expected_mask.astype(bool)
    assert np.array_equal(uo[keep], u[keep])


def test_uod_corner_uses_three_neighbours_and_smooth_field_passes():
    i, j = np.meshgrid(np.arange(4), np.arange(4))
    u = 0.1 * i + 0.2 * j
    v = np.zeros((4, 4))
    u[0, 0] = 50.0
    uo, _, mask = oracle.uod(u, v)
    expected = np.ones((4, 4), np.uint8)
    expected[0, 0] = 0
    assert np.array_equal(mask, expected)
    assert uo[0, 0] == pytest.approx(0.2, abs=1e-12)  # median of {0.1, 0.2, 0.3}
    i, j = np.meshgrid(np.arange(9), np.arange(7))
    _, _, m2 = oracle.uod(0.3 * i - 0.1 * j, 0.05 * j, thr=2.0, eps=0.1)
    assert m2.all()


def test_uod_invalid_flag_forces_replacement_and_no_valid_neighbour_keeps():
    u = 0.01 * np.arange(9.0).reshape(3, 3)
    v = np.zeros((3, 3))
    valid = np.ones((3, 3), np.int32)
    valid[1, 1] = 0
    uo, _, mask = oracle.uod(u, v, valid)
    # median of 0.00..0.08 without 0.04 -> (0.03 + 0.05)/2
    assert mask.sum() == 8 and mask[1, 1] == 0 and uo[1, 1] == pytest.approx(0.04, abs=1e-12)
    valid[:] = 0
    uo, _, mask = oracle.uod(u, v, valid)
    assert not mask.any() and np.array_equal(uo, u)


# ------------------------------------------------------------ grid / pyramid ---

def test_interp_grid_affine_and_level_map():
    sw, ss = 32, 16
    snx, sny = 7, 5
    Xs, Ys = np.meshgrid(np.arange(snx) * ss + 15.5, np.arange(sny) * ss + 15.5)
    su = 0.02 * Xs + 0.01 * Ys + 1.0
    sv = -0.03 * Xs + 2.0
    # same level: destination nodes inside the source hull get the affine value
    dw, ds, dnx, dny = 16, 8, 13, 9
    du, dv = oracle.interp_grid(su, sv, sw, ss, dnx, dny, dw, ds, 0)
    Xd, Yd = np.meshgrid(np.arange(dnx) * ds + 7.5, np.arange(dny) * ds + 7.5)
    inside = (Xd >= 15.5) & (Xd <= 15.5 + 6 * 16) & (Yd >= 15.5) & (Yd <= 15.5 + 4 * 16)
    assert np.allclose(du[inside], (0.02 * Xd + 0.01 * Yd + 1.0)[inside], atol=1e-12)
    # one level up: X_src = (X - 0.5)/2 and the value doubles
    du1, dv1 = oracle.interp_grid(su, sv, sw, ss, dnx, dny, dw, ds, 1)
    Xs1, Ys1 = (Xd - 0.5) / 2, (Yd - 0.5) / 2
    ins1 = (Xs1 >= 15.5) & (Xs1 <= 111.5) & (Ys1 >= 15.5) & (Ys1 <= 79.5)
    assert ins1.any()
    assert np.allclose(dv1[ins1], (2 * (-0.03 * Xs1 + 2.0))[ins1], atol=1e-12)


def test_downsample_affine_and_odd_sizes():
    H, W = 21, 34
    y, x = np.mgrid[0:H, 0:W]
    img = 3.0 * x + 5.0 * y + 1.0
    d = oracle.downsample(img)
    assert d.shape == (10, 17)
    yy, xx = np.mgrid[0:10, 0:17]
    assert np.allclose(d, 3.0 * (2 * xx + 0.5) + 5.0 * (2 * yy + 0.5) + 1.0, atol=1e-12)
    assert np.all(oracle.downsample(np.full((8, 8), 42.0)) == 42.0)


# -------------------------------------------------------------- vorticity ---

def test_vorticity_solid_body_rotation_is_two_omega():
    s = 8
    X, Y = np.meshgrid(np.arange(11) * s + 7.5, np.arange(9) * s + 7.5)
    Om = 0.013
    om = oracle.vorticity(-Om * Y, Om * X, s)
    assert np.allclose(om, 2 * Om, atol=1e-15)


def test_vorticity_lamb_oseen_within_truncation_bound():
    import synth
    s = 8
    xc, yc, G, rc = 100.3, 96.7, 200.0, 20.0
    X, Y = np.meshgrid(np.arange(26) * s + 7.5, np.arange(25) * s + 7.5)
    f = synth.Flow(vortices=[(xc, yc, G, rc)])
    u, v = f.eval(X, Y)
    om = oracle.vorticity(u, v, s)
    ref = synth.lamb_oseen_vorticity(X, Y, xc, yc, G, rc)
    # central-difference truncation: |err| <= s^2/6 (max|d3v/dx3| + max|d3u/dy3|)
    h = 0.5
    gx = np.arange(0, 220, h)
    GX, GY = np.meshgrid(gx, gx)
    uu, vv = f.eval(GX, GY)
    d3v = np.diff(vv, 3, axis=1) / h ** 3
    d3u = np.diff(uu, 3, axis=0) / h ** 3
    bound = s * s / 6.0 * (np.max(np.abs(d3v)) + np.max(np.abs(d3u))) * 1.05
    inner = (slice(1, -1), slice(1, -1))
    assert np.max(np.abs(om[inner] - ref[inner])) <= bound
    # and the bound is not vacuous: the peak vorticity is captured to 15 %
    k = np.unravel_index(np.argmax(ref), ref.shape)
    assert abs(om[k] - ref[k]) < 0.15 * ref[k]


def test_sampled_window_evaluation_equals_the_full_pass():
    # the `only` mask selects windows; it changes no arithmetic
    w = wl.plain_256(seed=77)
    A, B = w.render()
    nx = oracle.grid_n(256, 32, 16)
    rng = np.random.default_rng(5)
    pu, pv = rng.uniform(2.5, 4.0, (nx, nx)), rng.uniform(-2.0, -1.0, (nx, nx))
    full = oracle.correlate_pass(A, B, 32, 16, 4, pu, pv, want_plane=True)
    m = rng.random((nx, nx)) < 0.3
    part = oracle.correlate_pass(A, B, 32, 16, 4, pu, pv, want_plane=True, only=m)
    assert np.array_equal(part.u[m], full.u[m]) and np.array_equal(part.v[m], full.v[m])
    assert np.array_equal(part.peaks[m], full.peaks[m]) and np.array_equal(part.plane[m], full.plane[m])
    assert np.all(part.valid[~m] == -1) and np.all(np.isnan(part.u[~m]))


def test_ema_special_cases_and_closed_form():
    rng = np.random.default_rng(12)
    x, s0 = rng.standard_normal(50), rng.standard_normal(50)
    assert np.array_equal(oracle.ema(x, s0, 1.0), x)
    assert np.array_equal(oracle.ema(x, s0, 0.0), s0)
    assert np.array_equal(oracle.ema(x, s0, 0.3, init=True), x)
    # a constant input: s_k = x + (1 - a)^k (s_0 - x)
    a, s = 0.35, s0.copy()
    for k in range(1, 9):
        s = oracle.ema(x, s, a)
        assert np.allclose(s, x + (1 - a) ** k * (s0 - x), rtol=0, atol=1e-12)
    # step response from zero: 1 - (1 - a)^k
    s = np.zeros(1)
    for k in range(1, 6):
        s = oracle.ema(np.ones(1), s, a)
    assert abs(s[0] - (1 - (1 - a) ** 5)) <= 1e-15


def _clahe_constant_closed_form(N, vmax, clip_pct):
    L = max(1, clip_pct * N // (100 * 256))
    E = N - L
    c0 = L + E // 256 + (1 if E % 256 > 0 else 0)
    return c0 * vmax / N


@pytest.mark.parametrize("W,H,tiles,clip", [(16, 16, (2, 2), 200), (40, 24, (4, 3), 300), (64, 64, (1, 1), 50000)])
def test_preprocess_constant_image_closed_form(W, H, tiles, clip):
    img = np.full((H, W), 1234.0)
    out = oracle.preprocess(img, 4095, hp=3, tiles=tiles, clip_pct=clip)
    # the high-pass leaves zero everywhere: every pixel falls in bin 0 of every tile
    tw, th = -(-W // tiles[0]), -(-H // tiles[1])
    for j in range(tiles[1]):
        for i in range(tiles[0]):
            N = (min(W, (i + 1) * tw) - i * tw) * (min(H, (j + 1) * th) - j * th)
            cy = j * th + (min(H, (j + 1) * th) - j * th - 1) // 2
            cx = i * tw + (min(W, (i + 1) * tw) - i * tw - 1) // 2
            if (min(W, (i + 1) * tw) - i * tw) % 2 == 1 and (min(H, (j + 1) * th) - j * th) % 2 == 1:
                # at a tile's own centre only its map contributes
                assert abs(out[cy, cx] - _clahe_constant_closed_form(N, 4095, clip)) <= 1e-12


def test_preprocess_highpass_removes_affine_background_and_identity():
    H, W = 40, 48
    Y, X = np.mgrid[0:H, 0:W]
    ramp = 30.0 + 2.0 * X + 3.0 * Y
    out = oracle.preprocess(ramp, 4095, hp=4, tiles=(1, 1), clip_pct=0)
    # the box mean of an affine image is its centre value: zero away from the borders
    assert np.all(out[4:-4, 4:-4] == 0.0)
    # hp = 0 and no CLAHE: the identity
    rng = np.random.default_rng(8)
    img = rng.integers(0, 4096, (H, W)).astype(np.float64)
    assert np.array_equal(oracle.preprocess(img, 4095, hp=0, tiles=(1, 1), clip_pct=0), img)


def test_preprocess_uniform_histogram_is_equalised_globally():
    # one tile, a clip limit above every count: plain histogram equalisation
    vmax = 255
    vals = np.repeat(np.arange(256, dtype=np.float64), 16).reshape(64, 64)
    out = oracle.preprocess(vals, vmax, hp=0, tiles=(1, 1), clip_pct=10 ** 6)
    # 16 pixels per bin: cdf(b) = 16 (b + 1), map = cdf vmax / N
    assert np.allclose(out, (vals + 1) / 256.0 * vmax, rtol=0, atol=1e-12)


def test_preprocess_tile_maps_blend_bilinearly_between_centres():
    # two tiles side by side with different constant content: pixels at the
    # centres take their own tile's map, halfway between them the mean
    W, H = 32, 9
    img = np.zeros((H, W))
    img[:, 16:] = 200.0
    rng = np.random.default_rng(3)
    img += rng.integers(0, 2, (H, W))  # two levels per tile
    out = oracle.preprocess(img, 255, hp=0, tiles=(2, 1), clip_pct=10 ** 6)
    left = oracle.preprocess(img[:, :16], 255, hp=0, tiles=(1, 1), clip_pct=10 ** 6)
    right = oracle.preprocess(img[:, 16:], 255, hp=0, tiles=(1, 1), clip_pct=10 ** 6)
    # centres at x = 7.5 and 23.5 (even widths): x <= 7.5 uses the left map alone
    assert np.allclose(out[:, :8], left[:, :8], atol=1e-12)
    assert np.allclose(out[:, 24:], right[:, 8:], atol=1e-12)
