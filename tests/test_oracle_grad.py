"""Pins of the oracle's analytic score gradient (finite differences, closed forms)."""
import numpy as np
import pytest

import oracle
import synth
from synth import workloads as wl


def _field_coords(nx, ny, w, s, gu, gv, W, H):
    """Sample coordinates x + d(x) of every pixel (for the kink-skip rule only)."""
    def axis(pos, n):
        f = (pos - 0.5 * (w - 1)) / s
        f = np.clip(f, 0, n - 1)
        i0 = np.minimum(np.floor(f).astype(int), max(n - 2, 0))
        t = f - i0 if n > 1 else np.zeros_like(f)
        i1 = np.minimum(i0 + 1, n - 1)
        return i0, i1, t
    i0, i1, tx = axis(np.arange(W, dtype=float), nx)
    j0, j1, ty = axis(np.arange(H, dtype=float), ny)
    def interp(g):
        top = (1 - tx)[None, :] * g[j0][:, i0] + tx[None, :] * g[j0][:, i1]
        bot = (1 - tx)[None, :] * g[j1][:, i0] + tx[None, :] * g[j1][:, i1]
        return (1 - ty)[:, None] * top + ty[:, None] * bot
    X = np.arange(W)[None, :] + interp(gu)
    Y = np.arange(H)[:, None] + interp(gv)
    return X, Y


def _setup(seed=3003, W=192, H=160):
    w = wl.diff_1mp()
    w.spec.W, w.spec.H, w.spec.seed = W, H, seed
    w.flow.vortices = [(0.5 * W, 0.5 * H, 200.0, 20.0)]
    A, B = w.render()
    ww, s = 32, 8
    nx, ny = oracle.grid_n(W, ww, s), oracle.grid_n(H, ww, s)
    X, Y = np.meshgrid(np.arange(nx) * s + 15.5, np.arange(ny) * s + 15.5)
    tu, tv = w.flow.eval(X, Y)
    # a field near, but not at, the truth, with non-trivial fractional parts
    rnd = synth.uniform(seed, 2 * nx * ny).reshape(2, ny, nx)
    gu = tu + 0.3 * (rnd[0] - 0.5)
    gv = tv + 0.3 * (rnd[1] - 0.5)
    return A.astype(float), B.astype(float), ww, s, gu, gv


def test_gradient_matches_central_differences_at_64_seeded_nodes():
    A, B, w, s, gu, gv = _setup()
    H, W = A.shape
    ny, nx = gu.shape
    S, Gu, Gv = oracle.score_grad(A, B, w, s, gu, gv)
    h = 1e-5
    X, Y = _field_coords(nx, ny, w, s, gu, gv, W, H)
    near_kink = (np.abs(X - np.round(X)) < 4 * h) | (np.abs(Y - np.round(Y)) < 4 * h)
    picks = synth.uniform(4242, 64)
    checked = 0
    for p in picks:
        k = int(p * nx * ny)
        j, i = divmod(k, nx)
        # skip a node if any pixel it influences samples within 4h of a pixel edge
        x0, x1 = max(0, int((i - 1) * s + 15.5)), min(W, int((i + 1) * s + 15.5) + 1)
        y0, y1 = max(0, int((j - 1) * s + 15.5)), min(H, int((j + 1) * s + 15.5) + 1)
        if near_kink[y0:y1, x0:x1].any():
            continue
        for comp, G in ((0, Gu), (1, Gv)):
            up = [gu.copy(), gv.copy()]
            dn = [gu.copy(), gv.copy()]
            up[comp][j, i] += h
            dn[comp][j, i] -= h
            fd = (oracle.score_grad(A, B, w, s, *up, grad=False) -
                  oracle.score_grad(A, B, w, s, *dn, grad=False)) / (2 * h)
            assert G[j, i] == pytest.approx(fd, rel=1e-5, abs=1e-7)
        checked += 1
    assert checked >= 40


def test_gradient_on_ramp_image_is_along_the_ramp():
    # B = alpha x + beta y + gamma: dB'/dd = (alpha, beta) everywhere inside,
    # so dS/du_k : dS/dv_k = alpha : beta at every node.
    H, W = 96, 112
    rng = np.random.default_rng(11)
    A = rng.uniform(0, 200, (H, W))
    yy, xx = np.mgrid[0:H, 0:W]
    alpha, beta = 1.7, -0.6
    B = alpha * xx + beta * yy + 300.0 + 0.0 * A
    w, s = 32, 16
    nx, ny = oracle.grid_n(W, w, s), oracle.grid_n(H, w, s)
    gu = np.full((ny, nx), 0.37)
    gv = np.full((ny, nx), -0.21)
    S, Gu, Gv = oracle.score_grad(A, B, w, s, gu, gv)
    # interior nodes: their bilinear support never reaches the clamped border pixels
    inner = (slice(1, -1), slice(1, -1))
    gu_i, gv_i = Gu[inner], Gv[inner]
    assert gu_i.size > 0 and np.all(np.abs(gv_i) > 1e-9)
    assert np.allclose(gu_i * beta, gv_i * alpha, rtol=1e-9, atol=1e-14)
    # and the score is smooth along the field: finite differences agree tightly
    h = 1e-3
    fd = (oracle.score_grad(A, B, w, s, gu + h, gv, grad=False) -
          oracle.score_grad(A, B, w, s, gu - h, gv, grad=False)) / (2 * h)
    assert np.sum(Gu) == pytest.approx(fd, rel=1e-7)


def test_uniform_perturbation_derivative_is_the_sum_of_node_gradients():
    A, B, w, s, gu, gv = _setup(seed=3004, W=160, H=128)
    S, Gu, Gv = oracle.score_grad(A, B, w, s, gu, gv)
    h = 1e-6
    fd = (oracle.score_grad(A, B, w, s, gu, gv + h, grad=False) -
          oracle.score_grad(A, B, w, s, gu, gv - h, grad=False)) / (2 * h)
    # a uniform shift moves every pixel: kinks may be crossed, so a looser bound
    assert np.sum(Gv) == pytest.approx(fd, rel=2e-2)


def test_refinement_rule_increases_the_score():
    A, B, w, s, gu, gv = _setup(seed=3005, W=128, H=128)
    u, v, hist = oracle.refine(A, B, w, s, gu, gv, steps=5)
    assert len(hist) == 6
    assert all(b >= a for a, b in zip(hist, hist[1:]))
    assert hist[-1] > hist[0]


def _quadratic(a, b):
    """S(u, v) = -(u - a)^2 - (v - b)^2 on a one-node field, with its gradient."""
    def f(u, v, grad=True):
        S = float(-np.sum((u - a) ** 2) - np.sum((v - b) ** 2))
        if not grad:
            return S
        return S, -2.0 * (u - a), -2.0 * (v - b)
    return f


def test_refinement_step_rule_follows_a_hand_computed_trace():
    # S = -(u - 1)^2 - (v - 0.5)^2 from (0, 0), eta0 = 3: g0 = (2, 1), max|g0| = 2.
    # k = 0: eta = 1.5 -> (3, 1.5), S = -5 < -1.25: halved; eta = 0.75 -> (1.5, 0.75), S = -0.3125, taken.
    # k = 1: g = (-1, -0.5), eta = 0.75 -> (0.75, 0.375), S = -0.078125, taken.
    # k = 2: g = (0.5, 0.25), eta = 0.375 -> (0.9375, 0.46875), S = -0.0048828125, taken.
    u, v, hist = oracle.ascend(_quadratic(1.0, 0.5), np.zeros((1, 1)), np.zeros((1, 1)), steps=3, eta0=3.0)
    assert hist == [-1.25, -0.3125, -0.078125, -0.0048828125]
    assert u[0, 0] == 0.9375 and v[0, 0] == 0.46875
    # a rule without the 0.5^k decay, or scaled by max|g_k| instead of max|g0|,
    # takes (1.5, 0.75) at k = 2 and ends at (1.125, 0.5625)


def test_refinement_keeps_the_field_when_every_halving_fails():
    # at the maximum the gradient is zero after the first step: S cannot increase,
    # all 1 + 3 tries fail and the field stays, the history repeats
    u, v, hist = oracle.ascend(_quadratic(1.0, 0.5), np.zeros((1, 1)), np.zeros((1, 1)), steps=3, eta0=2.0)
    # k = 0: eta = 1 -> (2, 1), S = -1.25 is not above -1.25: halved; eta = 0.5 -> (1, 0.5), S = 0, taken
    assert hist == [-1.25, 0.0, 0.0, 0.0]
    assert u[0, 0] == 1.0 and v[0, 0] == 0.5


def test_refinement_halves_at_most_three_times():
    # S = -(u - 1)^2, g0 = 2 at u = 0, eta0 = 40: the tries move u to 2 eta and
    # are taken only for 0 < eta < 1; eta runs 20, 10, 5, 2.5 (three halvings),
    # then 1.25 (a fourth) and 0.625 (a fifth, taken: u = 1.25, S = -0.0625)
    f = _quadratic(1.0, 0.0)
    z = np.zeros((1, 1))
    u, _, hist = oracle.ascend(f, z, z, steps=1, eta0=40.0)
    assert hist == [-1.0, -1.0] and u[0, 0] == 0.0
    u, _, hist = oracle.ascend(f, z, z, steps=1, eta0=40.0, halvings=4)
    assert hist == [-1.0, -1.0] and u[0, 0] == 0.0
    u, _, hist = oracle.ascend(f, z, z, steps=1, eta0=40.0, halvings=5)
    assert hist == [-1.0, -0.0625] and u[0, 0] == 1.25
