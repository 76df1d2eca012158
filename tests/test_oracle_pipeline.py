"""End-to-end pins of the oracle pipeline against imposed, known displacements."""
import json
import os

import numpy as np
import pytest

import oracle
from synth import workloads as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _nodes(n, w, s):
    return np.arange(n) * s + 0.5 * (w - 1)


@pytest.mark.parametrize("U,V", [(3.3, -1.7), (0.25, 0.5), (-7.6, 2.1)])
def test_uniform_shift_recovered_within_0p02_px(U, V):
    w = wl.uniform_shift(U, V)
    A, B = w.render()
    sc = w.schedule
    r = oracle.process_pair(A, B, sc.windows, sc.overlaps, sc.radii, sc.levels)
    assert r.mask.all()
    assert abs(np.mean(r.u) - U) <= 0.02 and abs(np.mean(r.v) - V) <= 0.02
    assert np.sqrt(np.mean((r.u - U) ** 2)) <= 0.03 and np.sqrt(np.mean((r.v - V) ** 2)) <= 0.03


def test_zero_displacement_noise_floor():
    w = wl.uniform_shift(0.0, 0.0, seed=2002)
    A, B = w.render()
    r = oracle.process_pair(A, B, (32,), (0.5,), (8,))
    assert abs(np.mean(r.u)) < 0.02 and abs(np.mean(r.v)) < 0.02
    assert np.max(np.abs(r.u)) < 0.1 and np.max(np.abs(r.v)) < 0.1


def test_two_pass_deformation_on_half_integer_shift():
    # With a predictor whose fractional part is 0 or 1/2 the bilinear warp has
    # symmetric weights, so the deformed pass must land on the imposed shift.
    w = wl.uniform_shift(2.5, -1.5, seed=2003)
    A, B = w.render()
    r = oracle.process_pair(A, B, (32, 32), (0.5, 0.5), (8, 2))
    assert abs(np.mean(r.u) - 2.5) <= 0.02 and abs(np.mean(r.v) + 1.5) <= 0.02


def test_supplied_predictor_is_used():
    # The true uniform field supplied as predictor: the deformed pass only
    # refines, so every integer peak is zero.
    w = wl.uniform_shift(5.0, -3.0, seed=2004)
    A, B = w.render()
    nx = oracle.grid_n(256, 32, 16)
    pred = (np.full((nx, nx), 5.0), np.full((nx, nx), -3.0))
    r = oracle.process_pair(A, B, (32,), (0.5,), (2,), pred=pred)
    assert np.all(r.trace[0].raw.peaks == 0)
    assert abs(np.mean(r.u) - 5.0) < 0.02


def test_vortex_field_against_analytic_truth():
    w = wl.plain_256()
    A, B = w.render()
    sc = w.schedule
    r = oracle.process_pair(A, B, sc.windows, sc.overlaps, sc.radii, sc.levels)
    xs = _nodes(15, 32, 16)
    X, Y = np.meshgrid(xs, xs)
    tu, tv = w.flow.eval(X, Y)
    assert np.sqrt(np.mean((r.u - tu) ** 2 + (r.v - tv) ** 2)) < 0.1
    # vorticity sign and location: the strongest rotation is at the vortex
    k = np.unravel_index(np.argmax(r.vort), r.vort.shape)
    assert abs(xs[k[1]] - 127.5) <= 16 and abs(xs[k[0]] - 127.5) <= 16


@pytest.mark.slow
def test_pyramid_recovers_displacement_beyond_the_search_radius():
    # 12 px uniform motion with a +-4 search: only the coarse-to-fine predictor
    # can reach it (4 x 3 px at the coarsest level).
    w = wl.paper_1mp(W=512, H=512)
    A, B = w.render()
    sc = w.schedule
    r = oracle.process_pair(A, B, sc.windows, sc.overlaps, sc.radii, sc.levels)
    ny, nx = r.u.shape
    xs = _nodes(nx, 16, 8)
    X, Y = np.meshgrid(xs, xs)
    tu, tv = w.flow.eval(X, Y)
    err = np.hypot(r.u - tu, r.v - tv)
    assert np.median(err) < 0.15
    assert r.mask.mean() > 0.95
    # without the pyramid the same schedule fails (zero predictor, +-4 < 12 px)
    r0 = oracle.process_pair(A, B, sc.windows, sc.overlaps, sc.radii, 0)
    assert np.median(np.hypot(r0.u - tu, r0.v - tv)) > 1.0


def test_paper_grid_count_identity():
    # 18 M vectors/s at 1150 pairs/s implies ~15.7 k vectors per 1 MP pair,
    # matching the grid formula n = floor((W - w)/s) + 1 at 16 px / 50 %.
    g = json.load(open(os.path.join(GOLD, "paper_numbers.json")))
    w = g["window_px"]
    s = oracle.step_of(w, g["overlap"])
    n = oracle.grid_n(1024, w, s)
    assert n == 127
    per_pair = g["throughput_rtx4080"]["vectors_per_s"] / g["throughput_rtx4080"]["pairs_per_s_at_1MP"]
    assert abs(per_pair / (n * n) - 1.0) < 0.05


def test_central_deformation_mode_runs_and_recovers_shift():
    # central warp moves each frame by d/2: an odd integer shift puts both
    # frames at half-pixel positions, where the bilinear weights are symmetric
    w = wl.uniform_shift(3.0, -1.0, seed=2005)
    A, B = w.render()
    r = oracle.process_pair(A, B, (32, 32), (0.5, 0.5), (8, 2), deform="central")
    assert abs(np.mean(r.u) - 3.0) <= 0.02 and abs(np.mean(r.v) + 1.0) <= 0.02
