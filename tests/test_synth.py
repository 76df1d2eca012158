"""The seeded input generator: RNG definition, determinism, recipe statistics."""
import json
import os

import numpy as np
import pytest

import synth
from synth import workloads as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_sequence():
    ref = json.load(open(os.path.join(GOLD, "splitmix64.json")))
    sm, _ = synth.rng_probe(ref["seed"], len(ref["first_outputs"]))
    assert sm == ref["first_outputs"]


def test_render_deterministic_and_seed_sensitive():
    w = wl.plain_256()
    a1, b1 = w.render()
    a2, b2 = w.render()
    assert np.array_equal(a1, a2) and np.array_equal(b1, b2)
    w.spec.seed += 1
    a3, _ = w.render()
    assert not np.array_equal(a1, a3)


def test_recipe_statistics():
    # 12-bit recipe: full scale 4095, bright particles, background near the noise floor
    w = wl.paper_1mp()
    a, b = w.render()
    assert a.dtype == np.uint16 and a.shape == (1024, 1024)
    assert a.max() <= 4095
    # clip at zero plus sigma = 2 % of full scale: the median pixel is background
    assert 0 <= np.median(a) < 0.05 * 4095
    # 8-bit recipe
    w8 = wl.plain_256()
    a8, _ = w8.render()
    assert a8.dtype == np.uint8


def test_integer_shift_without_noise_is_an_exact_translation():
    # With no noise and an integer uniform displacement, B is A translated.
    spec = synth.ImageSpec(W=128, H=96, bit_depth=8, ppp=0.05, noise_frac=0.0, seed=77)
    a, b = synth.render_pair(spec, synth.Flow(U=4.0, V=-2.0))
    # B(x, y) = A(x - 4, y + 2)
    core_b = b[10:-10, 10:-10].astype(int)
    core_a = a[12:-8, 6:-14].astype(int)
    diff = np.abs(core_b - core_a)
    assert diff.max() <= 1 and np.mean(diff > 0) < 1e-3


def test_lamb_oseen_flow_matches_closed_form_vorticity():
    # the generator's vortex: finite-difference curl of its displacement vs closed form
    f = synth.Flow(vortices=[(50.0, 40.0, 200.0, 20.0)])
    h = 1e-4
    xs = np.array([50.0, 60.0, 71.3, 20.0])
    ys = np.array([40.0, 45.0, 30.2, 80.0])
    _, v1 = f.eval(xs + h, ys)
    _, v0 = f.eval(xs - h, ys)
    u1, _ = f.eval(xs, ys + h)
    u0, _ = f.eval(xs, ys - h)
    om = (v1 - v0) / (2 * h) - (u1 - u0) / (2 * h)
    ref = synth.lamb_oseen_vorticity(xs, ys, 50.0, 40.0, 200.0, 20.0)
    assert np.allclose(om, ref, rtol=1e-6, atol=1e-9)


def test_fourier_field_is_divergence_free_and_scaled():
    w = wl.fourier_8mp(W=384, H=216)
    f = w.flow
    h = 1e-3
    xs = np.linspace(10, 370, 7)
    ys = np.linspace(10, 200, 7)
    X, Y = np.meshgrid(xs, ys)
    u1, _ = f.eval(X + h, Y); u0, _ = f.eval(X - h, Y)
    _, v1 = f.eval(X, Y + h); _, v0 = f.eval(X, Y - h)
    div = (u1 - u0) / (2 * h) + (v1 - v0) / (2 * h)
    assert np.max(np.abs(div)) < 1e-6
    gx, gy = np.meshgrid(np.arange(0, 384, 4.0), np.arange(0, 216, 4.0))
    u, v = f.eval(gx, gy)
    assert abs(np.max(np.hypot(u, v)) - 16.0) < 1e-9
