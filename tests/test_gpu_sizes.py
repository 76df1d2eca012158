"""Parity at the ends of the image-size sweep (the paper's throughput-against-
size figure, Sec. 4.1, up to 8192 x 4096): full-size launches of the pass
kernels at 4096^2 and 8192 x 4096 on the 12-bit 1 MP recipe, compared with
the FP64 oracle on a seeded sample of windows (the oracle evaluates only the
sampled windows), at the FP32 bound and at the 16-bit bound (tolerances as
in test_gpu_parity.py, with the same fit-conditioning rule); and the whole
paper-shaped 16 px schedule at 8192 x 4096 against the analytic field and
across precisions, properties that hold at any size."""
import numpy as np
import pytest
import torch

import oracle
import paper_2504_17987_gb300 as rp
import synth
from fitcond import well_conditioned
from synth import workloads as wl

pytestmark = pytest.mark.gpu

TOL_PX = 1e-3
N_SAMPLE = 1200
SIZES = [(4096, 4096), (8192, 4096)]


@pytest.fixture(scope="module")
def pairs():
    from paper_2504_17987_gb300 import build
    build.build()
    oracle.build()
    out = {}
    for W, H in SIZES:
        wk = wl.paper_1mp(seed=1002, W=W, H=H)
        out[(W, H)] = (wk, *wk.render())
    return out


def _sample(nx, ny, n, seed):
    k = np.unique((synth.uniform(seed, n) * nx * ny).astype(np.int64))
    m = np.zeros(nx * ny, bool)
    m[k] = True
    m[[0, nx - 1, nx * (ny - 1), nx * ny - 1]] = True  # corners and the ragged last row / column
    m.reshape(ny, nx)[-1, ::11] = True
    m.reshape(ny, nx)[::11, -1] = True
    return m.reshape(ny, nx)


def _predictor(flow, nx, ny, w, s, seed):
    """The analytic field at the nodes plus a smooth +-0.4 px perturbation."""
    X, Y = np.meshgrid(np.arange(nx) * s + 0.5 * (w - 1), np.arange(ny) * s + 0.5 * (w - 1))
    tu, tv = flow.eval(X, Y)
    r = synth.uniform(seed, 4)
    pu = tu + 0.4 * np.sin(X / 173.0 + 6 * r[0]) * np.cos(Y / 151.0 + 6 * r[1])
    pv = tv + 0.4 * np.cos(X / 131.0 + 6 * r[2]) * np.sin(Y / 199.0 + 6 * r[3])
    return pu.astype(np.float32), pv.astype(np.float32)


@pytest.mark.parametrize("W,H", SIZES)
@pytest.mark.parametrize("w,s,R,precision", [(32, 16, 4, "fp32"), (16, 8, 1, "fp32"), (16, 8, 4, "fp32"),
                                             (32, 16, 4, "bf16"), (16, 8, 4, "bf16")])
def test_sweep_end_pass_matches_oracle_on_sampled_windows(pairs, W, H, w, s, R, precision):
    wk, A, B = pairs[(W, H)]
    nx, ny = oracle.grid_n(W, w, s), oracle.grid_n(H, w, s)
    pu, pv = _predictor(wk.flow, nx, ny, w, s, seed=W + w + R)
    u, v, info = rp.stage_correlate(rp.to_device(A), rp.to_device(B), w, s, R, torch.from_numpy(pu).cuda(),
                                    torch.from_numpy(pv).cuda(), precision=precision)
    torch.cuda.synchronize()
    rp.stage_status()
    valid, ky, kx = [t.cpu().numpy() for t in rp.decode_info(info)]
    u, v = u.cpu().numpy(), v.cpu().numpy()
    m = _sample(nx, ny, N_SAMPLE, seed=9000 + w + R + H)
    p64 = (pu.astype(np.float64), pv.astype(np.float64))
    ref = oracle.correlate_pass(A, B, w, s, R, *p64, want_plane=True, only=m)
    forced = oracle.correlate_pass(A, B, w, s, R, *p64, force_peaks=np.stack([ky, kx], -1).astype(np.int32), only=m)
    assert np.array_equal(valid[m].astype(int), ref.valid[m])
    same = (ky == ref.peaks[..., 0]) & (kx == ref.peaks[..., 1])
    P = ref.plane.reshape(ny, nx, -1)
    q = (ky.astype(int) + R) * (2 * R + 1) + (kx.astype(int) + R)
    gap = P.max(axis=2) - np.take_along_axis(P, q[..., None], axis=2)[..., 0]
    disagree = m & ~same
    agree = {"fp32": 0.999, "bf16": 0.99}[precision]
    assert same[m].mean() >= agree, f"{precision} peak agreement {same[m].mean():.5f}"
    # the 1e-3 px bound where the Gaussian fit is well-conditioned (tests/fitcond.py)
    vm = m & (valid == 1)
    wc = vm & well_conditioned(forced.c5)
    assert (vm & ~wc).sum() <= 0.02 * vm.sum()
    assert np.isfinite(u[m]).all() and np.isfinite(v[m]).all()
    if precision == "fp32":
        assert (gap[disagree] <= 2e-5).all()
        err = np.maximum(np.abs(u - ref.u), np.abs(v - ref.v))
        assert err[wc & same].max() <= TOL_PX
        assert np.median(err[m & same]) <= 1e-6, f"median {np.median(err[m & same]):.3g} px"
    else:
        assert (gap[disagree] <= 0.02).all()
    errf = np.maximum(np.abs(u - forced.u), np.abs(v - forced.v))
    assert errf[wc].max() <= TOL_PX, f"refit at the chosen peak: {errf[wc].max():.3g}"


def test_paper_16px_schedule_at_33mp(pairs):
    """The sweep's schedule (pyramid, 32 px +-4, then 16 px +-1) on the largest
    size: the field against the analytic one, and BF16 against FP32."""
    wk, A, B = pairs[(8192, 4096)]
    sc = wl.paper_1mp_r1().schedule
    fields = {}
    for precision in ("fp32", "bf16"):
        cfg = rp.Config.from_schedule(8192, 4096, sc, bit_depth=12, precision=precision, max_batch=1)
        eng = rp.Engine(cfg)
        u, v, om, mask = eng.process_pair(rp.to_device(A), rp.to_device(B))
        torch.cuda.synchronize()
        fields[precision] = [t.cpu().numpy() for t in (u, v, om, mask)]
        eng.close()
    u32, v32, om32, m32 = fields["fp32"]
    ny, nx = u32.shape
    assert (nx, ny) == (oracle.grid_n(8192, 16, 8), oracle.grid_n(4096, 16, 8))
    X, Y = np.meshgrid(np.arange(nx) * 8 + 7.5, np.arange(ny) * 8 + 7.5)
    tu, tv = wk.flow.eval(X, Y)
    e = np.hypot(u32 - tu, v32 - tv)
    assert np.median(e) <= 0.1 and np.percentile(e, 95) <= 0.5, (np.median(e), np.percentile(e, 95))
    assert m32.mean() >= 0.98
    u, v = fields["bf16"][:2]
    d = np.maximum(np.abs(u - u32), np.abs(v - v32))
    assert np.percentile(d, 99) <= 0.01, np.percentile(d, 99)
