"""CUDA path vs the FP64 oracle on identical seeded inputs, through the C ABI.

Tolerances (FP32 path): integer peaks identical on >= 99.9 % of windows, every
disagreement a near-tie of the FP64 plane; u, v within 1e-3 px wherever the
peaks agree; with the oracle refitted at the GPU's peaks, every window within
1e-3 px.  BF16/FP16 planes only choose the peak (the stencil is refitted in
FP32): peaks may differ on near-ties of the bf16-rounded plane, the refit at
the chosen peak is within 1e-3 px, and the end-to-end field within 0.01 px at
the 99th percentile.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2504_17987_gb300 as rp
import synth
from synth import workloads as wl

pytestmark = pytest.mark.gpu

TOL_PX = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2504_17987_gb300 import build
    build.build()
    oracle.build()


def dev(x):
    return rp.to_device(x, "cuda:0")


def smooth_field(nx, ny, w, s, seed, amp=1.5, base=(0.0, 0.0)):
    r = synth.uniform(seed, 6)
    X, Y = np.meshgrid(np.arange(nx) * s + 0.5 * (w - 1), np.arange(ny) * s + 0.5 * (w - 1))
    pu = base[0] + amp * np.sin(X / 97.0 + 6 * r[0]) * np.cos(Y / 83.0 + 6 * r[1]) + r[2] - 0.5
    pv = base[1] + amp * np.cos(X / 71.0 + 6 * r[3]) * np.sin(Y / 101.0 + 6 * r[4]) + r[5] - 0.5
    return pu, pv


def near_tie_ok(plane, ky, kx, R, tol):
    """True where the GPU's peak is within tol of the FP64 plane maximum."""
    ny, nx = ky.shape
    P = plane.reshape(ny, nx, -1)
    best = P.max(axis=2)
    q = (ky.astype(int) + R) * (2 * R + 1) + (kx.astype(int) + R)
    got = np.take_along_axis(P, q[..., None], axis=2)[..., 0]
    return best - got <= tol


def compare_pass(A, B, w, s, R, pu, pv, precision="fp32", deform="b"):
    a, b = dev(A), dev(B)
    tpu = torch.from_numpy(pu.astype(np.float32)).cuda() if pu is not None else None
    tpv = torch.from_numpy(pv.astype(np.float32)).cuda() if pv is not None else None
    u, v, info = rp.stage_correlate(a, b, w, s, R, tpu, tpv, precision=precision, deform=deform)
    torch.cuda.synchronize()
    valid, ky, kx = [t.cpu().numpy() for t in rp.decode_info(info)]
    u, v = u.cpu().numpy(), v.cpu().numpy()
    H, W = A.shape
    nx, ny = oracle.grid_n(W, w, s), oracle.grid_n(H, w, s)
    # the oracle sees the predictor exactly as the GPU stored it (FP32 values)
    opu = np.zeros((ny, nx)) if pu is None else pu.astype(np.float32).astype(np.float64)
    opv = np.zeros((ny, nx)) if pv is None else pv.astype(np.float32).astype(np.float64)
    ref = oracle.correlate_pass(A, B, w, s, R, opu, opv, deform=deform, want_plane=True)
    forced = oracle.correlate_pass(A, B, w, s, R, opu, opv, deform=deform,
                                   force_peaks=np.stack([ky, kx], -1).astype(np.int32))
    return dict(u=u, v=v, valid=valid, ky=ky, kx=kx, ref=ref, forced=forced)


def check_fp32_pass(r, R, tie_tol=2e-5):
    ref = r["ref"]
    assert np.array_equal(r["valid"].astype(int), ref.valid)
    same = (r["ky"] == ref.peaks[..., 0]) & (r["kx"] == ref.peaks[..., 1])
    assert same.mean() >= 0.999, f"peak agreement {same.mean():.5f}"
    assert near_tie_ok(ref.plane, r["ky"], r["kx"], R, tie_tol)[~same].all()
    err = np.maximum(np.abs(r["u"] - ref.u), np.abs(r["v"] - ref.v))
    assert err[same].max() <= TOL_PX, f"max |du,dv| at agreeing peaks {err[same].max():.3g}"
    f = r["forced"]
    errf = np.maximum(np.abs(r["u"] - f.u), np.abs(r["v"] - f.v))
    assert errf.max() <= TOL_PX, f"max refit error {errf.max():.3g}"
    return same.mean(), err.max()


# ----------------------------------------------------------------- stages ---

@pytest.mark.parametrize("kind", ["u8", "u16", "f32"])
def test_downsample_bit_exact(kind):
    rng = np.random.default_rng(1)
    H, W = 91, 130  # odd sizes: last row dropped
    if kind == "u8":
        img = rng.integers(0, 256, (H, W)).astype(np.uint8)
    elif kind == "u16":
        img = rng.integers(0, 4096, (H, W)).astype(np.uint16)
    else:
        img = (rng.integers(0, 4096 * 4, (H, W)) / 4.0).astype(np.float32)
    t = dev(img) if kind != "f32" else torch.from_numpy(img).cuda()
    out = rp.stage_downsample(t).cpu().numpy()
    ref = oracle.downsample(img.astype(np.float64))
    assert out.shape == ref.shape
    assert np.array_equal(out.astype(np.float64), ref)


def test_correlate_zero_predictor_plain_256():
    w = wl.plain_256()
    A, B = w.render()
    r = compare_pass(A, B, 32, 16, 8, None, None)
    check_fp32_pass(r, 8)


@pytest.mark.parametrize("form", ["tiles", "strips"])
@pytest.mark.parametrize("w,s,R", [(64, 32, 4), (32, 16, 4), (16, 8, 4), (32, 8, 8), (48, 24, 6), (16, 8, 1),
                                   (24, 12, 6), (16, 8, 0), (20, 10, 3), (16, 12, 2), (32, 16, 1), (64, 32, 1)])
def test_correlate_with_predictor_fp32(w, s, R, form, monkeypatch):
    # strips (32 and 64 px windows at 50 %, r = 1 and 4) are taken at launch
    # only for large batches; the threshold is lowered here to run them on one
    # pair, and raised to keep the tile kernels
    monkeypatch.setenv("RPIV_STRIP_MIN_CTAS", "1" if form == "strips" else str(1 << 40))
    wk = wl.paper_1mp(W=320, H=288)
    A, B = wk.render()
    nx, ny = oracle.grid_n(320, w, s), oracle.grid_n(288, w, s)
    pu, pv = smooth_field(nx, ny, w, s, seed=w * 31 + R, base=(12.0, 0.0))
    r = compare_pass(A, B, w, s, R, pu, pv)
    check_fp32_pass(r, R)


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
@pytest.mark.parametrize("w,s,R", [(64, 32, 4), (32, 16, 4), (16, 8, 4), (32, 8, 8), (48, 24, 6), (24, 12, 6)])
def test_correlate_tensor_core_planes(precision, w, s, R):
    wk = wl.paper_1mp(W=320, H=288)
    A, B = wk.render()
    nx, ny = oracle.grid_n(320, w, s), oracle.grid_n(288, w, s)
    pu, pv = smooth_field(nx, ny, w, s, seed=w * 17 + R, base=(12.0, 0.0))
    r = compare_pass(A, B, w, s, R, pu, pv, precision=precision)
    ref = r["ref"]
    same = (r["ky"] == ref.peaks[..., 0]) & (r["kx"] == ref.peaks[..., 1])
    # the 16-bit plane chooses the peak; disagreements must be near-ties of the FP64 plane
    assert same.mean() >= 0.99, f"{precision} peak agreement {same.mean():.4f}"
    assert near_tie_ok(ref.plane, r["ky"], r["kx"], R, 0.02)[~same].all()
    f = r["forced"]
    errf = np.maximum(np.abs(r["u"] - f.u), np.abs(r["v"] - f.v))
    assert errf.max() <= TOL_PX, f"refit at the chosen peak: {errf.max():.3g}"


def test_correlate_central_deformation():
    wk = wl.paper_1mp(W=256, H=256)
    A, B = wk.render()
    nx = oracle.grid_n(256, 32, 16)
    pu, pv = smooth_field(nx, nx, 32, 16, seed=5, base=(12.0, 0.0))
    r = compare_pass(A, B, 32, 16, 4, pu, pv, deform="central")
    check_fp32_pass(r, 4)


def test_correlate_degenerate_windows_and_minimum_size():
    # flat left half: invalid windows keep the predictor; image exactly w + 2(R+1) tall
    rng = np.random.default_rng(3)
    H, W = 16 + 2 * 5, 96
    A = rng.integers(0, 255, (H, W)).astype(np.uint8)
    A[:, :40] = 77
    B = np.roll(A, 2, axis=1)
    nx, ny = oracle.grid_n(W, 16, 8), oracle.grid_n(H, 16, 8)
    pu = np.full((ny, nx), 0.25)
    pv = np.full((ny, nx), -0.5)
    r = compare_pass(A, B, 16, 8, 4, pu, pv)
    assert (r["valid"] == 0).any() and (r["valid"] == 1).any()
    check_fp32_pass(r, 4)
    inv = r["valid"] == 0
    assert np.all(r["u"][inv] == np.float32(0.25)) and np.all(r["v"][inv] == np.float32(-0.5))


def test_validate_matches_oracle():
    rng = np.random.default_rng(9)
    ny, nx = 37, 53
    i, j = np.meshgrid(np.arange(nx), np.arange(ny))
    u = (0.05 * i + 0.02 * j + 0.05 * rng.standard_normal((ny, nx))).astype(np.float32)
    v = (0.01 * i - 0.03 * j + 0.05 * rng.standard_normal((ny, nx))).astype(np.float32)
    spikes = rng.random((ny, nx)) < 0.03
    u[spikes] += rng.uniform(-5, 5, spikes.sum()).astype(np.float32)
    info = np.ones((ny, nx), np.int32)
    info[rng.random((ny, nx)) < 0.01] = 0
    tu, tv, ti = (torch.from_numpy(x).cuda() for x in (u, v, info))
    uo, vo, m = rp.stage_validate(tu, tv, ti, 2.0, 0.1, True)
    uo, vo, m = uo.cpu().numpy(), vo.cpu().numpy(), m.cpu().numpy()
    ru, rv, rm = oracle.uod(u.astype(np.float64), v.astype(np.float64), info, 2.0, 0.1, True)
    assert np.array_equal(m, rm)
    assert np.abs(uo - ru).max() <= 1e-6 and np.abs(vo - rv).max() <= 1e-6


def test_interp_and_vorticity_match_oracle():
    rng = np.random.default_rng(4)
    su = rng.standard_normal((7, 9)).astype(np.float32)
    sv = rng.standard_normal((7, 9)).astype(np.float32)
    tsu, tsv = torch.from_numpy(su).cuda(), torch.from_numpy(sv).cuda()
    for (dw, ds, dnx, dny, L) in [(32, 16, 31, 27, 0), (16, 8, 63, 55, 1), (64, 32, 15, 13, 2)]:
        du, dv = rp.stage_interp(tsu, tsv, 64, 32, dnx, dny, dw, ds, L)
        ru, rv = oracle.interp_grid(su, sv, 64, 32, dnx, dny, dw, ds, L)
        assert np.abs(du.cpu().numpy() - ru).max() <= 1e-5 * max(1, np.abs(ru).max())
        assert np.abs(dv.cpu().numpy() - rv).max() <= 1e-5 * max(1, np.abs(rv).max())
    om = rp.stage_vorticity(tsu, tsv, 8).cpu().numpy()
    assert np.abs(om - oracle.vorticity(su, sv, 8)).max() <= 1e-5


# --------------------------------------------------------------- pipeline ---

def run_engine(A, B, sched, bit_depth, precision="fp32", pred=None):
    H, W = A.shape
    cfg = rp.Config.from_schedule(W, H, sched, bit_depth=bit_depth, precision=precision)
    eng = rp.Engine(cfg)
    p = None
    if pred is not None:
        p = tuple(torch.from_numpy(x.astype(np.float32)).cuda() for x in pred)
    u, v, om, m = eng.process_pair(dev(A), dev(B), pred=p)
    torch.cuda.synchronize()
    out = tuple(t.cpu().numpy() for t in (u, v, om, m))
    eng.close()
    return out


def test_pipeline_plain_256_end_to_end():
    w = wl.plain_256()
    A, B = w.render()
    sc = w.schedule
    u, v, om, m = run_engine(A, B, sc, 8)
    ref = oracle.process_pair(A, B, sc.windows, sc.overlaps, sc.radii, sc.levels)
    err = np.maximum(np.abs(u - ref.u), np.abs(v - ref.v))
    assert np.mean(err <= TOL_PX) >= 0.999 and err.max() <= 5e-3
    assert np.array_equal(m, ref.mask)
    assert np.abs(om - ref.vort).max() <= 2e-4


def test_pipeline_paper_1mp_end_to_end_stagewise():
    """1 MP, 12-bit, pyramid + 64 -> 32 -> 16: end-to-end statistics, and each
    pass against the oracle fed the GPU's own predictor for that pass."""
    w = wl.paper_1mp()
    A, B = w.render()
    sc = w.schedule
    u, v, om, m = run_engine(A, B, sc, 12)
    ref = oracle.process_pair(A, B, sc.windows, sc.overlaps, sc.radii, sc.levels)
    err = np.maximum(np.abs(u - ref.u), np.abs(v - ref.v))
    assert np.mean(err <= TOL_PX) >= 0.99, f"within 1e-3: {np.mean(err <= TOL_PX):.4f}"
    assert np.percentile(err, 99) <= 0.05
    assert np.mean(m == ref.mask) >= 0.99


@pytest.mark.parametrize("form", ["tiles", "strips"])
def test_pipeline_supplied_predictor_and_batch_equals_single(form, monkeypatch):
    # the engine's 64 and 32 px passes as tiles, and as strips (forced at any batch size)
    monkeypatch.setenv("RPIV_STRIP_MIN_CTAS", "1" if form == "strips" else str(1 << 40))
    w = wl.paper_1mp(W=512, H=512)
    A, B = w.render()
    sc = w.schedule
    H, W = A.shape
    cfg = rp.Config.from_schedule(W, H, sc, bit_depth=12, max_batch=3)
    eng = rp.Engine(cfg)
    a, b = dev(A), dev(B)
    # a second pair: swap roles (different content, same size)
    a2, b2 = dev(B), dev(A)
    single = [t.clone() for t in eng.process_pair(a, b)]
    single2 = [t.clone() for t in eng.process_pair(a2, b2)]
    # predictor: the first result, for pair 3 only
    pred = (single[0].clone(), single[1].clone())
    outs = eng.process_batch([a, a2, a], [b, b2, b], preds=[None, None, pred])
    again = eng.process_batch([a, a2, a], [b, b2, b], preds=[None, None, pred])  # graph replay
    torch.cuda.synchronize()
    for k in range(4):
        assert torch.equal(outs[k][0], single[k]), k
        assert torch.equal(outs[k][1], single2[k]), k
        assert torch.equal(again[k][0], single[k]), k
    # pair 3 used the predictor: its result equals process_pair with that predictor
    with_pred = eng.process_pair(a, b, pred=pred)
    torch.cuda.synchronize()
    for k in range(4):
        assert torch.equal(outs[k][2], with_pred[k]), k
    ny, nx = single[0].shape
    ref = oracle.process_pair(A, B, sc.windows, sc.overlaps, sc.radii, sc.levels,
                              pred=(pred[0].cpu().numpy().astype(np.float64), pred[1].cpu().numpy().astype(np.float64)))
    err = np.maximum(np.abs(with_pred[0].cpu().numpy() - ref.u), np.abs(with_pred[1].cpu().numpy() - ref.v))
    assert np.mean(err <= TOL_PX) >= 0.99
    eng.close()


def test_split_batch_equals_pairs_alone():
    # batches of 16 pairs and more are captured as two halves on forked streams
    wk = wl.paper_1mp(W=512, H=512)
    sc = wk.schedule
    cfg = rp.Config.from_schedule(512, 512, sc, bit_depth=12, max_batch=16)
    eng = rp.Engine(cfg)
    pairs = []
    for k in range(16):
        A, B = wl.paper_1mp(W=512, H=512, seed=2000 + k).render()
        pairs.append((dev(A), dev(B)))
    alone = [[t.clone() for t in eng.process_pair(a, b)] for a, b in pairs]
    outs = eng.process_batch([p[0] for p in pairs], [p[1] for p in pairs])  # eager first run
    again = eng.process_batch([p[0] for p in pairs], [p[1] for p in pairs])  # the split graph
    torch.cuda.synchronize()
    for i in range(16):
        for k in range(4):
            assert torch.equal(outs[k][i], alone[i][k]), (i, k)
            assert torch.equal(again[k][i], alone[i][k]), (i, k)
    eng.close()


def test_pipeline_bf16_within_0p01_px():
    w = wl.paper_1mp(W=512, H=512)
    A, B = w.render()
    sc = w.schedule
    u, v, _, _ = run_engine(A, B, sc, 12, precision="bf16")
    ref = oracle.process_pair(A, B, sc.windows, sc.overlaps, sc.radii, sc.levels)
    err = np.maximum(np.abs(u - ref.u), np.abs(v - ref.v))
    assert np.percentile(err, 99) <= 0.01, f"p99 {np.percentile(err, 99):.4f}"


def test_pipeline_paper_exact_variant_central_warp_zero_radius():
    """The paper's own correction (Sec. 2): both frames warped by central
    differences and the 5-point stencil fixed at the predicted peak (r = 0),
    after a pyramid and a 32 px +-4 pass; end to end against the oracle."""
    w = wl.paper_1mp(W=512, H=384)
    A, B = w.render()
    sc = wl.Schedule((32, 16), (0.5, 0.5), (4, 0), levels=2)
    H, W = A.shape
    cfg = rp.Config.from_schedule(W, H, sc, bit_depth=12, deform="central")
    eng = rp.Engine(cfg)
    u, v, om, m = [t.cpu().numpy() for t in eng.process_pair(dev(A), dev(B))]
    eng.close()
    ref = oracle.process_pair(A, B, sc.windows, sc.overlaps, sc.radii, sc.levels, deform="central")
    err = np.maximum(np.abs(u - ref.u), np.abs(v - ref.v))
    assert np.mean(err <= TOL_PX) >= 0.99, f"within 1e-3: {np.mean(err <= TOL_PX):.4f}"
    assert np.percentile(err, 99) <= 0.05
    assert np.mean(m == ref.mask) >= 0.99


def test_ema_stage_matches_oracle():
    rng = np.random.default_rng(21)
    x = rng.standard_normal(10007).astype(np.float32)
    st = rng.standard_normal(10007).astype(np.float32)
    tx, ts = torch.from_numpy(x).cuda(), torch.from_numpy(st).cuda()
    for alpha in (0.0, 0.25, 0.5, 1.0):
        out = rp.stage_ema(tx, ts.clone(), alpha).cpu().numpy()
        ref = oracle.ema(x, st, alpha)
        assert np.abs(out - ref).max() <= 1e-6 * max(1.0, np.abs(ref).max())
    out = rp.stage_ema(tx, ts.clone(), 0.5, init=True).cpu().numpy()
    assert np.array_equal(out, x)
    with pytest.raises(rp.RpivError):
        rp.stage_ema(tx, ts.clone(), 1.5)


@pytest.mark.parametrize("w,s,R,precision", [(32, 16, 12, "fp32"), (128, 64, 4, "fp32"), (8, 4, 2, "fp32"),
                                             (16, 8, 16, "fp32"), (96, 48, 4, "bf16"), (16, 8, 8, "bf16")])
def test_correlate_edge_shapes(w, s, R, precision):
    # runtime-radius kernel (r 12, 16), the largest window, the smallest, and
    # tensor-core shapes outside the benchmark's; ragged tails on both axes
    W, H = 8 * w + 2 * R + 11, 6 * w + 2 * R + 7
    wk = wl.paper_1mp(W=W, H=H)
    A, B = wk.render()
    nx, ny = oracle.grid_n(W, w, s), oracle.grid_n(H, w, s)
    pu, pv = smooth_field(nx, ny, w, s, seed=w + 3 * R, base=(12.0, 0.0), amp=1.0)
    r = compare_pass(A, B, w, s, R, pu, pv, precision=precision)
    if precision == "fp32":
        check_fp32_pass(r, R)
    else:
        ref = r["ref"]
        same = (r["ky"] == ref.peaks[..., 0]) & (r["kx"] == ref.peaks[..., 1])
        assert same.mean() >= 0.98, f"{precision} peak agreement {same.mean():.4f}"
        assert near_tie_ok(ref.plane, r["ky"], r["kx"], R, 0.02)[~same].all()
        f = r["forced"]
        assert np.maximum(np.abs(r["u"] - f.u), np.abs(r["v"] - f.v)).max() <= TOL_PX


def test_tensor_core_path_rejects_windows_beyond_shared_memory():
    # a 128 px window's 16-bit copies do not fit one CTA's shared memory: a clear
    # UNSUPPORTED status, not a launch failure
    A = np.zeros((300, 300), np.uint8)
    with pytest.raises(rp.RpivError) as ei:
        rp.stage_correlate(dev(A), dev(A), 128, 64, 4, None, None, precision="bf16")
    assert ei.value.status == 2
