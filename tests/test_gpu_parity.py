"""CUDA path vs the FP64 oracle on identical seeded inputs, through the C ABI.

Tolerances (FP32 path): integer peaks identical on >= 99.9 % of windows, every
disagreement a near-tie of the FP64 plane; u, v within 1e-3 px wherever the
peaks agree and the Gaussian fit is well-conditioned (tests/fitcond.py; at
most 2 % of the windows are not, and their fits must be finite); with the
oracle refitted at the GPU's peaks, the same.  BF16/FP16 planes only choose
the peak (the stencil is refitted in FP32): peaks identical on >= 99.9 %
(FP16) or >= 99 % (BF16) of windows, the others near-ties of the FP64
plane, the refit at the chosen peak within 1e-3 px, and the end-to-end field
within 0.01 px at the 99th percentile with at most 0.1 % (1 MP) or 0.2 %
(512^2) of the vectors beyond 0.01 px.  On the 1 MP workload every stage has
>= 99.9 % (FP32) and >= 99.8 % (BF16) identical peaks.
"""
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


# integer peaks identical to the FP64 plane's on at least this share of windows;
# BF16 keeps 8 significant bits and flips more near-ties than the other forms
PEAK_AGREE = {"fp32": 0.999, "fp16": 0.999, "bf16": 0.99}
ILL_MAX = 0.02  # ill-conditioned Gaussian fits (fitcond) allowed among valid windows


def check_refit(r, f_u, f_v, c5):
    """The FP32 refit against an FP64 one at the same peaks: within 1e-3 px
    where the fit is well-conditioned; finite and rare elsewhere."""
    valid = r["valid"].astype(bool)
    wc = well_conditioned(c5) & valid
    errf = np.maximum(np.abs(r["u"] - f_u), np.abs(r["v"] - f_v))
    assert errf[wc].max(initial=0.0) <= TOL_PX, f"refit error {errf[wc].max(initial=0.0):.3g}"
    assert np.isfinite(r["u"]).all() and np.isfinite(r["v"]).all()
    assert (valid & ~wc).sum() <= ILL_MAX * max(1, valid.sum())
    return wc


def check_fp32_pass(r, R, tie_tol=2e-5):
    ref = r["ref"]
    assert np.array_equal(r["valid"].astype(int), ref.valid)
    same = (r["ky"] == ref.peaks[..., 0]) & (r["kx"] == ref.peaks[..., 1])
    assert same.mean() >= PEAK_AGREE["fp32"], f"peak agreement {same.mean():.5f}"
    assert near_tie_ok(ref.plane, r["ky"], r["kx"], R, tie_tol)[~same].all()
    wc = check_refit(r, r["forced"].u, r["forced"].v, r["forced"].c5)
    err = np.maximum(np.abs(r["u"] - ref.u), np.abs(r["v"] - ref.v))
    ok = same & wc
    assert err[ok].max(initial=0.0) <= TOL_PX, f"max |du,dv| at agreeing peaks {err[ok].max(initial=0.0):.3g}"
    return same.mean(), err[ok].max(initial=0.0)


def check_16bit_pass(r, R, precision, tie_tol=0.02):
    """BF16/FP16 planes choose the peak: identical to the FP64 plane's on at
    least PEAK_AGREE of the windows, every disagreement a near-tie of the FP64
    plane (within tie_tol of its maximum), and the FP32 refit at the chosen
    peak within 1e-3 px of the FP64 refit at that peak (well-conditioned fits)."""
    ref = r["ref"]
    assert np.array_equal(r["valid"].astype(int), ref.valid)
    same = (r["ky"] == ref.peaks[..., 0]) & (r["kx"] == ref.peaks[..., 1])
    assert same.mean() >= PEAK_AGREE[precision], f"{precision} peak agreement {same.mean():.5f}"
    assert near_tie_ok(ref.plane, r["ky"], r["kx"], R, tie_tol)[~same].all()
    check_refit(r, r["forced"].u, r["forced"].v, r["forced"].c5)
    return same.mean()


# ----------------------------------------------------------------- stages ---

@pytest.mark.parametrize("kind", ["u8", "u16", "f32"])
@pytest.mark.parametrize("H, W, Wp", [(91, 130, 130), (37, 270, 272), (40, 256, 256)])
def test_downsample_bit_exact(kind, H, W, Wp):
    """2x2 box level against the oracle, bit for bit: odd sizes (last row and
    column dropped), unaligned rows (scalar loads), and rows aligned for the
    kernel's vector loads with a ragged end of row (W / 2 not a multiple of 4)
    and output rows of mixed alignment (W / 2 = 135 floats apart)."""
    rng = np.random.default_rng(1)
    if kind == "u8":
        img = rng.integers(0, 256, (H, Wp)).astype(np.uint8)
    elif kind == "u16":
        img = rng.integers(0, 4096, (H, Wp)).astype(np.uint16)
    else:
        img = (rng.integers(0, 4096 * 4, (H, Wp)) / 4.0).astype(np.float32)
    t = dev(img) if kind != "f32" else torch.from_numpy(img).cuda()
    t = t[:, :W]  # rows Wp pixels apart
    out = rp.stage_downsample(t).cpu().numpy()
    ref = oracle.downsample(img[:, :W].astype(np.float64))
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


@pytest.mark.parametrize("form", ["tiles", "strips"])
@pytest.mark.parametrize("w,s,R", [(64, 32, 4), (32, 16, 4), (16, 8, 4)])
def test_correlate_peaks_at_the_search_edge(w, s, R, form, monkeypatch):
    """A predictor R - 0.3 px short of the workload's analytic flow in x puts
    the integer peaks on the edge of the +-R search, where the 5-point stencil
    reaches shift R + 1 outside the plane: the direct FP32 stencil phase
    (which a tile or strip step runs only when some window needs it) must then
    match the oracle like the plane-supplied stencils."""
    monkeypatch.setenv("RPIV_STRIP_MIN_CTAS", "1" if form == "strips" else str(1 << 40))
    wk = wl.paper_1mp(W=320, H=288)
    A, B = wk.render()
    nx, ny = oracle.grid_n(320, w, s), oracle.grid_n(288, w, s)
    X, Y = np.meshgrid(np.arange(nx) * s + 0.5 * (w - 1), np.arange(ny) * s + 0.5 * (w - 1))
    fu, fv = wk.flow.eval(X, Y)
    pu = np.asarray(fu, dtype=np.float64) - (R - 0.3)
    pv = np.asarray(fv, dtype=np.float64)
    r = compare_pass(A, B, w, s, R, pu, pv)
    edge = r["valid"].astype(bool) & (np.abs(r["kx"]) == R)
    assert edge.mean() >= 0.1, f"only {edge.mean():.3f} of the windows peak at the search edge"
    check_fp32_pass(r, R)


@pytest.mark.parametrize("kernel", ["tcgen05", "mma"])
@pytest.mark.parametrize("precision", ["bf16", "fp16"])
@pytest.mark.parametrize("w,s,R", [(64, 32, 4), (32, 16, 4), (16, 8, 4), (32, 8, 8), (48, 24, 6), (24, 12, 6)])
def test_correlate_tensor_core_planes(precision, w, s, R, kernel, monkeypatch):
    # the mma.sync kernel runs every shape by default; RPIV_TC_PLANES=1 runs
    # the tcgen05 kernel for 50 % overlap with 8/16/32 px steps at r = 4
    if kernel == "tcgen05":
        if not (R == 4 and w == 2 * s):
            pytest.skip("shape runs the mma.sync kernel only")
        monkeypatch.setenv("RPIV_TC_PLANES", "1")
    wk = wl.paper_1mp(W=320, H=288)
    A, B = wk.render()
    nx, ny = oracle.grid_n(320, w, s), oracle.grid_n(288, w, s)
    pu, pv = smooth_field(nx, ny, w, s, seed=w * 17 + R, base=(12.0, 0.0))
    r = compare_pass(A, B, w, s, R, pu, pv, precision=precision)
    check_16bit_pass(r, R, precision)


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


def gpu_schedule_by_stages(A, B, sched, precision):
    """The engine's schedule composed from the stage entry points on the GPU:
    2x2 pyramid levels; at the coarsest a pass with a zero predictor, at each
    finer level a pass predicted by the level above (interpolated one level
    up); then the full-resolution passes, each predicted by the previous;
    outlier detection after every pass; vorticity of the last field.  Returns
    the per-stage records (the GPU's own predictor, raw result and validated
    field) and the final (u, v, vorticity, mask)."""
    H, W = A.shape
    steps = [oracle.step_of(w, o) for w, o in zip(sched.windows, sched.overlaps)]
    L = sched.levels
    a, b = dev(A), dev(B)
    levels = [(a, b, A.astype(np.float64), B.astype(np.float64))]
    for _ in range(L):
        ad, bd = rp.stage_downsample(levels[-1][0]), rp.stage_downsample(levels[-1][1])
        levels.append((ad, bd, ad.cpu().numpy().astype(np.float64), bd.cpu().numpy().astype(np.float64)))
    w0, s0, r0 = sched.windows[0], steps[0], sched.radii[0]
    stages, field = [], None

    def run(kind, idx, al, bl, Al, Bl, w, s, r, pu, pv):
        u, v, info = rp.stage_correlate(al, bl, w, s, r, pu, pv, precision=precision)
        uu, vv, mk = rp.stage_validate(u, v, info, sched.uod_threshold, sched.uod_eps, sched.replace)
        torch.cuda.synchronize()
        ny, nx = u.shape
        npf = (lambda t: np.zeros((ny, nx)) if t is None else t.cpu().numpy().astype(np.float64))
        stages.append(dict(kind=kind, idx=idx, A=Al, B=Bl, w=w, s=s, r=r, pu=npf(pu), pv=npf(pv),
                           u=u.cpu().numpy(), v=v.cpu().numpy(), info=info.cpu().numpy(),
                           uu=uu.cpu().numpy(), vv=vv.cpu().numpy(), mk=mk.cpu().numpy()))
        return uu, vv, mk

    for lvl in range(L, 0, -1):
        al, bl, Al, Bl = levels[lvl]
        nxl, nyl = oracle.grid_n(Al.shape[1], w0, s0), oracle.grid_n(Al.shape[0], w0, s0)
        pu = pv = None
        if field is not None:
            pu, pv = rp.stage_interp(field[0], field[1], w0, s0, nxl, nyl, w0, s0, 1)
        uu, vv, _ = run("level", lvl, al, bl, Al, Bl, w0, s0, r0, pu, pv)
        field = (uu, vv)
    nx0, ny0 = oracle.grid_n(W, w0, s0), oracle.grid_n(H, w0, s0)
    pu = pv = None
    if field is not None:
        pu, pv = rp.stage_interp(field[0], field[1], w0, s0, nx0, ny0, w0, s0, 1)
    for p, (w, s, r) in enumerate(zip(sched.windows, steps, sched.radii)):
        if p > 0:
            pw, ps = sched.windows[p - 1], steps[p - 1]
            pu, pv = rp.stage_interp(uu, vv, pw, ps, oracle.grid_n(W, w, s), oracle.grid_n(H, w, s), w, s, 0)
        uu, vv, mk = run("pass", p, a, b, levels[0][2], levels[0][3], w, s, r, pu, pv)
    om = rp.stage_vorticity(uu, vv, steps[-1])
    return stages, tuple(t.cpu().numpy() for t in (uu, vv, om, mk))


def check_stage(st, precision):
    """One stage against the oracle fed the GPU's own predictor for it: the
    pass (peaks, u, v, refit at the GPU's peaks) and the outlier test on the
    GPU's raw field."""
    R = st["r"]
    ref = oracle.correlate_pass(st["A"], st["B"], st["w"], st["s"], R, st["pu"].astype(np.float32).astype(np.float64),
                                st["pv"].astype(np.float32).astype(np.float64), want_plane=True)
    info = torch.from_numpy(st["info"])
    valid, ky, kx = [t.numpy() for t in rp.decode_info(info)]
    forced = oracle.correlate_pass(st["A"], st["B"], st["w"], st["s"], R,
                                   st["pu"].astype(np.float32).astype(np.float64),
                                   st["pv"].astype(np.float32).astype(np.float64),
                                   force_peaks=np.stack([ky, kx], -1).astype(np.int32))
    r = dict(u=st["u"], v=st["v"], valid=valid, ky=ky, kx=kx, ref=ref, forced=forced)
    if precision == "fp32":
        agree, _ = check_fp32_pass(r, R)
    else:
        agree = check_16bit_pass(r, R, precision)
    # the 1 MP workload: identical peaks at every stage on >= 99.9 % of the windows
    # in FP32 and >= 99.8 % in BF16 (measured minimum 99.86 %, mma.sync kernel,
    # 16 px pass; the tcgen05 kernel >= 99.9 % at every stage)
    floor = 0.999 if precision == "fp32" else 0.998
    assert agree >= floor, f"{precision} {st['kind']} {st['idx']}: peak agreement {agree:.5f}"
    ru, rv, rm = oracle.uod(st["u"].astype(np.float64), st["v"].astype(np.float64), st["info"] & 1, 2.0, 0.1, True)
    assert np.array_equal(st["mk"], rm)
    assert np.abs(st["uu"] - ru).max() <= 1e-6 and np.abs(st["vv"] - rv).max() <= 1e-6
    return agree


@pytest.mark.parametrize("precision,kernel", [("fp32", ""), ("bf16", "mma"), ("bf16", "tcgen05")])
def test_pipeline_paper_1mp_stagewise(precision, kernel, monkeypatch):
    """The 1 MP workload (12-bit, pyramid + 64 -> 32 -> 16, +-4): every pyramid
    level and every pass against the oracle fed the GPU's own predictor for
    that stage, at the bound of each form (integer peaks identical on
    >= 99.9 % (FP32) or >= 99.8 % (BF16) of windows, disagreements near-ties of
    the FP64 plane; FP32: u, v within 1e-3 px at agreeing peaks; every form: the
    FP32 refit at the GPU's peaks within 1e-3 px); the stage composition equals
    the engine's result; end to end against the oracle.  BF16 runs with the
    default (mma.sync) and the tcgen05 plane kernel."""
    if kernel == "tcgen05":
        monkeypatch.setenv("RPIV_TC_PLANES", "1")
    w = wl.paper_1mp()
    A, B = w.render()
    sc = w.schedule
    stages, (u, v, om, m) = gpu_schedule_by_stages(A, B, sc, precision)
    assert [(st["kind"], st["idx"]) for st in stages] == [("level", 2), ("level", 1), ("pass", 0), ("pass", 1),
                                                           ("pass", 2)]
    for st in stages:
        check_stage(st, precision)
    # the engine computes the same schedule
    eu, ev, eom, em = run_engine(A, B, sc, 12, precision=precision)
    assert np.mean(np.maximum(np.abs(eu - u), np.abs(ev - v)) <= 1e-5) >= 0.999
    assert np.mean(em == m) >= 0.999
    # end to end
    ref = oracle.process_pair(A, B, sc.windows, sc.overlaps, sc.radii, sc.levels)
    err = np.maximum(np.abs(eu - ref.u), np.abs(ev - ref.v))
    if precision == "fp32":
        assert np.mean(err <= TOL_PX) >= 0.999, f"within 1e-3: {np.mean(err <= TOL_PX):.5f}"
        assert np.percentile(err, 99) <= 1e-4, f"p99 {np.percentile(err, 99):.3g}"
    else:
        # the stated bound of the 16-bit forms: p99 <= 0.01 px, and at most 0.1 % of
        # the vectors (near-tie peak flips) beyond 0.01 px
        assert np.percentile(err, 99) <= 0.01, f"p99 {np.percentile(err, 99):.4f}"
        assert np.mean(err > 0.01) <= 1e-3, f"beyond 0.01 px: {np.mean(err > 0.01):.5f}"
    assert np.mean(em == ref.mask) >= 0.999


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


def test_split_batch_equals_pairs_alone(monkeypatch):
    """Batches of 16 pairs and more are captured as two halves on forked
    streams: every pair's fields must be bit-identical to the pair alone.  A
    launch takes the strip or the tile form of a pass by its CTA count, and the
    two forms agree only within FP32 rounding (their box-sum runs start at
    different rows), so the strip form is pinned here wherever the plan has
    one: strips of any segment length give identical results."""
    monkeypatch.setenv("RPIV_STRIP_MIN_CTAS", "1")
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


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
def test_pipeline_16bit_within_0p01_px(precision):
    w = wl.paper_1mp(W=512, H=512)
    A, B = w.render()
    sc = w.schedule
    u, v, _, _ = run_engine(A, B, sc, 12, precision=precision)
    ref = oracle.process_pair(A, B, sc.windows, sc.overlaps, sc.radii, sc.levels)
    err = np.maximum(np.abs(u - ref.u), np.abs(v - ref.v))
    assert np.percentile(err, 99) <= 0.01, f"p99 {np.percentile(err, 99):.4f}"
    assert np.mean(err > 0.01) <= 2e-3, f"beyond 0.01 px: {np.mean(err > 0.01):.5f}"


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
        check_16bit_pass(r, R, precision)


def test_tensor_core_path_rejects_windows_beyond_shared_memory():
    # a 128 px window's 16-bit copies do not fit one CTA's shared memory: a clear
    # UNSUPPORTED status, not a launch failure
    A = np.zeros((300, 300), np.uint8)
    with pytest.raises(rp.RpivError) as ei:
        rp.stage_correlate(dev(A), dev(A), 128, 64, 4, None, None, precision="bf16")
    assert ei.value.status == 2
