"""Pre-processing (high-pass against the background, CLAHE; Sec. 2) on the
GPU against the FP64 oracle, and the correction path on pre-processed float
frames.  Bins and cumulative counts are integers on both sides, so a single
wrong bin would show as an error of the order of vmax / 256; the tolerance
(1e-4 vmax) only admits float rounding of the maps and blend weights."""
import numpy as np
import pytest
import torch

import oracle
import paper_2504_17987_gb300 as rp
from synth import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2504_17987_gb300 import build
    build.build()
    oracle.build()


@pytest.mark.parametrize("W,H,dtype,vmax,hp,tiles,clip", [
    (300, 200, np.uint16, 4095, 5, (4, 3), 250),
    (257, 129, np.uint8, 255, 7, (8, 8), 200),
    (64, 48, np.uint16, 4095, 0, (1, 1), 0),
    (96, 80, np.uint8, 255, 3, (5, 2), 100000),
])
def test_preprocess_matches_oracle(W, H, dtype, vmax, hp, tiles, clip):
    rng = np.random.default_rng(W + H)
    img = rng.integers(0, vmax + 1, (H, W)).astype(dtype)
    img[: H // 3, : W // 4] = vmax // 3  # a flat patch: a peaked histogram that clipping acts on
    out = rp.stage_preprocess(rp.to_device(img), vmax, hp=hp, tiles=tiles, clip_pct=clip).cpu().numpy()
    ref = oracle.preprocess(img.astype(np.float64), vmax, hp=hp, tiles=tiles, clip_pct=clip)
    err = np.abs(out.astype(np.float64) - ref)
    assert err.max() <= 1e-4 * vmax, f"max error {err.max():.3g}"
    if hp == 0 and clip == 0:
        assert np.array_equal(out, img.astype(np.float32))


def test_correction_path_on_preprocessed_frames():
    # pre-processed 12-bit frames (GPU) fed to an engine built for float frames,
    # against the oracle run on the same float frames
    wk = wl.paper_1mp(W=384, H=320)
    A, B = wk.render()
    H, W = A.shape
    pa = rp.stage_preprocess(rp.to_device(A), 4095, hp=7, tiles=(4, 4), clip_pct=300)
    pb = rp.stage_preprocess(rp.to_device(B), 4095, hp=7, tiles=(4, 4), clip_pct=300)
    cfg = rp.Config.from_schedule(W, H, wk.schedule, bit_depth=12, float_frames=True)
    eng = rp.Engine(cfg)
    u, v, om, m = [t.cpu().numpy() for t in eng.process_pair(pa, pb)]
    eng.close()
    fa, fb = pa.cpu().numpy().astype(np.float64), pb.cpu().numpy().astype(np.float64)
    sc = wk.schedule
    ref = oracle.process_pair(fa, fb, sc.windows, sc.overlaps, sc.radii, sc.levels)
    err = np.maximum(np.abs(u - ref.u), np.abs(v - ref.v))
    assert np.mean(err <= 1e-3) >= 0.99, f"within 1e-3: {np.mean(err <= 1e-3):.4f}"
    assert np.mean(m == ref.mask) >= 0.99
