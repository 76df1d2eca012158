"""FP64 CPU oracle of the PIV correction path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product path (the CUDA library and its
binding) never imports, links or calls it, and it shares no code with it.

The heavy loops live in ``rpiv_oracle.c`` (plain double-precision C); this
module loads it with ctypes and composes the stages in the order the method
applies them (paper Sec. 2): predictor (coarse-to-fine correlation pyramid
standing in for the optical-flow engine), image deformation, correlation
stencil/plane, integer peak, three-point Gaussian fit, universal outlier
detection with median replacement, pass-to-pass interpolation, vorticity.

Parity status per function (what pins it, see tests/test_oracle_*.py):
  bilinear / deform      pinned: integer shifts, affine images
  zncc / plane           pinned: FFT cross-correlation, self-correlation,
                         affine invariance, integer circular shifts
  gauss3                 pinned: exact recovery of sampled Gaussians and
                         parabolas
  uod                    pinned: hand-built fields with known medians
  interp_grid            pinned: affine fields, pyramid position map
  downsample             pinned: affine images, constant images
  vorticity              pinned: solid-body rotation, Lamb-Oseen bound
  score_grad             pinned: central finite differences
  ema                    pinned: alpha 0 and 1, the geometric closed form of a
                         constant input, the step response
  preprocess             pinned: constant and affine images (high-pass zero
                         inside), global histogram equalisation of a uniform
                         histogram, the clipped constant image in closed form
  process_pair           pinned: imposed uniform shifts (<= 0.02 px), zero
                         displacement, vortex field against its analytic truth
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rpiv_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_up = ctypes.POINTER(ctypes.c_ubyte)


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc -O2, no fast-math: IEEE double throughout)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"],
                   check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.orc_grid_n.argtypes = [ctypes.c_int] * 3
        L.orc_grid_n.restype = ctypes.c_int
        L.orc_bilinear.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double]
        L.orc_bilinear.restype = ctypes.c_double
        L.orc_field_at.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_double, _dp, _dp]
        L.orc_field_at.restype = None
        L.orc_deform_ext.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp]
        L.orc_deform_ext.restype = None
        L.orc_pad_ext.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
        L.orc_pad_ext.restype = None
        L.orc_zncc.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.c_int, ctypes.c_int, _dp]
        L.orc_zncc.restype = ctypes.c_double
        L.orc_gauss3.argtypes = [ctypes.c_double] * 3
        L.orc_gauss3.restype = ctypes.c_double
        L.orc_pass.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.c_int, _dp, _dp, _ip, _up, _dp, _dp, _ip, _dp, _dp, _ip, _dp]
        L.orc_pass.restype = None
        L.orc_median.argtypes = [_dp, ctypes.c_int]
        L.orc_median.restype = ctypes.c_double
        L.orc_uod.argtypes = [_dp, _dp, _ip, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                              ctypes.c_int, _dp, _dp, _up]
        L.orc_uod.restype = None
        L.orc_interp_grid.argtypes = [_dp, _dp] + [ctypes.c_int] * 4 + [ctypes.c_int] * 4 + [ctypes.c_int, _dp, _dp]
        L.orc_interp_grid.restype = None
        L.orc_downsample.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp]
        L.orc_downsample.restype = None
        L.orc_vorticity.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
        L.orc_vorticity.restype = None
        L.orc_preprocess.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, _dp]
        L.orc_preprocess.restype = None
        L.orc_score_grad.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp,
                                     _dp, _dp]
        L.orc_score_grad.restype = ctypes.c_double
        _lib = L
    return _lib


def _d(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# ----------------------------------------------------------------- stages ---

def grid_n(extent: int, w: int, s: int) -> int:
    return lib().orc_grid_n(int(extent), int(w), int(s))


def step_of(w: int, overlap: float) -> int:
    s = w * (1.0 - overlap)
    si = int(round(s))
    if si < 1 or abs(s - si) > 1e-6:
        raise ValueError(f"window {w} with overlap {overlap} gives a non-integer step {s}")
    return si


def bilinear(img, X: float, Y: float) -> float:
    img = _f64(img)
    H, W = img.shape
    return lib().orc_bilinear(_d(img), W, H, float(X), float(Y))


def field_at(gu, gv, w: int, s: int, x: float, y: float) -> Tuple[float, float]:
    gu, gv = _f64(gu), _f64(gv)
    ny, nx = gu.shape
    a, b = ctypes.c_double(), ctypes.c_double()
    lib().orc_field_at(_d(gu), _d(gv), nx, ny, w, s, float(x), float(y), ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def deform_ext(img, gu, gv, w: int, s: int, M: int, scale: float = 1.0) -> np.ndarray:
    img, gu, gv = _f64(img), _f64(gu), _f64(gv)
    H, W = img.shape
    ny, nx = gu.shape
    out = np.empty((H + 2 * M, W + 2 * M), np.float64)
    lib().orc_deform_ext(_d(img), W, H, _d(gu), _d(gv), nx, ny, w, s, M, float(scale), _d(out))
    return out


def pad_ext(img, M: int) -> np.ndarray:
    img = _f64(img)
    H, W = img.shape
    out = np.empty((H + 2 * M, W + 2 * M), np.float64)
    lib().orc_pad_ext(_d(img), W, H, M, _d(out))
    return out


def zncc(Aext, Bext, W: int, M: int, x0: int, y0: int, w: int, sx: int, sy: int) -> Tuple[float, float]:
    """(C, raw numerator) of one window at one shift on grown arrays."""
    Aext, Bext = _f64(Aext), _f64(Bext)
    num = ctypes.c_double()
    c = lib().orc_zncc(_d(Aext), _d(Bext), W, M, x0, y0, w, sx, sy, ctypes.byref(num))
    return c, num.value


def gauss3(cm: float, c0: float, cp: float) -> float:
    return lib().orc_gauss3(float(cm), float(c0), float(cp))


def median(vals: Sequence[float]) -> float:
    a = _f64(vals)
    return lib().orc_median(_d(a), a.size)


@dataclasses.dataclass
class PassResult:
    u: np.ndarray
    v: np.ndarray
    peaks: np.ndarray      # (ny, nx, 2): ky, kx
    sub: np.ndarray        # (ny, nx, 2): dy, dx
    c5: np.ndarray         # (ny, nx, 5)
    valid: np.ndarray      # (ny, nx) int
    plane: Optional[np.ndarray] = None


def correlate_pass(A, B, w: int, s: int, r: int, pu, pv, *, deform: str = "b",
                   force_peaks=None, want_plane: bool = False, only=None) -> PassResult:
    """One correlation pass (deform, plane, peak, Gaussian fit) on one grid.

    pu, pv: predictor on this grid's nodes.  deform: "b" (frame B only,
    B'(x) = B(x + d(x))) or "central" (A'(x) = A(x - d/2), B'(x) = B(x + d/2)).
    only: optional (ny, nx) boolean mask; windows outside it are not evaluated
    (u, v NaN, valid -1), so that large grids can be checked on a sample.
    """
    A, B, pu, pv = _f64(A), _f64(B), _f64(pu), _f64(pv)
    H, W = A.shape
    nx, ny = grid_n(W, w, s), grid_n(H, w, s)
    assert pu.shape == (ny, nx) and pv.shape == (ny, nx)
    M = r + 2
    if deform == "b":
        Aext = pad_ext(A, M)
        Bext = deform_ext(B, pu, pv, w, s, M, 1.0)
    elif deform == "central":
        Aext = deform_ext(A, pu, pv, w, s, M, -0.5)
        Bext = deform_ext(B, pu, pv, w, s, M, 0.5)
    else:
        raise ValueError(deform)
    u = np.empty((ny, nx)); v = np.empty((ny, nx))
    peaks = np.zeros((ny, nx, 2), np.int32); sub = np.zeros((ny, nx, 2)); c5 = np.zeros((ny, nx, 5))
    valid = np.zeros((ny, nx), np.int32)
    npl = 2 * r + 1
    plane = np.zeros((ny, nx, npl, npl)) if want_plane else None
    fp = None
    if force_peaks is not None:
        fp = np.ascontiguousarray(np.asarray(force_peaks, np.int32).reshape(ny, nx, 2))
    om = None
    if only is not None:
        om = np.ascontiguousarray(np.asarray(only, bool).reshape(ny, nx).astype(np.uint8))
    lib().orc_pass(_d(Aext), _d(Bext), W, H, M, w, s, r, _d(pu), _d(pv),
                   fp.ctypes.data_as(_ip) if fp is not None else None,
                   om.ctypes.data_as(_up) if om is not None else None,
                   _d(u), _d(v), peaks.ctypes.data_as(_ip), _d(sub), _d(c5), valid.ctypes.data_as(_ip),
                   _d(plane) if plane is not None else None)
    return PassResult(u, v, peaks, sub, c5, valid, plane)


def uod(u, v, valid=None, thr: float = 2.0, eps: float = 0.1, replace: bool = True):
    """Universal outlier detection + median replacement -> (u, v, mask)."""
    u, v = _f64(u), _f64(v)
    ny, nx = u.shape
    uo = np.empty_like(u); vo = np.empty_like(v); mask = np.empty((ny, nx), np.uint8)
    va = None
    if valid is not None:
        va = np.ascontiguousarray(np.asarray(valid, np.int32))
    lib().orc_uod(_d(u), _d(v), va.ctypes.data_as(_ip) if va is not None else None, nx, ny, float(thr),
                  float(eps), int(bool(replace)), _d(uo), _d(vo), mask.ctypes.data_as(_up))
    return uo, vo, mask


def interp_grid(su, sv, sw: int, ss: int, dnx: int, dny: int, dw: int, ds: int, levels_up: int = 0):
    su, sv = _f64(su), _f64(sv)
    sny, snx = su.shape
    du = np.empty((dny, dnx)); dv = np.empty((dny, dnx))
    lib().orc_interp_grid(_d(su), _d(sv), snx, sny, sw, ss, dnx, dny, dw, ds, levels_up, _d(du), _d(dv))
    return du, dv


def downsample(img) -> np.ndarray:
    img = _f64(img)
    H, W = img.shape
    out = np.empty((H // 2, W // 2))
    lib().orc_downsample(_d(img), W, H, _d(out))
    return out


def vorticity(u, v, s: int) -> np.ndarray:
    u, v = _f64(u), _f64(v)
    ny, nx = u.shape
    w = np.empty_like(u)
    lib().orc_vorticity(_d(u), _d(v), nx, ny, s, _d(w))
    return w


def preprocess(img, vmax: int, hp: int = 7, tiles=(8, 8), clip_pct: int = 200) -> np.ndarray:
    """High-pass filter and CLAHE before the flow estimate (Sec. 2); the
    readings are stated in rpiv_oracle.c.  Returns a float image in [0, vmax]."""
    I = _f64(img)
    H, W = I.shape
    out = np.empty((H, W))
    lib().orc_preprocess(_d(I), W, H, int(vmax), int(hp), int(tiles[0]), int(tiles[1]), int(clip_pct), _d(out))
    return out


def ema(x, state, alpha: float, init: bool = False) -> np.ndarray:
    """Exponential smoothing in time (Sec. 2, constants alpha_1 for the
    predictor and alpha_2 for the output): the new state is x on the first
    frame, else alpha * x + (1 - alpha) * state."""
    x = _f64(x)
    if init:
        return x.copy()
    return alpha * x + (1.0 - alpha) * _f64(state)


def score_grad(A, B, w: int, s: int, gu, gv, grad: bool = True):
    """Score S = sum_w C_w(0) and, if grad, (dS/du, dS/dv) on the grid."""
    A, B, gu, gv = _f64(A), _f64(B), _f64(gu), _f64(gv)
    H, W = A.shape
    ny, nx = gu.shape
    assert (ny, nx) == (grid_n(H, w, s), grid_n(W, w, s))
    if grad:
        ou = np.empty_like(gu); ov = np.empty_like(gv)
        S = lib().orc_score_grad(_d(A), _d(B), W, H, w, s, _d(gu), _d(gv), _d(ou), _d(ov))
        return S, ou, ov
    S = lib().orc_score_grad(_d(A), _d(B), W, H, w, s, _d(gu), _d(gv), None, None)
    return S


# --------------------------------------------------------------- pipeline ---

@dataclasses.dataclass
class StageTrace:
    kind: str            # "level" or "pass"
    index: int           # pyramid level or pass number
    w: int
    s: int
    r: int
    pred_u: np.ndarray
    pred_v: np.ndarray
    raw: PassResult
    u: np.ndarray
    v: np.ndarray
    mask: np.ndarray


@dataclasses.dataclass
class PipelineResult:
    u: np.ndarray
    v: np.ndarray
    vort: np.ndarray
    mask: np.ndarray
    trace: List[StageTrace]


def process_pair(A, B, windows: Sequence[int], overlaps: Sequence[float], radii: Sequence[int],
                 levels: int = 0, uod_threshold: float = 2.0, uod_eps: float = 0.1, replace: bool = True,
                 pred: Optional[Tuple[np.ndarray, np.ndarray]] = None, deform: str = "b",
                 **_ignored) -> PipelineResult:
    """Full schedule on one pair.

    Predictor: a caller-supplied field on the final-pass grid, else (levels > 0)
    the coarse-to-fine pyramid: 2x2 box levels 1..L; at the coarsest level a
    pass with a zero predictor, at each finer level a pass predicted by the
    level above (upsampled); every pyramid pass uses the first pass's window,
    step and radius and is followed by outlier detection.  Then the
    full-resolution passes, each predicted by the previous (interpolated onto
    its grid), each followed by outlier detection; vorticity of the last field.
    """
    A = _f64(A); B = _f64(B)
    H, W = A.shape
    steps = [step_of(w, o) for w, o in zip(windows, overlaps)]
    trace: List[StageTrace] = []
    nx0, ny0 = grid_n(W, windows[0], steps[0]), grid_n(H, windows[0], steps[0])
    if pred is not None:
        nxl, nyl = grid_n(W, windows[-1], steps[-1]), grid_n(H, windows[-1], steps[-1])
        gu, gv = _f64(pred[0]).reshape(nyl, nxl), _f64(pred[1]).reshape(nyl, nxl)
        pu, pv = interp_grid(gu, gv, windows[-1], steps[-1], nx0, ny0, windows[0], steps[0], 0)
    elif levels > 0:
        pyr = [(A, B)]
        for _ in range(levels):
            pyr.append((downsample(pyr[-1][0]), downsample(pyr[-1][1])))
        field = None
        w0, s0, r0 = windows[0], steps[0], radii[0]
        for lvl in range(levels, 0, -1):
            Al, Bl = pyr[lvl]
            hl, wl = Al.shape
            nxl, nyl = grid_n(wl, w0, s0), grid_n(hl, w0, s0)
            if field is None:
                pu, pv = np.zeros((nyl, nxl)), np.zeros((nyl, nxl))
            else:
                pu, pv = interp_grid(field[0], field[1], w0, s0, nxl, nyl, w0, s0, 1)
            raw = correlate_pass(Al, Bl, w0, s0, r0, pu, pv, deform=deform)
            uu, vv, mk = uod(raw.u, raw.v, raw.valid, uod_threshold, uod_eps, replace)
            trace.append(StageTrace("level", lvl, w0, s0, r0, pu, pv, raw, uu, vv, mk))
            field = (uu, vv)
        pu, pv = interp_grid(field[0], field[1], w0, s0, nx0, ny0, w0, s0, 1)
    else:
        pu, pv = np.zeros((ny0, nx0)), np.zeros((ny0, nx0))
    uu = vv = mk = None
    for p, (w, s, r) in enumerate(zip(windows, steps, radii)):
        nxp, nyp = grid_n(W, w, s), grid_n(H, w, s)
        if p > 0:
            pu, pv = interp_grid(uu, vv, windows[p - 1], steps[p - 1], nxp, nyp, w, s, 0)
        raw = correlate_pass(A, B, w, s, r, pu, pv, deform=deform)
        uu, vv, mk = uod(raw.u, raw.v, raw.valid, uod_threshold, uod_eps, replace)
        trace.append(StageTrace("pass", p, w, s, r, pu, pv, raw, uu, vv, mk))
    om = vorticity(uu, vv, steps[-1])
    return PipelineResult(uu, vv, om, mk, trace)


def ascend(f, u0, v0, steps: int = 5, eta0: float = 0.25, halvings: int = 3):
    """The refinement's step rule on any score: f(u, v) -> (S, gu, gv), and
    f(u, v, grad=False) -> S.

    g0 = grad S at the start; step k moves along the current gradient with
    eta_k = eta0 * 0.5^k / max|g0|; the step is accepted only if S increases,
    otherwise eta is halved and the step retried, at most `halvings` times
    (the field stays where it was if every try fails).  Returns
    (u, v, [S at the start and after each step]).
    """
    u = _f64(u0).copy(); v = _f64(v0).copy()
    S, gu, gv = f(u, v)
    gmax = max(float(np.max(np.abs(gu))), float(np.max(np.abs(gv))))
    hist = [S]
    if gmax == 0.0:
        return u, v, hist
    for k in range(steps):
        eta = eta0 * 0.5 ** k / gmax
        for _ in range(halvings + 1):
            cu, cv = u + eta * gu, v + eta * gv
            Sc = f(cu, cv, grad=False)
            if Sc > S:
                u, v, S = cu, cv, Sc
                break
            eta *= 0.5
        S, gu, gv = f(u, v)
        hist.append(S)
    return u, v, hist


def refine(A, B, w: int, s: int, u0, v0, steps: int = 5, eta0: float = 0.25, halvings: int = 3):
    """Gradient-ascent refinement of the correlation score S (differentiation
    pattern): ascend() on score_grad of the pair."""
    def f(u, v, grad=True):
        return score_grad(A, B, w, s, u, v, grad=grad)
    return ascend(f, u0, v0, steps, eta0, halvings)
