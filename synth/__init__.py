"""Seeded synthetic PIV image pairs (inputs only; no correlation arithmetic).

The C generator (``synth.c``) renders tracer-particle pairs displaced by an
analytic flow; this module builds it with gcc, wraps it with ctypes and names
the workloads used by tests and the benchmark.  Both the FP64 oracle and the
CUDA path take their inputs from here, and from nowhere else.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
from typing import Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_SRC = os.path.join(_HERE, "synth.c")

MAX_VORTEX = 8
MAX_MODES = 16


class _Flow(ctypes.Structure):
    _fields_ = [
        ("U", ctypes.c_double), ("V", ctypes.c_double),
        ("n_vortex", ctypes.c_int),
        ("vx", ctypes.c_double * MAX_VORTEX), ("vy", ctypes.c_double * MAX_VORTEX),
        ("gamma", ctypes.c_double * MAX_VORTEX), ("rc", ctypes.c_double * MAX_VORTEX),
        ("shear_dU", ctypes.c_double), ("shear_y0", ctypes.c_double), ("shear_delta", ctypes.c_double),
        ("n_modes", ctypes.c_int),
        ("kx", ctypes.c_double * MAX_MODES), ("ky", ctypes.c_double * MAX_MODES),
        ("amp", ctypes.c_double * MAX_MODES), ("phase", ctypes.c_double * MAX_MODES),
        ("Lx", ctypes.c_double), ("Ly", ctypes.c_double),
    ]


class _Params(ctypes.Structure):
    _fields_ = [
        ("W", ctypes.c_int), ("H", ctypes.c_int), ("bit_depth", ctypes.c_int),
        ("ppp", ctypes.c_double), ("dp_min", ctypes.c_double), ("dp_max", ctypes.c_double),
        ("i0_min", ctypes.c_double), ("i0_max", ctypes.c_double),
        ("noise_frac", ctypes.c_double), ("loss_frac", ctypes.c_double),
        ("margin", ctypes.c_double), ("seed", ctypes.c_uint64),
    ]


def build(force: bool = False) -> str:
    """Compile libsynth.so next to its source (gcc, OpenMP when available)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.synth_render_pair.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(_Flow), ctypes.c_void_p, ctypes.c_void_p]
        lib.synth_render_pair.restype = ctypes.c_long
        lib.synth_flow_eval.argtypes = [ctypes.POINTER(_Flow), ctypes.c_long, dp, dp, dp, dp]
        lib.synth_flow_eval.restype = None
        lib.synth_uniform.argtypes = [ctypes.c_uint64, ctypes.c_long, dp]
        lib.synth_uniform.restype = None
        lib.synth_rng_probe.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64),
                                        ctypes.POINTER(ctypes.c_uint64)]
        lib.synth_rng_probe.restype = None
        _lib = lib
    return _lib


@dataclasses.dataclass
class Flow:
    """Analytic displacement field in px/frame (x = column, y = row, down)."""
    U: float = 0.0
    V: float = 0.0
    vortices: Sequence[Tuple[float, float, float, float]] = ()  # (xc, yc, Gamma, rc)
    shear: Optional[Tuple[float, float, float]] = None            # (dU, y0, delta) on u
    modes: Sequence[Tuple[float, float, float, float]] = ()       # (kx, ky, amp, phase)
    L: Tuple[float, float] = (1.0, 1.0)                           # mode periods (Lx, Ly)

    def _c(self) -> _Flow:
        f = _Flow()
        f.U, f.V = float(self.U), float(self.V)
        if len(self.vortices) > MAX_VORTEX or len(self.modes) > MAX_MODES:
            raise ValueError("too many vortices or modes")
        f.n_vortex = len(self.vortices)
        for i, (xc, yc, g, rc) in enumerate(self.vortices):
            f.vx[i], f.vy[i], f.gamma[i], f.rc[i] = xc, yc, g, rc
        if self.shear is not None:
            f.shear_dU, f.shear_y0, f.shear_delta = self.shear
        else:
            f.shear_dU, f.shear_y0, f.shear_delta = 0.0, 0.0, 1.0
        f.n_modes = len(self.modes)
        for i, (kx, ky, a, ph) in enumerate(self.modes):
            f.kx[i], f.ky[i], f.amp[i], f.phase[i] = kx, ky, a, ph
        f.Lx, f.Ly = float(self.L[0]), float(self.L[1])
        return f

    def eval(self, x, y) -> Tuple[np.ndarray, np.ndarray]:
        """Displacement (u, v) at arrays of positions."""
        x = np.ascontiguousarray(np.broadcast_to(np.asarray(x, np.float64), np.broadcast(x, y).shape))
        y = np.ascontiguousarray(np.broadcast_to(np.asarray(y, np.float64), x.shape))
        u = np.empty_like(x)
        v = np.empty_like(x)
        dp = ctypes.POINTER(ctypes.c_double)
        f = self._c()
        _load().synth_flow_eval(ctypes.byref(f), x.size, x.ctypes.data_as(dp), y.ctypes.data_as(dp),
                                u.ctypes.data_as(dp), v.ctypes.data_as(dp))
        return u, v


@dataclasses.dataclass
class ImageSpec:
    W: int
    H: int
    bit_depth: int = 8
    ppp: float = 0.05
    dp: Tuple[float, float] = (2.5, 2.5)
    i0: Tuple[float, float] = (150.0, 255.0)
    noise_frac: float = 0.02
    loss_frac: float = 0.0
    margin: Optional[float] = None  # default: max |d| + 4 px, from the flow
    seed: int = 1001


def render_pair(spec: ImageSpec, flow: Flow) -> Tuple[np.ndarray, np.ndarray]:
    """Render (A, B) as uint8 (8-bit) or uint16 (12/16-bit) arrays of shape (H, W)."""
    margin = spec.margin
    if margin is None:
        gx, gy = np.meshgrid(np.arange(0, spec.W, 8.0), np.arange(0, spec.H, 8.0))
        u, v = flow.eval(gx, gy)
        margin = float(np.max(np.hypot(u, v))) + 4.0
    p = _Params()
    p.W, p.H, p.bit_depth = spec.W, spec.H, spec.bit_depth
    p.ppp = spec.ppp
    p.dp_min, p.dp_max = spec.dp
    p.i0_min, p.i0_max = spec.i0
    p.noise_frac, p.loss_frac = spec.noise_frac, spec.loss_frac
    p.margin = margin
    p.seed = spec.seed & 0xFFFFFFFFFFFFFFFF
    dt = np.uint8 if spec.bit_depth <= 8 else np.uint16
    a = np.zeros((spec.H, spec.W), dt)
    b = np.zeros((spec.H, spec.W), dt)
    f = flow._c()
    n = _load().synth_render_pair(ctypes.byref(p), ctypes.byref(f), a.ctypes.data, b.ctypes.data)
    if n < 0:
        raise RuntimeError("synth_render_pair failed")
    return a, b


def uniform(seed: int, n: int) -> np.ndarray:
    out = np.empty(n, np.float64)
    _load().synth_uniform(seed & 0xFFFFFFFFFFFFFFFF, n, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def rng_probe(seed: int, n: int):
    sm = (ctypes.c_uint64 * n)()
    xo = (ctypes.c_uint64 * n)()
    _load().synth_rng_probe(seed & 0xFFFFFFFFFFFFFFFF, n, sm, xo)
    return list(sm), list(xo)


def lamb_oseen_vorticity(x, y, xc, yc, gamma, rc):
    """Closed-form vorticity dv/dx - du/dy of one Lamb-Oseen vortex (1/frame)."""
    r2 = (np.asarray(x) - xc) ** 2 + (np.asarray(y) - yc) ** 2
    return gamma / (math.pi * rc * rc) * np.exp(-r2 / (rc * rc))
