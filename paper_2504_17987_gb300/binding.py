"""ctypes binding of librpiv (include/rpiv.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Torch tensors supply device memory and the current stream.
There is no CPU fallback: if librpiv.so is missing or no GPU is present the
calls raise.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import List, Optional, Sequence, Tuple

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librpiv.so")

RPIV_U8, RPIV_U16, RPIV_F32 = 1, 2, 3


def _poison() -> bool:
    """RPIV_POISON_SCRATCH=1 (a test setting): scratch and outputs start as
    0xFF bytes (NaN as float), so that a value no kernel wrote surfaces."""
    return os.environ.get("RPIV_POISON_SCRATCH", "") == "1"


def _fresh(t: torch.Tensor) -> torch.Tensor:
    if _poison():
        t.view(torch.uint8).fill_(0xFF)
    return t
RPIV_FP32, RPIV_BF16, RPIV_FP16 = 0, 1, 2
RPIV_DEFORM_B, RPIV_DEFORM_CENTRAL = 0, 1
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED", 3: "OOM", 4: "CUDA", 5: "TIMEOUT", 6: "BUSY", 7: "NO_DEVICE"}
PRECISIONS = {"fp32": RPIV_FP32, "bf16": RPIV_BF16, "fp16": RPIV_FP16}

EXPORTED = sorted(["rpiv_config_default", "rpiv_validate_config", "rpiv_create", "rpiv_grid_shape",
                   "rpiv_workspace_bytes", "rpiv_process_pair", "rpiv_process_batch", "rpiv_backward", "rpiv_refine",
                   "rpiv_wait", "rpiv_destroy", "rpiv_last_error", "rpiv_stage_correlate", "rpiv_stage_correlate_scratch_bytes",
                   "rpiv_stage_correlate_noalloc", "rpiv_stage_status", "rpiv_stage_validate",
                   "rpiv_stage_interp", "rpiv_stage_vorticity", "rpiv_stage_downsample", "rpiv_stage_ema",
                   "rpiv_stage_preprocess", "rpiv_stage_preprocess_scratch_bytes",
                   "rpiv_trace_enable", "rpiv_trace_read"])


class RpivError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"rpiv {STATUS.get(status, status)}: {msg}")
        self.status = status


class TraceRecord(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int), ("total_ms", ctypes.c_float),
                ("width", ctypes.c_int), ("height", ctypes.c_int), ("window", ctypes.c_int), ("step", ctypes.c_int),
                ("radius", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("pairs", ctypes.c_int)]


class _Config(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int), ("height", ctypes.c_int), ("fmt", ctypes.c_int), ("bit_depth", ctypes.c_int),
        ("n_passes", ctypes.c_int), ("window", ctypes.c_int * 4), ("overlap", ctypes.c_float * 4),
        ("search_radius", ctypes.c_int * 4), ("predictor_levels", ctypes.c_int),
        ("uod_threshold", ctypes.c_float), ("uod_eps", ctypes.c_float), ("replace_outliers", ctypes.c_int),
        ("precision", ctypes.c_int), ("deform_mode", ctypes.c_int), ("max_batch", ctypes.c_int),
        ("host_frames", ctypes.c_int),
    ]


_lib = None


def load(path: str = LIB_PATH):
    """Load librpiv.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2504_17987_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp, i32, sz, f32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_float
    cfgp = ctypes.POINTER(_Config)
    L.rpiv_last_error.restype = ctypes.c_char_p
    L.rpiv_last_error.argtypes = []
    L.rpiv_config_default.argtypes = [cfgp]
    L.rpiv_validate_config.argtypes = [cfgp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.rpiv_create.argtypes = [cfgp, i32, ctypes.POINTER(vp)]
    L.rpiv_grid_shape.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.rpiv_workspace_bytes.argtypes = [vp, ctypes.POINTER(sz)]
    L.rpiv_process_pair.argtypes = [vp, vp, vp, sz, vp, vp, vp, vp, vp, vp, vp]
    pa = ctypes.POINTER(vp)
    L.rpiv_process_batch.argtypes = [vp, i32, pa, pa, sz, pa, pa, pa, pa, pa, pa, vp]
    L.rpiv_backward.argtypes = [vp, vp, vp, sz, vp, vp, f32, vp, vp, vp, vp]
    L.rpiv_refine.argtypes = [vp, vp, vp, sz, vp, vp, i32, f32, i32, ctypes.POINTER(f32), vp]
    L.rpiv_wait.argtypes = [vp, i32]
    L.rpiv_destroy.argtypes = [vp]
    L.rpiv_stage_correlate.argtypes = [vp, vp, sz, i32, i32, i32, i32, i32, i32, i32, i32, vp, vp, vp, vp, vp, vp, sz,
                                       vp]
    L.rpiv_stage_correlate_scratch_bytes.argtypes = [i32, i32, i32, i32, ctypes.POINTER(sz)]
    L.rpiv_stage_correlate_noalloc.argtypes = [vp, vp, sz, i32, i32, i32, i32, i32, i32, i32, i32, vp, vp, vp, vp,
                                               vp, vp]
    L.rpiv_stage_status.argtypes = [vp, i32]
    L.rpiv_stage_validate.argtypes = [vp, vp, vp, i32, i32, f32, f32, i32, vp, vp, vp, vp]
    L.rpiv_stage_interp.argtypes = [vp, vp, i32, i32, i32, i32, vp, vp, i32, i32, i32, i32, i32, vp]
    L.rpiv_stage_vorticity.argtypes = [vp, vp, i32, i32, i32, vp, vp]
    L.rpiv_stage_ema.argtypes = [vp, vp, sz, ctypes.c_float, i32, vp]
    L.rpiv_stage_preprocess_scratch_bytes.argtypes = [i32, i32, i32, i32, ctypes.POINTER(sz)]
    L.rpiv_stage_preprocess.argtypes = [vp, sz, i32, i32, i32, i32, i32, i32, i32, i32, vp, vp, sz, vp]
    L.rpiv_stage_downsample.argtypes = [vp, sz, i32, i32, i32, vp, vp]
    L.rpiv_trace_enable.argtypes = [vp, i32]
    L.rpiv_trace_read.argtypes = [vp, ctypes.POINTER(TraceRecord), i32, ctypes.POINTER(i32)]
    for name in EXPORTED:
        if name != "rpiv_last_error":
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(st: int):
    if st != 0:
        raise RpivError(st, load().rpiv_last_error().decode(errors="replace"))


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


@dataclasses.dataclass
class Config:
    """Mirror of rpiv_config (window/overlap/radius per full-resolution pass)."""
    width: int
    height: int
    windows: Sequence[int] = (16,)
    overlaps: Sequence[float] = (0.5,)
    radii: Sequence[int] = (1,)
    levels: int = 0
    bit_depth: int = 8
    uod_threshold: float = 2.0
    uod_eps: float = 0.1
    replace: bool = True
    precision: str = "fp32"
    deform: str = "b"
    max_batch: int = 1
    float_frames: bool = False  # frames are float32 (for example pre-processed), not u8/u16
    host_frames: bool = False   # process_pair/process_batch take page-locked host (pinned CPU) tensors

    @property
    def fmt(self) -> int:
        if self.float_frames:
            return RPIV_F32
        return RPIV_U8 if self.bit_depth == 8 else RPIV_U16

    def to_c(self) -> _Config:
        c = _Config()
        c.width, c.height = self.width, self.height
        c.fmt = self.fmt
        c.bit_depth = self.bit_depth
        n = len(self.windows)
        if not (len(self.overlaps) == len(self.radii) == n):
            raise ValueError("windows, overlaps and radii must have the same length")
        c.n_passes = n
        for i in range(min(n, 4)):
            c.window[i], c.overlap[i], c.search_radius[i] = self.windows[i], self.overlaps[i], self.radii[i]
        c.predictor_levels = self.levels
        c.uod_threshold, c.uod_eps = self.uod_threshold, self.uod_eps
        c.replace_outliers = 1 if self.replace else 0
        c.precision = PRECISIONS[self.precision]
        c.deform_mode = RPIV_DEFORM_CENTRAL if self.deform == "central" else RPIV_DEFORM_B
        c.max_batch = self.max_batch
        c.host_frames = 1 if self.host_frames else 0
        return c

    @classmethod
    def from_schedule(cls, W: int, H: int, sched, bit_depth: int = 8, **kw) -> "Config":
        return cls(width=W, height=H, windows=tuple(sched.windows), overlaps=tuple(sched.overlaps),
                   radii=tuple(sched.radii), levels=sched.levels, bit_depth=bit_depth,
                   uod_threshold=sched.uod_threshold, uod_eps=sched.uod_eps, replace=sched.replace, **kw)


def validate_config(cfg: Config) -> Tuple[int, int]:
    """Host-only check; returns the final-pass grid (nx, ny)."""
    c = cfg.to_c()
    nx, ny = ctypes.c_int(), ctypes.c_int()
    _check(load().rpiv_validate_config(ctypes.byref(c), ctypes.byref(nx), ctypes.byref(ny)))
    return nx.value, ny.value


_PTR_ARRAYS = {}


def _ptr_array(n: int):
    """ctypes array type of n pointers (one type per n, made once)."""
    t = _PTR_ARRAYS.get(n)
    if t is None:
        t = _PTR_ARRAYS[n] = ctypes.c_void_p * n
    return t


def _entry_ptrs(x, n: int):
    """Addresses of the n per-pair outputs: rows of one contiguous (n, ...)
    tensor by stride arithmetic, or the entries of a list."""
    if isinstance(x, torch.Tensor) and x.dim() >= 1 and x.shape[0] == n:
        base, step = x.data_ptr(), x.stride(0) * x.element_size()
        return [base + i * step for i in range(n)]
    return [x[i].data_ptr() for i in range(n)]


def _img_check(t: torch.Tensor, cfg_fmt: int, host: bool = False):
    if host:
        # that the memory is page-locked is checked by the library, once per
        # image (rpiv_process_batch rejects it with a status and a message);
        # a second driver query here would cost the serving loop per image
        if t.is_cuda:
            raise ValueError("a host_frames engine takes pinned CPU tensors")
    elif not t.is_cuda:
        raise ValueError("images must be CUDA tensors")
    if cfg_fmt == RPIV_F32:
        ok = t.dtype == torch.float32
    else:
        ok = not t.is_floating_point() and t.element_size() == (1 if cfg_fmt == RPIV_U8 else 2)
    if not ok:
        raise ValueError(f"image dtype {t.dtype} does not match the handle's pixel format")
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("images must be 2-D with unit column stride")


def to_device(img, device="cuda", pin: bool = False) -> torch.Tensor:
    """numpy uint8/uint16 image -> torch tensor (uint16 is carried as int16
    bits; the kernels read the raw 16-bit values as unsigned)."""
    import numpy as np
    arr = np.ascontiguousarray(img)
    if arr.dtype == np.uint16:
        arr = arr.view(np.int16)
    t = torch.from_numpy(arr)
    if pin:
        return t.pin_memory()
    return t.to(device)


class Engine:
    """Owns an rpiv handle (workspace, graphs) for one image size and schedule."""

    def __init__(self, cfg: Config, device: int = 0):
        self.cfg = cfg
        self.device = device
        L = load()
        c = cfg.to_c()
        h = ctypes.c_void_p()
        _check(L.rpiv_create(ctypes.byref(c), device, ctypes.byref(h)))
        self._h = h
        nx, ny = ctypes.c_int(), ctypes.c_int()
        _check(L.rpiv_grid_shape(h, ctypes.byref(nx), ctypes.byref(ny)))
        self.nx, self.ny = nx.value, ny.value

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("engine is closed")
        return self._h

    def workspace_bytes(self) -> int:
        b = ctypes.c_size_t()
        _check(load().rpiv_workspace_bytes(self.handle, ctypes.byref(b)))
        return b.value

    def empty_outputs(self, n: int = 1):
        """(u, v, vort, mask) for n pairs: u, v and vort are views of one float
        allocation (two allocations instead of four per call)."""
        dev = torch.device("cuda", self.device)
        shp = (n, self.ny, self.nx) if n > 1 else (self.ny, self.nx)
        f = torch.empty((3,) + shp, dtype=torch.float32, device=dev)
        return f[0], f[1], f[2], torch.empty(shp, dtype=torch.uint8, device=dev)

    def process_pair(self, a: torch.Tensor, b: torch.Tensor, pred=None, out=None, stream=None):
        """Returns (u, v, vort, mask) on the final-pass grid (asynchronous)."""
        _img_check(a, self.cfg.fmt, self.cfg.host_frames)
        _img_check(b, self.cfg.fmt, self.cfg.host_frames)
        if a.stride(0) != b.stride(0):
            raise ValueError("A and B must share the row pitch")
        u, v, w, m = out if out is not None else self.empty_outputs(1)
        pu, pv = (None, None) if pred is None else pred
        _check(load().rpiv_process_pair(self.handle, _ptr(a), _ptr(b), a.stride(0) * a.element_size(), _ptr(pu),
                                        _ptr(pv), _ptr(u), _ptr(v), _ptr(w), _ptr(m), _stream(stream)))
        return u, v, w, m

    def process_batch(self, a_list: List[torch.Tensor], b_list: List[torch.Tensor], preds=None, outs=None,
                      stream=None):
        """n pairs in one launch sequence.  outs: tuple (u, v, vort, mask) of lists
        (or (n, ny, nx) tensors); preds: list of (pu, pv) or None entries."""
        n = len(a_list)
        if n != len(b_list):
            raise ValueError("a_list and b_list differ in length")
        pitch = a_list[0].stride(0) * a_list[0].element_size()
        for t in list(a_list) + list(b_list):
            _img_check(t, self.cfg.fmt, self.cfg.host_frames)
            if t.stride(0) * t.element_size() != pitch:
                raise ValueError("all images of a batch must share the row pitch")
        if outs is None:
            outs = self.empty_outputs(n if n > 1 else 1)
            if n == 1:
                outs = tuple(o.unsqueeze(0) for o in outs)
        u, v, w, m = outs
        arr = _ptr_array(n)
        A = arr(*[t.data_ptr() for t in a_list])
        B = arr(*[t.data_ptr() for t in b_list])
        U = arr(*_entry_ptrs(u, n))
        V = arr(*_entry_ptrs(v, n))
        Wv = arr(*_entry_ptrs(w, n)) if w is not None else None
        M = arr(*_entry_ptrs(m, n)) if m is not None else None
        PU = PV = None
        if preds is not None and any(p is not None for p in preds):
            PU = arr(*[(p[0].data_ptr() if p is not None else None) for p in preds])
            PV = arr(*[(p[1].data_ptr() if p is not None else None) for p in preds])
        _check(load().rpiv_process_batch(self.handle, n, A, B, pitch, PU, PV, U, V, Wv, M, _stream(stream)))
        return u, v, w, m

    def score_and_grad(self, a: torch.Tensor, b: torch.Tensor, u: torch.Tensor, v: torch.Tensor,
                       grad_score: float = 1.0, want_grad: bool = True, stream=None):
        """S = sum_w C_w(0) on the first pass's grid and grad_score * dS/d(u, v)."""
        _img_check(a, self.cfg.fmt)
        _img_check(b, self.cfg.fmt)
        u = u.contiguous().float()
        v = v.contiguous().float()
        dev = u.device
        score = torch.empty((), dtype=torch.float32, device=dev)
        gu = torch.empty_like(u) if want_grad else None
        gv = torch.empty_like(v) if want_grad else None
        _check(load().rpiv_backward(self.handle, _ptr(a), _ptr(b), a.stride(0) * a.element_size(), _ptr(u), _ptr(v),
                                    float(grad_score), _ptr(gu), _ptr(gv), _ptr(score), _stream(stream)))
        return score, gu, gv

    def trace(self, enable: bool = True):
        """Stage tracing: eager launches bracketed by CUDA events."""
        _check(load().rpiv_trace_enable(self.handle, 1 if enable else 0))

    def trace_read(self):
        """Per-stage records since the last read (synchronises the handle's work)."""
        cap = 64
        recs = (TraceRecord * cap)()
        n = ctypes.c_int()
        _check(load().rpiv_trace_read(self.handle, recs, cap, ctypes.byref(n)))
        out = []
        for r in recs[:min(cap, n.value)]:
            out.append(dict(name=r.name.decode(), launches=r.launches, total_ms=r.total_ms, width=r.width,
                            height=r.height, window=r.window, step=r.step, radius=r.radius, nx=r.nx, ny=r.ny,
                            pairs=r.pairs))
        return out

    def wait(self, timeout_ms: int = 60000):
        _check(load().rpiv_wait(self.handle, int(timeout_ms)))

    def close(self):
        if self._h is not None:
            load().rpiv_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ stage calls --

def _fmt_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return 0
    return RPIV_U8 if t.element_size() == 1 else RPIV_U16


def stage_status(stream=None, timeout_ms: int = 10000):
    """Raises RpivError (TIMEOUT) if a stage kernel's bounded wait gave up
    since the last call, or the stream's work did not finish in time
    (rpiv_stage_status)."""
    _check(load().rpiv_stage_status(_stream(stream), int(timeout_ms)))


def stage_correlate(a, b, w: int, s: int, r: int, pred_u=None, pred_v=None, precision: str = "fp32",
                    deform: str = "b", stream=None):
    """One correlation pass; returns (u, v, info) raw (pre-validation)."""
    H, W = a.shape
    nx, ny = (W - w) // s + 1, (H - w) // s + 1
    dev = a.device
    u = _fresh(torch.empty((ny, nx), dtype=torch.float32, device=dev))
    v = _fresh(torch.empty_like(u))
    info = _fresh(torch.empty((ny, nx), dtype=torch.int32, device=dev))
    dm = RPIV_DEFORM_CENTRAL if deform == "central" else RPIV_DEFORM_B
    nbytes = ctypes.c_size_t()
    _check(load().rpiv_stage_correlate_scratch_bytes(W, H, r, dm, ctypes.byref(nbytes)))
    scratch = _fresh(torch.empty(max(1, nbytes.value), dtype=torch.uint8, device=dev))
    _check(load().rpiv_stage_correlate(_ptr(a), _ptr(b), a.stride(0) * a.element_size(), _fmt_code(a), W, H, w, s, r,
                                       PRECISIONS[precision], dm, _ptr(pred_u), _ptr(pred_v), _ptr(u), _ptr(v),
                                       _ptr(info), _ptr(scratch), nbytes.value, _stream(stream)))
    return u, v, info


def decode_info(info: torch.Tensor):
    """(valid, ky, kx) from the packed int32 pass info."""
    i = info.to(torch.int64)
    valid = (i & 1).to(torch.bool)
    ky = ((i >> 8) & 0xFF).to(torch.int8)
    kx = ((i >> 16) & 0xFF).to(torch.int8)
    return valid, ky, kx


def stage_validate(u, v, info=None, thr: float = 2.0, eps: float = 0.1, replace: bool = True, stream=None):
    ny, nx = u.shape
    uo, vo = torch.empty_like(u), torch.empty_like(v)
    mask = torch.empty((ny, nx), dtype=torch.uint8, device=u.device)
    _check(load().rpiv_stage_validate(_ptr(u), _ptr(v), _ptr(info), nx, ny, float(thr), float(eps), int(replace),
                                      _ptr(uo), _ptr(vo), _ptr(mask), _stream(stream)))
    return uo, vo, mask


def stage_interp(su, sv, sw: int, ss: int, dnx: int, dny: int, dw: int, ds: int, levels_up: int = 0, stream=None):
    sny, snx = su.shape
    du = torch.empty((dny, dnx), dtype=torch.float32, device=su.device)
    dv = torch.empty_like(du)
    _check(load().rpiv_stage_interp(_ptr(su), _ptr(sv), snx, sny, sw, ss, _ptr(du), _ptr(dv), dnx, dny, dw, ds,
                                    levels_up, _stream(stream)))
    return du, dv


def stage_vorticity(u, v, s: int, stream=None):
    ny, nx = u.shape
    o = torch.empty_like(u)
    _check(load().rpiv_stage_vorticity(_ptr(u), _ptr(v), nx, ny, s, _ptr(o), _stream(stream)))
    return o


def stage_preprocess(img, vmax: int, hp: int = 7, tiles=(8, 8), clip_pct: int = 200, stream=None, out=None,
                     scratch=None):
    """High-pass filter and CLAHE (Sec. 2) of a u8/u16 device image; returns a
    float32 image in [0, vmax] (rpiv_stage_preprocess).  out (H x W float32)
    and scratch (uint8, at least preprocess_scratch_bytes) may be supplied for
    reuse."""
    H, W = img.shape
    nbytes = preprocess_scratch_bytes(W, H, tiles)
    if scratch is None:
        scratch = _fresh(torch.empty(nbytes, dtype=torch.uint8, device=img.device))
    elif scratch.dtype != torch.uint8 or scratch.numel() < nbytes or not scratch.is_contiguous():
        raise ValueError(f"scratch: a contiguous uint8 tensor of at least {nbytes} bytes")
    if out is None:
        out = torch.empty((H, W), dtype=torch.float32, device=img.device)
    elif out.dtype != torch.float32 or tuple(out.shape) != (H, W) or not out.is_contiguous():
        raise ValueError("out: a contiguous float32 tensor of the image's shape")
    _check(load().rpiv_stage_preprocess(_ptr(img), img.stride(0) * img.element_size(), _fmt_code(img), W, H,
                                        int(vmax), int(hp), int(tiles[0]), int(tiles[1]), int(clip_pct), _ptr(out),
                                        _ptr(scratch), scratch.numel(), _stream(stream)))
    return out


def preprocess_scratch_bytes(W: int, H: int, tiles=(8, 8)) -> int:
    """Scratch bytes rpiv_stage_preprocess needs for a W x H image."""
    nbytes = ctypes.c_size_t()
    _check(load().rpiv_stage_preprocess_scratch_bytes(W, H, int(tiles[0]), int(tiles[1]), ctypes.byref(nbytes)))
    return nbytes.value


def stage_ema(x, state, alpha: float, init: bool = False, stream=None):
    """state <- x (init) or alpha x + (1 - alpha) state, in place; returns state."""
    if x.dtype != torch.float32 or state.dtype != torch.float32 or x.numel() != state.numel():
        raise ValueError("x and state: float32 tensors of the same size")
    if not (x.is_contiguous() and state.is_contiguous()):
        raise ValueError("x and state must be contiguous")
    _check(load().rpiv_stage_ema(_ptr(x), _ptr(state), x.numel(), float(alpha), 1 if init else 0, _stream(stream)))
    return state


def stage_downsample(img, stream=None):
    H, W = img.shape
    out = torch.empty((H // 2, W // 2), dtype=torch.float32, device=img.device)
    _check(load().rpiv_stage_downsample(_ptr(img), img.stride(0) * img.element_size(), _fmt_code(img), W, H, _ptr(out),
                                        _stream(stream)))
    return out


# ------------------------------------------------------- differentiation --

class CorrelationScore(torch.autograd.Function):
    """S(u, v) = sum over windows of the zero-shift correlation coefficient
    between A and B warped by the grid field (u, v); backward runs the
    library's adjoint kernels (deformed windows recomputed, not stored)."""

    @staticmethod
    def forward(ctx, u, v, engine: Engine, a, b):
        score, _, _ = engine.score_and_grad(a, b, u.detach(), v.detach(), want_grad=False)
        ctx.engine = engine
        ctx.save_for_backward(u.detach(), v.detach(), a, b)
        return score

    @staticmethod
    def backward(ctx, grad_out):
        u, v, a, b = ctx.saved_tensors
        # grad_out is a 0-d device tensor; the adjoint scales by a host float
        g = float(grad_out.detach().cpu())
        _, gu, gv = ctx.engine.score_and_grad(a, b, u, v, grad_score=g, want_grad=True)
        return gu, gv, None, None, None


def refine(engine: Engine, a, b, u0, v0, steps: int = 5, eta0: float = 0.25, halvings: int = 3, stream=None):
    """Gradient-ascent refinement of the correlation score (rpiv_refine): eta_k
    = eta0 0.5^k / max|g0| along the current gradient, a step kept only if S
    increases, else eta halved up to `halvings` times.  Returns (u, v,
    [S at the start and after each step])."""
    _img_check(a, engine.cfg.fmt)
    _img_check(b, engine.cfg.fmt)
    u = u0.detach().clone().float().contiguous()
    v = v0.detach().clone().float().contiguous()
    hist = (ctypes.c_float * (steps + 1))()
    _check(load().rpiv_refine(engine.handle, _ptr(a), _ptr(b), a.stride(0) * a.element_size(), _ptr(u), _ptr(v),
                              int(steps), float(eta0), int(halvings), hist, _stream(stream)))
    return u, v, [float(x) for x in hist]
