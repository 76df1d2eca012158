"""Named synthetic workloads: image recipe, analytic flow and processing schedule.

Each workload mirrors one of the configurations the method is evaluated on
(uniform motion plus a Lamb-Oseen vortex, a paper-scale 12-bit pair with a
shear layer and out-of-plane loss, the differentiation case, the 8 MP
Fourier-mode case and the serving mix).  The schedule entries are plain
processing parameters (window, overlap, search radius, passes, pyramid
levels), handed unchanged to whichever implementation runs.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Tuple

import numpy as np

from . import Flow, ImageSpec, render_pair, uniform


@dataclasses.dataclass
class Schedule:
    windows: Tuple[int, ...]
    overlaps: Tuple[float, ...]
    radii: Tuple[int, ...]
    levels: int = 0
    uod_threshold: float = 2.0
    uod_eps: float = 0.1
    replace: bool = True

    def as_dict(self) -> Dict:
        return dataclasses.asdict(self)


@dataclasses.dataclass
class Workload:
    name: str
    spec: ImageSpec
    flow: Flow
    schedule: Schedule

    def render(self):
        return render_pair(self.spec, self.flow)


def plain_256(seed: int = 1001) -> Workload:
    """256x256 u8, 0.05 ppp, d_p 2.5, uniform (3.3, -1.7) + centred Lamb-Oseen
    vortex (Gamma 200 px^2/frame, rc 20); one pass of 32 px windows, 50 %
    overlap, search +-8, zero predictor (15 x 15 vectors)."""
    spec = ImageSpec(W=256, H=256, bit_depth=8, ppp=0.05, dp=(2.5, 2.5), i0=(150, 255),
                     noise_frac=0.02, seed=seed)
    flow = Flow(U=3.3, V=-1.7, vortices=[(127.5, 127.5, 200.0, 20.0)])
    return Workload("plain_256_u8", spec, flow, Schedule((32,), (0.5,), (8,), levels=0))


def paper_1mp(seed: int = 1002, W: int = 1024, H: int = 1024) -> Workload:
    """1024x1024 12-bit (uint16), 0.03 ppp, d_p U(2,4), 10 % of particles
    replaced between frames; uniform 12 px + tanh shear layer (dU 6, delta 10,
    max gradient 0.3 px/px) at y = 0.35 H + Lamb-Oseen vortex at (0.5 W, 0.65 H);
    three passes 64 -> 32 -> 16 at 50 %, search +-4, 2-level predictor pyramid
    (127 x 127 vectors)."""
    spec = ImageSpec(W=W, H=H, bit_depth=12, ppp=0.03, dp=(2.0, 4.0), i0=(150, 255),
                     noise_frac=0.02, loss_frac=0.10, seed=seed)
    flow = Flow(U=12.0, V=0.0, vortices=[(0.5 * W, 0.65 * H, 200.0, 20.0)],
                shear=(6.0, 0.35 * H, 10.0))
    return Workload("paper_1mp_u16", spec, flow,
                    Schedule((64, 32, 16), (0.5, 0.5, 0.5), (4, 4, 4), levels=2))


def paper_1mp_r1(seed: int = 1002) -> Workload:
    """The paper's own operating point at 1 MP: 16 px windows, 50 % step,
    a +-1 search (the 5-point stencil around the predicted peak), 2-level
    predictor pyramid feeding a 32 -> 16 schedule."""
    w = paper_1mp(seed)
    return Workload("paper_1mp_16px_r1", w.spec, w.flow,
                    Schedule((32, 16), (0.5, 0.5), (4, 1), levels=2))


def diff_1mp(seed: int = 1003) -> Workload:
    """1024x1024 u8 with the plain_256 recipe; 32 px windows at 75 % overlap
    (125 x 125 vectors), search +-8: the field the score gradient is taken on."""
    spec = ImageSpec(W=1024, H=1024, bit_depth=8, ppp=0.05, dp=(2.5, 2.5), i0=(150, 255),
                     noise_frac=0.02, seed=seed)
    flow = Flow(U=3.3, V=-1.7, vortices=[(511.5, 511.5, 200.0, 20.0)])
    return Workload("diff_1mp_u8", spec, flow, Schedule((32,), (0.75,), (8,), levels=0))


def fourier_8mp(seed: int = 1004, W: int = 3840, H: int = 2160) -> Workload:
    """3840x2160 u8, 0.05 ppp, d_p 2.5; divergence-free field from a
    streamfunction of 8 seeded Fourier modes (integer wavevectors in [1,4]^2,
    amplitudes N(0,1), phases U(0, 2 pi)) scaled to max |d| = 16 px; passes
    48 -> 24 at 50 %, search +-6, 2-level pyramid (319 x 179 vectors)."""
    rnd = uniform(seed ^ 0x5EED, 64)
    modes = []
    for m in range(8):
        kx = 1 + int(rnd[4 * m] * 4) % 4
        ky = 1 + int(rnd[4 * m + 1] * 4) % 4
        # amplitude N(0,1) by Box-Muller from two uniforms, phase U(0, 2 pi)
        u1 = max(rnd[4 * m + 2], 1e-300)
        amp = math.sqrt(-2.0 * math.log(u1)) * math.cos(2 * math.pi * rnd[4 * m + 3])
        ph = 2 * math.pi * rnd[32 + m]
        modes.append((float(kx), float(ky), amp, ph))
    base = Flow(modes=modes, L=(float(W), float(H)))
    gx, gy = np.meshgrid(np.arange(0, W, 4.0), np.arange(0, H, 4.0))
    u, v = base.eval(gx, gy)
    scale = 16.0 / float(np.max(np.hypot(u, v)))
    modes = [(kx, ky, a * scale, ph) for (kx, ky, a, ph) in modes]
    spec = ImageSpec(W=W, H=H, bit_depth=8, ppp=0.05, dp=(2.5, 2.5), i0=(150, 255),
                     noise_frac=0.02, seed=seed)
    return Workload("fourier_8mp_u8", spec, Flow(modes=modes, L=(float(W), float(H))),
                    Schedule((48, 24), (0.5, 0.5), (6, 6), levels=2))


def uniform_shift(U: float, V: float, W: int = 256, H: int = 256, seed: int = 2001,
                  window: int = 32, radius: int = 8, bit_depth: int = 8) -> Workload:
    """Uniform displacement (U, V) on a particle pair; one pass, zero predictor."""
    spec = ImageSpec(W=W, H=H, bit_depth=bit_depth, ppp=0.05, dp=(2.5, 2.5), i0=(150, 255),
                     noise_frac=0.02, seed=seed)
    return Workload(f"uniform_{U}_{V}", spec, Flow(U=U, V=V),
                    Schedule((window,), (0.5,), (radius,), levels=0))


# serving mix: frame sizes and weights, pixel formats
SERVING_SIZES: List[Tuple[int, int, float]] = [
    (512, 512, 0.3), (1024, 1024, 0.4), (2048, 2048, 0.2), (3840, 2160, 0.1)]


def serving_stream_flow(stream: int, frame: int, W: int, H: int) -> Flow:
    """Per-stream field: uniform 4 px plus a Lamb-Oseen vortex advected by
    0.5 px per frame (wrapping across the image)."""
    rnd = uniform(0xC0FFEE + stream, 4)
    x0 = 0.25 * W + 0.5 * W * rnd[0]
    y0 = 0.25 * H + 0.5 * H * rnd[1]
    xc = (x0 + 0.5 * frame) % W
    sign = 1.0 if rnd[2] < 0.5 else -1.0
    return Flow(U=4.0, V=0.0, vortices=[(xc, y0, sign * 200.0, 20.0)])


def poisson_arrivals(n: int, rate: float, seed: int) -> List[float]:
    """Arrival times (s) of a Poisson process of the given rate: exponential
    gaps by the inverse CDF of seeded uniforms."""
    u = uniform(seed, n)
    t, out = 0.0, []
    for x in u:
        t += -math.log(max(1.0 - float(x), 1e-300)) / rate
        out.append(t)
    return out
