"""Continuous-batching server for streams of PIV image pairs.

Each camera stream delivers pairs of one size and pixel format; a stream's
previous velocity field is kept on the device and predicts its next pair
(the paper runs the optical-flow predictor per frame; a stream of smooth
flow lets the last field play that role, Sec. 2).  A stream's first pair has
no predictor and runs a cold schedule (coarse-to-fine pyramid and a 32 -> 16 px
pass pair); later pairs run a warm single 16 px pass around the predictor.
Both end on the same 16 px / 50 % grid.

Scheduling (host side, one thread):
  * arrivals enter per-stream FIFOs; a stream's head request is eligible once
    its previous request has completed (its field is the predictor);
  * eligible requests are grouped by (size, format, mode) into batches of at
    most `max_batch`, oldest head first;
  * a batch is admitted when a slot (a CUDA stream with its own engine
    handles) is free and the bytes it needs fit the HBM budget together with
    the engines' workspaces and the other batches in flight;
  * completions are detected by polling CUDA events; the latency of a request
    is arrival -> its results complete on the device.
Requests that arrive while batches run are admitted as slots and memory free
up, so work of different sizes overlaps on the device.

While a run is live the cyclic garbage collector does not run on its own: the
objects alive at the start are frozen out of its scans, and only the young
generations are collected, at moments when the loop is waiting on the device.
A full (generation-2) pass over a run's requests and tensors takes tens of
milliseconds on one host core and would otherwise stall every request
queued behind it.  The kernels treat
every pair independently (the batch index only selects data), so a request's
result does not depend on what it is batched with.

The executor is pluggable: `GpuExecutor` runs librpiv; tests drive the
scheduler with a host-only fake to exercise admission, ordering and failure
handling without a GPU.
"""
from __future__ import annotations

import collections
import dataclasses
import gc
import heapq
import math
import time
from typing import Callable, Deque, Dict, List, Optional, Sequence, Tuple

Key = Tuple[int, int, int]  # (width, height, bit_depth)

COLD, WARM = "cold", "warm"


@dataclasses.dataclass
class Request:
    rid: int
    stream: int
    frame: int
    arrival: float                 # seconds since the start of the run
    key: Key
    payload: object = None         # executor-specific input (e.g. pinned host tensors)
    mode: str = ""
    dispatched: float = math.nan
    done: float = math.nan
    result: object = None          # executor-specific output (u, v, vort, mask)
    error: Optional[str] = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclasses.dataclass
class Batch:
    key: Key
    mode: str
    requests: List[Request]
    slot: int
    nbytes: int
    token: object = None           # executor handle of the in-flight work


class Executor:
    """Interface of what runs batches.  All methods are called from the scheduler thread."""

    def engine_bytes(self, key: Key, mode: str) -> int:
        """Device bytes of one engine (handle workspace) for this key and mode."""
        raise NotImplementedError

    def request_bytes(self, key: Key) -> int:
        """Device bytes one request needs while in flight (inputs, outputs)."""
        raise NotImplementedError

    def max_pairs(self, key: Key, mode: str) -> int:
        """Largest batch one engine of this key and mode takes."""
        raise NotImplementedError

    def drop_engine(self, key: Key, mode: str, slot: int) -> None:
        """Release an idle engine (its workspace)."""
        raise NotImplementedError

    def submit(self, slot: int, key: Key, mode: str, reqs: Sequence[Request], preds: Sequence[object]) -> object:
        """Enqueue the batch asynchronously; returns a token for poll()."""
        raise NotImplementedError

    def poll(self, token: object) -> bool:
        """True once the batch's results are complete."""
        raise NotImplementedError

    def collect(self, token: object, reqs: Sequence[Request]) -> None:
        """Attach results to the requests (after poll() returned True)."""
        raise NotImplementedError

    def field_of(self, req: Request) -> object:
        """The request's result in the form submit() takes as a predictor."""
        raise NotImplementedError


class Scheduler:
    def __init__(self, executor: Executor, max_batch: int = 64, slots: int = 4, hbm_budget: float = 40e9,
                 clock: Callable[[], float] = time.perf_counter):
        if max_batch < 1 or slots < 1:
            raise ValueError("max_batch and slots must be >= 1")
        self.ex = executor
        self.max_batch = max_batch
        self.slots = slots
        self.budget = float(hbm_budget)
        self.clock = clock
        self.fifo: Dict[int, Deque[Request]] = collections.defaultdict(collections.deque)
        self.prev_field: Dict[int, object] = {}
        self.busy_stream: Dict[int, bool] = collections.defaultdict(bool)
        self.failed_streams: set = set()
        self.in_flight: List[Batch] = []
        self.free_slots = list(range(slots))
        self.engines: Dict[Tuple[Key, str, int], List] = {}  # (key, mode, slot) -> [bytes, last use]
        self.used = 0.0
        self.done: List[Request] = []
        self.dropped: List[Request] = []
        self.t0 = 0.0
        self.batches = 0
        self.host_busy = 0.0           # seconds of loop iterations that completed or started work

    # ---------------------------------------------------------- accounting --
    def _engine_charge(self, key: Key, mode: str, slot: int) -> int:
        return 0 if (key, mode, slot) in self.engines else self.ex.engine_bytes(key, mode)

    def _fits(self, key: Key, mode: str, slot: int, n: int, evict: bool = False) -> bool:
        need = self._engine_charge(key, mode, slot) + n * self.ex.request_bytes(key)
        if self.used + need <= self.budget:
            return True
        if not evict:
            return False
        # free idle engines, least recently used first
        busy = {(b.key, b.mode, b.slot) for b in self.in_flight}
        idle = sorted((v[1], k) for k, v in self.engines.items() if k not in busy and k != (key, mode, slot))
        for _, k in idle:
            self.used -= self.engines.pop(k)[0]
            self.ex.drop_engine(*k)
            if self.used + need <= self.budget:
                return True
        return False

    # ----------------------------------------------------------- lifecycle --
    def mark_stream_failed(self, stream: int, reason: str = "stream failed"):
        """Host-side failure of a stream: its queued requests are dropped and
        no new ones of it are admitted; batches in flight finish normally."""
        self.failed_streams.add(stream)
        q = self.fifo.get(stream)
        while q:
            r = q.popleft()
            r.error = reason
            self.dropped.append(r)

    def _eligible(self) -> Dict[Tuple[Key, str], List[Request]]:
        groups: Dict[Tuple[Key, str], List[Request]] = collections.defaultdict(list)
        for s, q in self.fifo.items():
            if not q or self.busy_stream[s] or s in self.failed_streams:
                continue
            r = q[0]
            r.mode = WARM if s in self.prev_field else COLD
            groups[(r.key, r.mode)].append(r)
        return groups

    def _dispatch(self, now: float) -> bool:
        if not self.free_slots:
            return False
        groups = self._eligible()
        if not groups:
            return False
        # oldest head first
        order = sorted(groups.items(), key=lambda kv: min(r.arrival for r in kv[1]))
        started = False
        for (key, mode), reqs in order:
            if not self.free_slots:
                break
            reqs.sort(key=lambda r: r.arrival)
            slot = self.free_slots[0]
            n = min(len(reqs), self.max_batch, self.ex.max_pairs(key, mode))
            while n > 0 and not self._fits(key, mode, slot, n, evict=(n == 1)):
                n //= 2
            if n == 0:
                continue
            take = reqs[:n]
            for r in take:
                self.fifo[r.stream].popleft()
                self.busy_stream[r.stream] = True
                r.dispatched = now
            preds = [self.prev_field.get(r.stream) if mode == WARM else None for r in take]
            if (key, mode, slot) not in self.engines:
                self.engines[(key, mode, slot)] = [self.ex.engine_bytes(key, mode), now]
                self.used += self.engines[(key, mode, slot)][0]
            self.engines[(key, mode, slot)][1] = now
            nbytes = n * self.ex.request_bytes(key)
            self.used += nbytes
            self.free_slots.pop(0)
            b = Batch(key, mode, take, slot, nbytes)
            b.token = self.ex.submit(slot, key, mode, take, preds)
            self.in_flight.append(b)
            self.batches += 1
            started = True
        return started

    def _complete(self, now_fn: Callable[[], float]) -> bool:
        finished = False
        still = []
        for b in self.in_flight:
            if self.ex.poll(b.token):
                t = now_fn()
                self.ex.collect(b.token, b.requests)
                for r in b.requests:
                    r.done = t
                    self.busy_stream[r.stream] = False
                    if r.error is None:
                        self.prev_field[r.stream] = self.ex.field_of(r)
                    self.done.append(r)
                self.used -= b.nbytes
                self.free_slots.append(b.slot)
                self.free_slots.sort()
                finished = True
            else:
                still.append(b)
        self.in_flight = still
        return finished

    def run(self, requests: Sequence[Request], realtime: bool = True, on_idle: Callable[[], None] = None,
            young_gc_at: int = 700) -> dict:
        """Serve all requests.  realtime: arrivals follow the wall clock;
        otherwise every request is available at once (saturation run).
        young_gc_at: allocations since the last young collection after which
        an idle loop iteration collects generations 0 and 1 (0: the
        collector is left as it is)."""
        arrivals = sorted(requests, key=lambda r: r.arrival)
        heap = [(r.arrival, r.rid, r) for r in arrivals]
        heapq.heapify(heap)
        pause_gc = young_gc_at > 0
        was_enabled = gc.isenabled()
        if pause_gc:
            gc.collect()
            gc.freeze()
            gc.disable()
        try:
            self.t0 = self.clock()
            now_fn = lambda: self.clock() - self.t0  # noqa: E731
            total = len(arrivals)
            while len(self.done) + len(self.dropped) < total:
                now = now_fn()
                while heap and (not realtime or heap[0][0] <= now):
                    _, _, r = heapq.heappop(heap)
                    if not realtime:
                        r.arrival = min(r.arrival, now)
                    if r.stream in self.failed_streams:
                        r.error = "stream failed"
                        self.dropped.append(r)
                    else:
                        self.fifo[r.stream].append(r)
                t_it = self.clock()
                progressed = self._complete(now_fn)
                progressed |= self._dispatch(now_fn())
                if progressed:
                    self.host_busy += self.clock() - t_it
                else:
                    if pause_gc and gc.get_count()[0] >= young_gc_at:
                        gc.collect(1)
                    if on_idle is not None:
                        on_idle()
            wall = now_fn()
        finally:
            if pause_gc:
                gc.unfreeze()
                if was_enabled:
                    gc.enable()
        return self.report(wall)

    def report(self, wall: float) -> dict:
        lat = sorted(r.latency for r in self.done if r.error is None)
        def pct(p):
            if not lat:
                return math.nan
            return lat[min(len(lat) - 1, int(math.ceil(p / 100.0 * len(lat))) - 1)]
        return {"requests": len(self.done), "dropped": len(self.dropped), "wall_s": wall,
                "pairs_per_s": len(self.done) / wall if wall > 0 else math.nan,
                "p50_ms": 1000 * pct(50), "p99_ms": 1000 * pct(99), "max_ms": 1000 * (lat[-1] if lat else math.nan),
                "batches": self.batches, "mean_batch": len(self.done) / max(1, self.batches),
                "host_busy_frac": self.host_busy / wall if wall > 0 else math.nan,
                "host_us_per_batch": 1e6 * self.host_busy / max(1, self.batches)}


# ------------------------------------------------------------- GPU executor --

def warm_config(W: int, H: int, bits: int, precision: str = "fp32", max_batch: int = 64, host_frames: bool = False):
    from .binding import Config
    return Config(W, H, windows=(16,), overlaps=(0.5,), radii=(4,), levels=0, bit_depth=bits,
                  precision=precision, max_batch=max_batch, host_frames=host_frames)


def cold_config(W: int, H: int, bits: int, precision: str = "fp32", max_batch: int = 64, host_frames: bool = False):
    from .binding import Config
    return Config(W, H, windows=(32, 16), overlaps=(0.5, 0.5), radii=(4, 4), levels=2, bit_depth=bits,
                  precision=precision, max_batch=max_batch, host_frames=host_frames)


class GpuExecutor(Executor):
    """Runs batches with librpiv; one engine per (key, mode, slot) and one
    CUDA stream per slot, so batches in different slots overlap."""

    def __init__(self, slots: int, precision: str = "fp32", max_batch: int = 64, cold_batch: int = 8,
                 device: int = 0, max_megapixels: float = 16.0, prewarm: bool = False, alpha1=None, alpha2=None,
                 host_frames: bool = True):
        import torch
        self.torch = torch
        self.precision = precision
        # requests carry pinned host frames: the engines read them with their
        # upload kernel (inside the captured graph) instead of one copy call
        # per image from this thread, which bounds how many batches a second
        # the scheduler can start
        self.host_frames = host_frames
        self.max_batch = max_batch
        self.cold_batch = cold_batch
        # pixels per launch are capped so that a batch of large frames holds
        # the GPU for about as long as a batch of small ones (tail latency)
        self.max_megapixels = max_megapixels
        # capture every batch size's graph when an engine is created, so that
        # no request waits for a first-use capture
        self.prewarm = prewarm
        # exponential smoothing in time (paper Sec. 2): alpha1 on the field a
        # stream passes on as its next predictor, alpha2 on the field it
        # outputs; None leaves the field as measured
        self.alpha1 = alpha1
        self.alpha2 = alpha2
        self.pred_state = {}
        self.out_state = {}
        self.device = device
        self.streams = [torch.cuda.Stream(device=device) for _ in range(slots)]
        self.slot_events = [torch.cuda.Event() for _ in range(slots)]
        self.engines = {}

    def max_pairs(self, key: Key, mode: str) -> int:
        cap = self.cold_batch if mode == COLD else self.max_batch
        mp = key[0] * key[1] / 1e6
        return max(1, min(cap, int(self.max_megapixels // mp)))

    def _cfg(self, key: Key, mode: str):
        W, H, bits = key
        f = warm_config if mode == WARM else cold_config
        return f(W, H, bits, self.precision, self.max_pairs(key, mode), self.host_frames)

    def drop_engine(self, key: Key, mode: str, slot: int) -> None:
        e = self.engines.pop((key, mode, slot), None)
        if e is not None:
            e.close()

    def _engine(self, key: Key, mode: str, slot: int):
        from .binding import Engine
        k = (key, mode, slot)
        if k not in self.engines:
            eng = Engine(self._cfg(key, mode), device=self.device)
            self.engines[k] = eng
            if self.prewarm:
                self._prewarm(eng, key, mode, slot)
        return self.engines[k]

    def _prewarm(self, eng, key: Key, mode: str, slot: int):
        torch = self.torch
        W, H, bits = key
        dt = torch.uint8 if bits == 8 else torch.int16
        st = self.streams[slot]
        with torch.cuda.stream(st):
            a = (torch.zeros((H, W), dtype=dt).pin_memory() if self.host_frames
                 else torch.zeros((H, W), dtype=dt, device=self.device))
            pu = torch.zeros((eng.ny, eng.nx), dtype=torch.float32, device=self.device)
            for n in range(1, self.max_pairs(key, mode) + 1):
                outs = eng.empty_outputs(n)
                if n == 1:
                    outs = tuple(o.unsqueeze(0) for o in outs)
                preds = [(pu, pu)] * n if mode == WARM else None
                eng.process_batch([a] * n, [a] * n, preds=preds, outs=outs, stream=st)
        st.synchronize()

    def engine_bytes(self, key: Key, mode: str) -> int:
        W, H, bits = key
        # workspace of the handle: warped frame with margin, the pyramid for the
        # cold schedule, per-stage fields (an upper estimate of rpiv_workspace_bytes)
        pix = (W + 48) * (H + 16)
        per_pair = 4 * pix + (2 * 4 * (W * H // 4 + W * H // 16) if mode == COLD else 0) + 64 * (W * H // 64)
        if self.host_frames:
            per_pair += 2 * (W + 16) * H * (1 if bits == 8 else 2)  # the uploaded frames
        return per_pair * self.max_pairs(key, mode)

    def request_bytes(self, key: Key) -> int:
        W, H, bits = key
        bpp = 1 if bits == 8 else 2
        nx, ny = (W - 16) // 8 + 1, (H - 16) // 8 + 1
        # device copies of the frames (unless the engine uploads them itself) and the fields
        return (0 if self.host_frames else 2 * W * H * bpp) + nx * ny * 13

    def submit(self, slot, key, mode, reqs, preds):
        torch = self.torch
        eng = self._engine(key, mode, slot)
        st = self.streams[slot]
        with torch.cuda.stream(st):
            if self.host_frames:
                a = [r.payload[0] for r in reqs]
                b = [r.payload[1] for r in reqs]
            else:
                a = [r.payload[0].to(self.device, non_blocking=True) for r in reqs]
                b = [r.payload[1].to(self.device, non_blocking=True) for r in reqs]
            outs = eng.empty_outputs(len(reqs))
            if len(reqs) == 1:
                outs = tuple(o.unsqueeze(0) for o in outs)
            p = list(preds) if mode == WARM else None
            if p is not None:
                for pr in p:
                    # produced on another slot's stream: keep the memory for this one
                    pr[0].record_stream(st)
                    pr[1].record_stream(st)
            eng.process_batch(a, b, preds=p, outs=outs, stream=st)
            smoothed = self._smooth(reqs, outs, st)
            # one event per slot: a slot runs one batch at a time, so its event
            # is free again once the batch it marked has been polled complete
            ev = self.slot_events[slot]
            ev.record(st)
        return (ev, outs, a, b, p, smoothed)

    def _smooth(self, reqs, outs, st):
        """Per request: the next predictor alpha1 x + (1 - alpha1) previous
        predictor (from a copy of the measured field), then the output
        alpha2 x + (1 - alpha2) previous output, in place; a stream's first
        frame starts both states."""
        from .binding import stage_ema
        preds = []
        for i, r in enumerate(reqs):
            nxt = None
            if self.alpha1 is not None:
                nxt = (outs[0][i].clone(), outs[1][i].clone())
                prev = self.pred_state.get(r.stream)
                if prev is not None:
                    for k in range(2):
                        prev[k].record_stream(st)
                        stage_ema(prev[k], nxt[k], 1.0 - self.alpha1, stream=st)
            preds.append(nxt)
            if self.alpha2 is not None:
                prev = self.out_state.get(r.stream)
                if prev is not None:
                    for k in range(3):
                        prev[k].record_stream(st)
                        stage_ema(prev[k], outs[k][i], 1.0 - self.alpha2, stream=st)
        return preds

    def poll(self, token) -> bool:
        return token[0].query()

    def collect(self, token, reqs):
        outs, smoothed = token[1], token[5]
        u, v, w, m = outs
        for i, r in enumerate(reqs):
            r.result = (u[i], v[i], w[i], m[i])
            if r.error is None:
                if self.alpha1 is not None:
                    self.pred_state[r.stream] = smoothed[i]
                if self.alpha2 is not None:
                    self.out_state[r.stream] = (u[i], v[i], w[i])

    def field_of(self, req):
        if self.alpha1 is not None and req.stream in self.pred_state:
            return self.pred_state[req.stream]
        return (req.result[0], req.result[1])

    def close(self):
        for e in self.engines.values():
            e.close()
        self.engines.clear()
