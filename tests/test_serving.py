"""Continuous-batching scheduler: host logic with a fake executor (CPU), and
the GPU executor's alone-vs-in-the-mix equality."""
import math

import numpy as np
import pytest

from paper_2504_17987_gb300 import serving as sv
from synth import workloads as wl


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeExecutor(sv.Executor):
    """Completes a batch after `polls` polls; records everything it sees."""

    def __init__(self, clock, polls=3, eng_bytes=100, req_bytes=10, max_pairs=8, fail_submit_stream=None):
        self.clock = clock
        self.polls = polls
        self.eng_bytes = eng_bytes
        self.req_bytes = req_bytes
        self.maxp = max_pairs
        self.submitted = []
        self.dropped_engines = []
        self.n = 0
        self.fail_submit_stream = fail_submit_stream

    def engine_bytes(self, key, mode):
        return self.eng_bytes

    def request_bytes(self, key):
        return self.req_bytes

    def max_pairs(self, key, mode):
        return self.maxp

    def drop_engine(self, key, mode, slot):
        self.dropped_engines.append((key, mode, slot))

    def submit(self, slot, key, mode, reqs, preds):
        self.n += 1
        self.submitted.append((slot, key, mode, [r.rid for r in reqs], list(preds)))
        return {"left": self.polls, "reqs": list(reqs)}

    def poll(self, token):
        self.clock.t += 1e-4
        token["left"] -= 1
        return token["left"] <= 0

    def collect(self, token, reqs):
        for r in reqs:
            r.result = ("field", r.stream, r.frame)
            if self.fail_submit_stream is not None and r.stream == self.fail_submit_stream:
                r.error = "executor error"

    def field_of(self, req):
        return req.result


def make_requests(n_streams=5, frames=6, keys=((64, 64, 8), (96, 64, 16)), rate=2000.0):
    arr = wl.poisson_arrivals(n_streams * frames, rate, seed=11)
    reqs, k = [], 0
    for f in range(frames):
        for s in range(n_streams):
            reqs.append(sv.Request(rid=k, stream=s, frame=f, arrival=arr[k], key=keys[s % len(keys)]))
            k += 1
    return reqs


def run(ex, clock, reqs, **kw):
    sch = sv.Scheduler(ex, clock=clock, **kw)
    rep = sch.run(reqs, realtime=True, on_idle=lambda: setattr(clock, "t", clock.t + 1e-4))
    return sch, rep


def test_every_request_served_in_stream_order_cold_then_warm():
    clock = FakeClock()
    ex = FakeExecutor(clock)
    reqs = make_requests()
    sch, rep = run(ex, clock, reqs, max_batch=4, slots=2, hbm_budget=1e9)
    assert rep["requests"] == len(reqs) and rep["dropped"] == 0
    by_stream = {}
    for r in sorted(sch.done, key=lambda r: r.dispatched):
        by_stream.setdefault(r.stream, []).append(r)
    for s, rs in by_stream.items():
        assert [r.frame for r in rs] == sorted(r.frame for r in rs)
        # a frame is dispatched only after the previous one completed
        for a, b in zip(rs, rs[1:]):
            assert b.dispatched >= a.done
        assert rs[0].mode == sv.COLD and all(r.mode == sv.WARM for r in rs[1:])
    # warm batches get the previous result of each stream as predictor
    for slot, key, mode, rids, preds in ex.submitted:
        assert len(rids) <= 4
        if mode == sv.WARM:
            for rid, p in zip(rids, preds):
                r = reqs[rid]
                assert p == ("field", r.stream, r.frame - 1)
        else:
            assert all(p is None for p in preds)
    assert math.isfinite(rep["p99_ms"]) and rep["p99_ms"] >= rep["p50_ms"]


def test_batches_are_homogeneous_and_respect_slots():
    clock = FakeClock()
    ex = FakeExecutor(clock, polls=5)
    reqs = make_requests(n_streams=9, frames=3)
    sch, rep = run(ex, clock, reqs, max_batch=3, slots=2, hbm_budget=1e9)
    for slot, key, mode, rids, _ in ex.submitted:
        assert slot in (0, 1)
        assert all(reqs[i].key == key for i in rids)
        assert len(rids) <= 3


def test_hbm_budget_is_never_exceeded_and_engines_are_evicted():
    clock = FakeClock()
    # budget for one engine and a handful of requests: keys must take turns
    ex = FakeExecutor(clock, eng_bytes=100, req_bytes=10)
    reqs = make_requests(n_streams=4, frames=4)
    sch = sv.Scheduler(ex, max_batch=8, slots=2, hbm_budget=150, clock=clock)
    peak = [0.0]
    orig = sch._dispatch

    def watch(now):
        r = orig(now)
        peak[0] = max(peak[0], sch.used)
        return r
    sch._dispatch = watch
    rep = sch.run(reqs, on_idle=lambda: setattr(clock, "t", clock.t + 1e-4))
    assert rep["requests"] == len(reqs)
    assert peak[0] <= 150
    assert ex.dropped_engines, "a second key cannot run without evicting the first key's engine"


def test_failed_stream_is_dropped_and_others_complete():
    clock = FakeClock()
    ex = FakeExecutor(clock)
    reqs = make_requests(n_streams=4, frames=5)
    sch = sv.Scheduler(ex, max_batch=4, slots=2, hbm_budget=1e9, clock=clock)
    fired = [False]

    def idle():
        clock.t += 1e-4
        if not fired[0] and len(sch.done) >= 6:
            sch.mark_stream_failed(2, "camera disconnected")
            fired[0] = True
    rep = sch.run(reqs, on_idle=idle)
    assert fired[0]
    assert rep["requests"] + rep["dropped"] == len(reqs)
    assert rep["dropped"] > 0
    assert all(r.stream == 2 and r.error for r in sch.dropped)
    for s in (0, 1, 3):
        assert sum(1 for r in sch.done if r.stream == s) == 5


def test_executor_error_keeps_the_old_predictor():
    clock = FakeClock()
    ex = FakeExecutor(clock, fail_submit_stream=1)
    reqs = make_requests(n_streams=2, frames=3)
    sch, rep = run(ex, clock, reqs, max_batch=2, slots=1, hbm_budget=1e9)
    errs = [r for r in sch.done if r.error]
    assert errs and all(r.stream == 1 for r in errs)
    # stream 1 never produced a field, so every frame of it ran cold
    assert all(r.mode == sv.COLD for r in sch.done if r.stream == 1)


def test_collector_paused_during_run_and_restored_after():
    import gc
    clock = FakeClock()
    ex = FakeExecutor(clock)
    reqs = make_requests(n_streams=3, frames=4)
    sch = sv.Scheduler(ex, max_batch=4, slots=2, hbm_budget=1e9, clock=clock)
    seen = {"enabled": set(), "young": 0}

    def idle():
        clock.t += 1e-4
        seen["enabled"].add(gc.isenabled())
        # garbage with reference cycles, so young collections have work
        for _ in range(50):
            a = []
            a.append(a)
        if gc.get_count()[0] < 5:
            seen["young"] += 1
    assert gc.isenabled()
    rep = sch.run(reqs, on_idle=idle, young_gc_at=100)
    assert rep["requests"] == len(reqs)
    assert seen["enabled"] == {False}
    assert seen["young"] > 0            # young generations were collected at idle
    assert gc.isenabled() and gc.get_freeze_count() == 0

    # young_gc_at=0 leaves the collector alone
    seen["enabled"].clear()
    sv.Scheduler(ex, max_batch=4, slots=2, hbm_budget=1e9, clock=clock).run(
        make_requests(n_streams=2, frames=2), on_idle=idle, young_gc_at=0)
    assert seen["enabled"] == {True}


def test_collector_restored_when_the_executor_raises():
    import gc

    class Boom(FakeExecutor):
        def submit(self, *a):
            raise RuntimeError("device lost")
    clock = FakeClock()
    with pytest.raises(RuntimeError):
        sv.Scheduler(Boom(clock), clock=clock).run(make_requests(n_streams=1, frames=1), realtime=False)
    assert gc.isenabled() and gc.get_freeze_count() == 0


# ------------------------------------------------------------------- GPU --

@pytest.mark.gpu
def test_gpu_mix_results_equal_alone_results():
    import torch
    import paper_2504_17987_gb300 as rp
    from paper_2504_17987_gb300 import build
    build.build()
    sizes = [(256, 256, 8), (320, 256, 16), (256, 192, 8)]
    n_streams, frames = 6, 3
    payload = {}
    reqs, k = [], 0
    arr = wl.poisson_arrivals(n_streams * frames, 400.0, seed=5)
    for f in range(frames):
        for s in range(n_streams):
            W, H, bits = sizes[s % len(sizes)]
            flow = wl.serving_stream_flow(s, f, W, H)
            import synth
            spec = synth.ImageSpec(W=W, H=H, bit_depth=bits, ppp=0.05, dp=(2.5, 2.5), seed=9000 + 97 * s + f)
            A, B = synth.render_pair(spec, flow)
            payload[k] = (rp.to_device(A, pin=True), rp.to_device(B, pin=True))
            reqs.append(sv.Request(rid=k, stream=s, frame=f, arrival=arr[k], key=(W, H, bits), payload=payload[k]))
            k += 1
    ex = sv.GpuExecutor(slots=3, precision="bf16", max_batch=8, cold_batch=4)
    sch = sv.Scheduler(ex, max_batch=8, slots=3, hbm_budget=4e9)
    # saturation: every request is available at once, so batches mix streams
    rep = sch.run(reqs, realtime=False)
    torch.cuda.synchronize()
    assert rep["requests"] == len(reqs) and rep["dropped"] == 0
    assert rep["mean_batch"] > 1.0  # requests were actually batched together
    # alone: each request again, by itself, with the predictor it had in the mix
    by_id = {r.rid: r for r in sch.done}
    for r in sch.done:
        W, H, bits = r.key
        cfg = (sv.warm_config if r.mode == sv.WARM else sv.cold_config)(W, H, bits, "bf16", 1)
        eng = rp.Engine(cfg)
        pred = None
        if r.mode == sv.WARM:
            prev = [q for q in sch.done if q.stream == r.stream and q.frame == r.frame - 1][0]
            pred = (prev.result[0], prev.result[1])
        a = r.payload[0].cuda()
        b = r.payload[1].cuda()
        u, v, w, m = eng.process_pair(a, b, pred=pred)
        torch.cuda.synchronize()
        assert torch.equal(u, r.result[0]) and torch.equal(v, r.result[1]), r.rid
        assert torch.equal(w, r.result[2]) and torch.equal(m, r.result[3]), r.rid
        eng.close()
    ex.close()


@pytest.mark.gpu
def test_gpu_temporal_smoothing_follows_the_recurrence():
    """alpha1 on the predictor a stream passes on, alpha2 on its output: the
    served fields equal the recurrence run frame by frame through the engine."""
    import torch
    import paper_2504_17987_gb300 as rp
    import synth
    from paper_2504_17987_gb300 import build
    build.build()
    W, H, bits = 256, 256, 8
    n_streams, frames, a1, a2 = 3, 4, 0.5, 0.25
    reqs, k = [], 0
    for f in range(frames):
        for s in range(n_streams):
            spec = synth.ImageSpec(W=W, H=H, bit_depth=bits, ppp=0.05, dp=(2.5, 2.5), seed=9100 + 31 * s + f)
            A, B = synth.render_pair(spec, wl.serving_stream_flow(s, f, W, H))
            reqs.append(sv.Request(rid=k, stream=s, frame=f, arrival=0.0, key=(W, H, bits),
                                   payload=(rp.to_device(A, pin=True), rp.to_device(B, pin=True))))
            k += 1
    ex = sv.GpuExecutor(slots=2, precision="fp32", max_batch=4, cold_batch=2, alpha1=a1, alpha2=a2)
    sch = sv.Scheduler(ex, max_batch=4, slots=2, hbm_budget=4e9)
    rep = sch.run(reqs, realtime=False)
    torch.cuda.synchronize()
    assert rep["requests"] == len(reqs)
    for s in range(n_streams):
        mine = sorted((r for r in sch.done if r.stream == s), key=lambda r: r.frame)
        pred = out = None
        for r in mine:
            cfg = (sv.warm_config if r.mode == sv.WARM else sv.cold_config)(W, H, bits, "fp32", 1)
            eng = rp.Engine(cfg)
            raw = [t.clone() for t in eng.process_pair(r.payload[0].cuda(), r.payload[1].cuda(), pred=pred)]
            torch.cuda.synchronize()
            eng.close()
            new_pred = (raw[0].clone(), raw[1].clone())
            if pred is not None:
                new_pred = (a1 * raw[0] + (1 - a1) * pred[0], a1 * raw[1] + (1 - a1) * pred[1])
            new_out = raw[:3] if out is None else [a2 * raw[i] + (1 - a2) * out[i] for i in range(3)]
            for i in range(3):
                assert torch.allclose(r.result[i], new_out[i], rtol=1e-5, atol=1e-5), (s, r.frame, i)
            pred, out = new_pred, new_out
    ex.close()
