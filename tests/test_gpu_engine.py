"""Engine behaviour on the GPU that the parity tests do not cover: the host
watchdog of rpiv_wait, the error word of the kernels' bounded waits, and
graph replay against the eager first call."""
import numpy as np
import pytest
import torch

import paper_2504_17987_gb300 as rp
from paper_2504_17987_gb300 import binding
from synth import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2504_17987_gb300 import build
    build.build()


def _engine_and_pair():
    wk = wl.plain_256(seed=6001)
    A, B = wk.render()
    cfg = rp.Config.from_schedule(256, 256, wk.schedule, bit_depth=8, max_batch=4)
    return rp.Engine(cfg), rp.to_device(A), rp.to_device(B)


def test_wait_times_out_on_work_in_flight_then_completes():
    eng, a, b = _engine_and_pair()
    eng.process_pair(a, b)  # first call: eager run and graph capture
    torch.cuda.synchronize()
    # a bounded ~0.1 s spin ahead of the graph replay on the same stream keeps the work in flight
    torch.cuda._sleep(200_000_000)
    u, v, w, m = eng.process_pair(a, b)
    with pytest.raises(binding.RpivError) as ei:
        eng.wait(0)
    assert ei.value.status == 5  # RPIV_ERR_TIMEOUT
    eng.wait(60_000)  # the same work completes; no error word was set
    assert bool(torch.isfinite(u).all()) and bool((m <= 1).all())
    eng.close()


def test_graph_replay_equals_the_eager_first_call():
    eng, a, b = _engine_and_pair()
    first = [t.clone() for t in eng.process_pair(a, b)]
    torch.cuda.synchronize()
    for _ in range(3):
        again = eng.process_pair(a, b)
    torch.cuda.synchronize()
    for x, y in zip(first, again):
        assert torch.equal(x, y)
    eng.close()


def test_batch_of_distinct_pairs_equals_pairs_one_by_one():
    wk = wl.plain_256()
    pairs = [wl.plain_256(seed=7000 + k).render() for k in range(3)]
    cfg = rp.Config.from_schedule(256, 256, wk.schedule, bit_depth=8, max_batch=4)
    eng = rp.Engine(cfg)
    a = [rp.to_device(p[0]) for p in pairs]
    b = [rp.to_device(p[1]) for p in pairs]
    outs = eng.process_batch(a, b)
    torch.cuda.synchronize()
    batch = [[t[k].clone() for t in outs] for k in range(3)] if outs[0].dim() == 3 else None
    for k in range(3):
        single = eng.process_pair(a[k], b[k])
        torch.cuda.synchronize()
        got = batch[k] if batch is not None else [outs[j][k] for j in range(4)]
        for x, y in zip(got, single):
            assert torch.equal(x, y)
    eng.close()


@pytest.mark.parametrize("stall,precision,tc", [(1, "fp32", "0"), (1, "bf16", "0"), (1, "bf16", "1"),
                                               (2, "bf16", "1")])
def test_stage_bounded_wait_runs_out_and_is_reported(stall, precision, tc, monkeypatch):
    """A stage kernel's bounded wait made to run out (the test hook waits on a
    barrier phase that nothing completes, after the region copies have landed
    or before any MMA is issued): the call itself succeeds, its windows are
    reported invalid with the predictor passed through, rpiv_stage_status
    returns TIMEOUT once, and the next call is unaffected."""
    from synth import workloads as wl
    A, B = wl.paper_1mp(W=256, H=224).render()
    a, b = rp.to_device(A, "cuda:0"), rp.to_device(B, "cuda:0")
    nx, ny = (256 - 16) // 8 + 1, (224 - 16) // 8 + 1
    pu = torch.full((ny, nx), 12.0, device="cuda:0")
    pv = torch.full((ny, nx), -0.5, device="cuda:0")
    monkeypatch.setenv("RPIV_TC_PLANES", tc)  # 1: the tcgen05 kernel (stall 2 waits on its MMA barrier)
    rp.stage_status()  # start from a clear word
    monkeypatch.setenv("RPIV_DEBUG_STALL", str(stall))
    u, v, info = rp.stage_correlate(a, b, 16, 8, 4, pu, pv, precision=precision)
    torch.cuda.synchronize()
    with pytest.raises(rp.RpivError) as ei:
        rp.stage_status()
    assert ei.value.status == 5
    assert int(info.count_nonzero()) == 0
    assert torch.equal(u, pu) and torch.equal(v, pv)
    rp.stage_status()  # read once, then clear
    monkeypatch.delenv("RPIV_DEBUG_STALL")
    u, v, info = rp.stage_correlate(a, b, 16, 8, 4, pu, pv, precision=precision)
    rp.stage_status()
    valid = rp.decode_info(info)[0]
    assert float(valid.float().mean()) > 0.99


@pytest.mark.parametrize("W,H,bits,levels", [(256, 256, 8, 1), (250, 198, 12, 0)])
def test_host_frames_equal_device_frames(W, H, bits, levels):
    """An engine built with host_frames reads pinned host images through its
    upload kernel; its fields equal a device-frames engine's bit for bit, on
    the eager first call and on graph replays, with and without a predictor.
    250 x 198 u16 rows (500 bytes) are not 16-byte multiples: the upload's
    byte path."""
    import synth
    flow = synth.Flow(U=3.3, V=-1.7, vortices=[(0.5 * W, 0.5 * H, 200.0, 20.0)])
    pairs = [synth.render_pair(synth.ImageSpec(W=W, H=H, bit_depth=bits, ppp=0.05, dp=(2.5, 2.5), seed=6100 + k), flow)
             for k in range(3)]
    kw = dict(windows=(32, 16), overlaps=(0.5, 0.5), radii=(4, 4), levels=levels, bit_depth=bits, max_batch=3)
    dev_eng = rp.Engine(rp.Config(W, H, **kw))
    host_eng = rp.Engine(rp.Config(W, H, host_frames=True, **kw))
    dev = [(rp.to_device(A), rp.to_device(B)) for A, B in pairs]
    host = [(rp.to_device(A, "cpu", pin=True), rp.to_device(B, "cpu", pin=True)) for A, B in pairs]
    assert all(t.is_pinned() for p in host for t in p)
    ref = dev_eng.process_batch([p[0] for p in dev], [p[1] for p in dev])
    pred = (ref[0][0].clone(), ref[1][0].clone())
    for rep in range(2):  # eager first call, then the captured graph
        got = host_eng.process_batch([p[0] for p in host], [p[1] for p in host])
        torch.cuda.synchronize()
        for k in range(4):
            assert torch.equal(got[k], ref[k]), (rep, k)
    r1 = dev_eng.process_pair(dev[1][0], dev[1][1], pred=pred)
    g1 = host_eng.process_pair(host[1][0], host[1][1], pred=pred)
    torch.cuda.synchronize()
    for k in range(4):
        assert torch.equal(g1[k], r1[k]), k
    # device images are refused by a host_frames engine, in the binding and in the library
    with pytest.raises(ValueError):
        host_eng.process_pair(dev[0][0], dev[0][1])
    import ctypes
    u, v, w, m = host_eng.empty_outputs(1)
    arr = ctypes.c_void_p * 1
    st = binding.load().rpiv_process_batch(host_eng.handle, 1, arr(dev[0][0].data_ptr()), arr(dev[0][1].data_ptr()),
                                           dev[0][0].stride(0) * dev[0][0].element_size(), None, None,
                                           arr(u.data_ptr()), arr(v.data_ptr()), None, None,
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 1 and b"page-locked" in binding.load().rpiv_last_error()
    dev_eng.close()
    host_eng.close()
