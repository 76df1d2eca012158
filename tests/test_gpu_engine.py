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
