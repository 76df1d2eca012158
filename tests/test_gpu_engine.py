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
