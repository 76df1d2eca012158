"""Host logic of bench.py that needs no device: the source hash that ties the
stored DRAM counters to the pass kernels' code, and the summary of the clock
samples taken around the timed region."""
import os
import shutil

import bench

FILES = ("pass_impl.cuh", "tc_pass.cuh", "k_pass_fp32.cu", "k_pass_tc.cu", "pass_plan.cpp")


def _copy_sources(tmp_path):
    src = os.path.join(bench.ROOT, "paper_2504_17987_gb300", "csrc")
    dst = tmp_path / "paper_2504_17987_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in FILES:
        shutil.copy(os.path.join(src, f), dst / f)
    return dst


def test_source_hash_ignores_comments_and_whitespace_but_not_code(tmp_path, monkeypatch):
    dst = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench._kernel_source_hash()

    plan = dst / "pass_plan.cpp"
    text = plan.read_text()
    plan.write_text("// a new line comment\n/* and a\n   block comment */\n" + text.replace("\n", "\n\n", 3) + "  \n")
    assert bench._kernel_source_hash() == h0

    # a changed constant is a changed kernel
    assert "kThreads = 256" in text
    plan.write_text(text.replace("kThreads = 256", "kThreads = 128"))
    assert bench._kernel_source_hash() != h0

    # so is a change to any of the other files
    plan.write_text(text)
    assert bench._kernel_source_hash() == h0
    impl = dst / "pass_impl.cuh"
    impl.write_text(impl.read_text() + "\nstatic int added_code = 1;\n")
    assert bench._kernel_source_hash() != h0


def _smi_line(t, sm, reason="Not Active"):
    import datetime
    stamp = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return f"{stamp}, {sm}, 2070, 900.00, 0x0000000000000000, {reason}, Not Active, Not Active, Not Active"


def test_clock_summary_keeps_the_samples_inside_the_timed_region():
    cs = bench.ClockSampler(0)
    base = 1_700_000_000.0
    cs.lines = [(base + 0.02 * k, _smi_line(base + 0.02 * k, 1200 if k < 5 or k > 12 else 2070,
                                            "Active" if k == 2 else "Not Active")) for k in range(16)]
    cs.t0, cs.t1 = base + 0.095, base + 0.245
    out = cs.summary()
    assert out["samples"] == 8 and out["sm_mhz"] == 2070 and out["reasons"] == []
    assert "nearest_outside_region" not in out and out["window_ms"] == 150.0
    # a slowdown inside the region is reported
    cs.t0 = base + 0.035
    assert cs.summary()["reasons"] == ["hw_slowdown"]


def test_clock_summary_of_a_region_shorter_than_the_interval_uses_the_nearest_samples():
    cs = bench.ClockSampler(0)
    base = 1_700_000_000.0
    cs.lines = [(base, _smi_line(base, 2070)), (base + 0.5, _smi_line(base + 0.5, 2050)),
                (base + 1.0, _smi_line(base + 1.0, 1000))]
    cs.t0, cs.t1 = base + 0.6, base + 0.7
    out = cs.summary()
    assert out["nearest_outside_region"] and out["samples"] == 2 and out["sm_mhz"] == 1525.0
    # no region marked: every sample counts
    cs.t0 = cs.t1 = None
    assert cs.summary()["samples"] == 3
    # unparseable output gives no clock rather than a wrong one
    cs.lines = [(base, "[N/A], [N/A]")]
    assert cs.summary()["sm_mhz"] is None


def test_stored_traffic_applies_only_to_the_pass_it_was_taken_on(tmp_path):
    import json
    h = bench._kernel_source_hash()
    entry = {"bytes_per_pair": 1000.0, "source_hash": h, "window": 64, "step": 32, "radius": 4}
    path = tmp_path / "traffic.json"
    path.write_text(json.dumps({"paper_1mp/fp32/pass/p0": entry}))
    dom = {"name": "pass/p0", "window": 64, "step": 32, "radius": 4, "pairs": 64}
    assert bench.stored_traffic("paper_1mp", "fp32", dom, str(path)) == 64000.0
    # another workload's pass of the same name (a 32 px pass there) gets nothing
    assert bench.stored_traffic("paper_1mp_r1", "fp32", dict(dom, window=32, step=16), str(path)) is None
    assert bench.stored_traffic("paper_1mp_r1", "fp32", dom, str(path)) is None
    # nor another precision, another geometry, or changed kernels
    assert bench.stored_traffic("paper_1mp", "bf16", dom, str(path)) is None
    assert bench.stored_traffic("paper_1mp", "fp32", dict(dom, radius=1), str(path)) is None
    path.write_text(json.dumps({"paper_1mp/fp32/pass/p0": dict(entry, source_hash="0" * 16)}))
    assert bench.stored_traffic("paper_1mp", "fp32", dom, str(path)) is None
    assert bench.stored_traffic("paper_1mp", "fp32", dom, str(tmp_path / "missing.json")) is None


def test_committed_traffic_entries_name_their_geometry():
    import json
    tr = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for key, ent in tr.items():
        workload, head, _, name = key.split("/")
        assert workload in ("paper_1mp", "paper_1mp_r1") and head in ("fp32", "bf16", "fp16")
        assert {"window", "step", "radius", "bytes_per_pair", "source_hash"} <= set(ent)


def test_kernel_bytes_count_each_frame_and_field_once():
    import bench
    rec = dict(pairs=64, width=1024, height=1024, nx=127, ny=127, launches=3, total_ms=3.0)
    b = lambda name, **k: bench.kernel_bytes({**rec, "name": name, **k}, 2, 8)  # noqa: E731
    assert b("ingest") == 64 * 1024 * 1024 * 6
    assert b("down/L1") == 64 * (1024 * 1024 * 2 + 512 * 512 * 4)
    assert b("down/L2", width=512, height=512) == 64 * (512 * 512 * 4 + 256 * 256 * 4)
    assert b("deform/p2") == 64 * (1024 * 1024 * 2 + 1040 * 1040 * 4)
    assert b("deform/L1", width=512, height=512) == 64 * (512 * 512 * 4 + 528 * 528 * 4)
    assert b("uod/p2") == 64 * 127 * 127 * 21 and b("vort") == 64 * 127 * 127 * 12
    assert b("interp/p1") == 64 * 127 * 127 * 16
    assert b("pass/p2") == 64 * 1024 * 1024 * 8
    rows = bench.kernel_roofline([{**rec, "name": "vort"}], 2, 8, 6789.0)
    assert rows[0]["ms_per_launch"] == 1.0 and abs(rows[0]["gbs"] - 64 * 127 * 127 * 12 / 1e-3 / 1e9) < 0.1
