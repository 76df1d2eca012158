"""Host logic of bench.py that needs no device: the source hash that ties the
stored DRAM counters to the pass kernels' code."""
import os
import shutil

import bench

FILES = ("pass_impl.cuh", "k_pass_fp32.cu", "k_pass_bf16.cu", "k_pass_fp16.cu", "pass_plan.cpp")


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
