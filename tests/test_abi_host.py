"""The C ABI on the host: the library loads, exports every declared entry
point, and validates configurations (no device needed)."""
import ctypes
import os
import re

import pytest

import paper_2504_17987_gb300 as rp
from paper_2504_17987_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2504_17987_gb300 import build
    build.build()
    return rp.load()


def test_every_declared_symbol_is_exported(lib):
    hdr = open(os.path.join(ROOT, "include", "rpiv.h")).read()
    declared = sorted(set(re.findall(r"\b(rpiv_[a-z_]+)\s*\(", hdr)))
    assert len(declared) >= 16
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(binding.EXPORTED) == declared


def test_config_default_matches_paper_settings(lib):
    c = binding._Config()
    assert lib.rpiv_config_default(ctypes.byref(c)) == 0
    assert c.window[0] == 16 and abs(c.overlap[0] - 0.5) < 1e-7
    assert abs(c.uod_threshold - 2.0) < 1e-7 and abs(c.uod_eps - 0.1) < 1e-7


@pytest.mark.parametrize("cfg,grid", [
    (dict(width=256, height=256, windows=(32,), overlaps=(0.5,), radii=(8,)), (15, 15)),
    (dict(width=1024, height=1024, windows=(64, 32, 16), overlaps=(0.5,) * 3, radii=(4,) * 3, levels=2,
          bit_depth=12), (127, 127)),
    (dict(width=1024, height=1024, windows=(32,), overlaps=(0.75,), radii=(8,)), (125, 125)),
    (dict(width=3840, height=2160, windows=(48, 24), overlaps=(0.5, 0.5), radii=(6, 6), levels=2), (319, 179)),
    (dict(width=1024, height=1024, windows=(16,), overlaps=(0.5,), radii=(1,)), (127, 127)),
])
def test_grid_shapes(lib, cfg, grid):
    assert rp.validate_config(rp.Config(**cfg)) == grid


@pytest.mark.parametrize("bad,msg", [
    (dict(windows=(15,)), "even"),
    (dict(windows=(6,)), "even"),
    (dict(overlaps=(1.0,)), "overlap"),
    (dict(overlaps=(0.3,)), "integer"),
    (dict(radii=(17,)), "search_radius"),
    (dict(radii=(-1,)), "search_radius"),
    (dict(width=30, height=30, windows=(16,), radii=(8,)), "smaller"),
    (dict(levels=5), "predictor_levels"),
    (dict(levels=4, width=128, height=128), "smaller"),
    (dict(max_batch=65), "max_batch"),
    (dict(max_batch=0), "max_batch"),
    (dict(bit_depth=10), "bit_depth"),
    (dict(uod_threshold=0.0), "uod"),
    (dict(precision="bf16", radii=(5,)), "not built"),
])
def test_invalid_configs_are_rejected(lib, bad, msg):
    base = dict(width=256, height=256, windows=(32,), overlaps=(0.5,), radii=(4,))
    base.update(bad)
    with pytest.raises(rp.RpivError) as ei:
        rp.validate_config(rp.Config(**base))
    assert ei.value.status == 1
    assert msg in str(ei.value)


def test_unknown_enum_and_null_rejected(lib):
    c = rp.Config(256, 256, (32,), (0.5,), (4,)).to_c()
    c.precision = 7
    assert lib.rpiv_validate_config(ctypes.byref(c), None, None) == 1
    assert b"precision" in lib.rpiv_last_error()
    assert lib.rpiv_validate_config(None, None, None) == 1
    assert lib.rpiv_create(None, 0, None) == 1


def test_binding_config_mirrors_the_header_struct(lib, tmp_path):
    # the ctypes mirror must have the C struct's size and field offsets
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no host C compiler")
    inc = os.path.join(ROOT, "include")
    cuda_inc = next((d for d in ("/usr/local/cuda/include",) if os.path.isdir(d)), None)
    if cuda_inc is None:
        pytest.skip("CUDA headers not found")
    src = tmp_path / "sz.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "rpiv.h"\n'
                   'int main(void) { printf("%zu %zu %zu\\n", sizeof(rpiv_config), '
                   'offsetof(rpiv_config, max_batch), offsetof(rpiv_config, host_frames)); return 0; }\n')
    exe = tmp_path / "sz"
    subprocess.run([cc, "-I", inc, "-I", cuda_inc, str(src), "-o", str(exe)], check=True)
    size, off_mb, off_hf = (int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                                            check=True).stdout.split())
    assert ctypes.sizeof(binding._Config) == size
    assert binding._Config.max_batch.offset == off_mb and binding._Config.host_frames.offset == off_hf


def test_host_frames_flag_default_and_range(lib):
    c = binding._Config()
    assert lib.rpiv_config_default(ctypes.byref(c)) == 0
    assert c.host_frames == 0
    c = rp.Config(256, 256, (32,), (0.5,), (4,), host_frames=True).to_c()
    assert c.host_frames == 1 and lib.rpiv_validate_config(ctypes.byref(c), None, None) == 0
    c.host_frames = 2
    assert lib.rpiv_validate_config(ctypes.byref(c), None, None) == 1
    assert b"host_frames" in lib.rpiv_last_error()


def test_create_without_device_reports_no_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    c = rp.Config(256, 256, (32,), (0.5,), (4,)).to_c()
    h = ctypes.c_void_p()
    st = lib.rpiv_create(ctypes.byref(c), 0, ctypes.byref(h))
    assert st == 7 and not h.value


def test_product_path_does_not_touch_the_oracle():
    # the package and the CUDA sources never import, link or name the oracle
    pkg = os.path.join(ROOT, "paper_2504_17987_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "liboracle" not in txt and "rpiv_oracle" not in txt, f
