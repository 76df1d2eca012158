"""The correlation-pass planner on the host: pass_plan.cpp built with the host
compiler against stub launchers (tests/plan_probe.cpp), run over many window
sizes, steps, radii, grid sizes and precisions.  The checks are the plan's
invariants, not particular tile shapes: tiles cover the grid, the layout fits
shared memory, strips are planned only for the kernels specialised to them,
and the box-sum runs cover every output once within the one-round rule."""
import math
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2504_17987_gb300", "csrc")
THREADS = 256
SMEM_MAX = 227 * 1024


def _cuda_include():
    for base in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if base and os.path.exists(os.path.join(base, "include", "cuda_runtime.h")):
            return os.path.join(base, "include")
    nvcc = shutil.which("nvcc")
    if nvcc:
        inc = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")
        if os.path.exists(os.path.join(inc, "cuda_runtime.h")):
            return inc
    return None


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("host C++ compiler or CUDA headers not found")
    exe = str(tmp_path_factory.mktemp("plan") / "plan_probe")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", inc, "-I", CSRC, os.path.join(ROOT, "tests", "plan_probe.cpp"),
                    os.path.join(CSRC, "pass_plan.cpp"), "-o", exe], check=True, capture_output=True, text=True)
    env = {k: v for k, v in os.environ.items()
           if k not in ("RPIV_MIN_CTAS", "RPIV_TILE_SMEM_KB", "RPIV_PLANE_ITEMS", "RPIV_STRIP_ROWS", "RPIV_TC_PLANES")}

    def run(cases, extra_env=None):
        text = "".join(f"{w} {s} {R} {nx} {ny} {p}\n" for (w, s, R, nx, ny, p) in cases)
        out = subprocess.run([exe], input=text, check=True, capture_output=True, text=True,
                             env={**env, **(extra_env or {})}).stdout
        res = []
        for line in out.strip().splitlines():
            a, b, c = line.split("|")
            t, st, tc = [int(x) for x in a.split()], [int(x) for x in b.split()], [int(x) for x in c.split()]
            res.append(dict(ok=t[0], TX=t[1], TY=t[2], tiles_x=t[3], tiles_y=t[4], smem=t[5], RG=t[6], lv=t[7],
                            lh=t[8], nv=t[9], nh=t[10],
                            strip=dict(TX=st[0], rows=st[1], tiles_x=st[2], tiles_y=st[3], smem=st[4], lv=st[5],
                                       lh=st[6], nv=st[7], nh=st[8]),
                            tc=dict(zip(("tc off_p off_red off_gst off_h off_slab slab_rows slab_lbo off_cp cp_bytes "
                                         "cp_lbo nbuf off_ebuf tmem_cols off_c5 off_dpart cp_group off_refit").split(),
                                        tc))))
        assert len(res) == len(cases)
        return res
    return run


def _cases():
    out = []
    for w in (8, 12, 16, 20, 24, 32, 48, 64):
        for s in sorted({w, w // 2, w // 4} - {0}):
            for R in (0, 1, 2, 4, 6, 8):
                for nx, ny in ((1, 1), (3, 2), (7, 9), (63, 63), (127, 127), (319, 179)):
                    for prec in (0, 1, 2):
                        out.append((w, s, R, nx, ny, prec))
    # the benchmark workloads' passes
    out += [(64, 32, 4, 31, 31, 0), (32, 16, 4, 63, 63, 0), (16, 8, 4, 127, 127, 0), (16, 8, 1, 127, 127, 0),
            (64, 32, 4, 15, 15, 0), (64, 32, 4, 7, 7, 0), (48, 24, 6, 159, 89, 0), (24, 12, 6, 319, 179, 0)]
    return out


def _check_runs(L, n_runs, n, across):
    # runs of L outputs, n_runs of them per line, cover the n outputs of a
    # full tile's line; a run longer than 8 is taken only when all runs of
    # the pass fit one round of the CTA's threads with 7/8 of them busy
    assert 8 <= L <= 16
    assert n_runs == math.ceil(n / L)
    if L > 8:
        assert across * n_runs <= THREADS and 8 * across * n_runs >= 7 * THREADS


def _box(TX, TY, w, s, R):
    aw, ah = (TX - 1) * s + w, (TY - 1) * s + w
    BC, BR = aw + 2 * (R + 1), ah + 2 * (R + 1)
    return BC, BR - w + 1, BC - w + 1  # columns, column-run outputs, row-run outputs


def test_plans_cover_the_grid_fit_shared_memory_and_size_box_runs(probe):
    cases = _cases()
    longer = 0
    for (w, s, R, nx, ny, prec), p in zip(cases, probe(cases)):
        G = math.gcd(w, s)
        if prec != 0 and G % 2:
            assert not p["ok"], (w, s, R, prec)  # paired 16-bit loads need even blocks
            continue
        assert p["ok"], (w, s, R, nx, ny, prec)
        assert 1 <= p["TX"] <= min(8, nx) and 1 <= p["TY"] <= min(8, ny)
        assert p["tiles_x"] == math.ceil(nx / p["TX"]) and p["tiles_y"] == math.ceil(ny / p["TY"])
        assert 0 < p["smem"] <= SMEM_MAX
        RG = p["RG"]
        assert RG >= 1 and RG & (RG - 1) == 0 and G % RG == 0
        BC, vh, hw = _box(p["TX"], p["TY"], w, s, R)
        _check_runs(p["lv"], p["nv"], vh, BC)
        _check_runs(p["lh"], p["nh"], hw, vh)
        longer += p["lv"] > 8 or p["lh"] > 8

        st = p["strip"]
        if st["TX"]:
            assert prec == 0 and w == 2 * s and s in (16, 32) and R in (1, 4) and ny >= 2
            assert st["rows"] == min(8, ny) and st["tiles_y"] == math.ceil(ny / st["rows"])
            assert 1 <= st["TX"] <= min(8, nx) and st["tiles_x"] == math.ceil(nx / st["TX"])
            assert 0 < st["smem"] <= SMEM_MAX
            BC, vh, hw = _box(st["TX"], 1, w, s, R)
            _check_runs(st["lv"], st["nv"], vh, BC)
            _check_runs(st["lh"], st["nh"], hw, vh)
        else:
            assert not (prec == 0 and w == 2 * s and s in (16, 32) and R in (1, 4) and ny >= 2 and nx >= 2), \
                (w, s, R, nx, ny)
    assert longer > 0


def test_the_16px_pass_of_the_1mp_workload_takes_longer_box_runs(probe):
    # measured on GB300: 12- and 10-output runs took this pass from 1.200 to
    # 1.130 ms per 64-pair launch; the strips keep runs of 8
    p16, p64, p32 = probe([(16, 8, 4, 127, 127, 0), (64, 32, 4, 31, 31, 0), (32, 16, 4, 63, 63, 0)])
    assert p16["lv"] > 8 and p16["lh"] > 8
    for p in (p64, p32):
        assert p["strip"]["TX"] and p["strip"]["lv"] == 8 and p["strip"]["lh"] == 8


def test_tensor_core_tiles_keep_every_operand_read_inside_shared_memory(probe):
    """tcgen05 tiles (16-bit, 50 % overlap with 8/16/32 px steps, r = 4): the
    MMA operands are read through descriptors, so every address an MMA can form
    must lie in the tile's shared memory.  A copy buffer's MMAs reach past the
    last group's chunks (the unused shift slots) and must stay in the buffer,
    the slab's reach (2R above to 16 - 4 below the window) must stay in the
    slab, and the TMEM columns must cover 16 per window with at most 512 per SM
    at the occupancy the shared memory allows."""
    cases = []
    for s in (8, 16, 32):
        for prec in (1, 2):
            for nx, ny in [(1, 1), (2, 3), (7, 5), (31, 31), (127, 127), (63, 9), (159, 89), (11, 255)]:
                cases.append((2 * s, s, 4, nx, ny, prec))
    res = probe(cases, {"RPIV_TC_PLANES": "1"})
    R, rows = 4, 4
    for (w, s, _, nx, ny, prec), r in zip(cases, res):
        t = r["tc"]
        assert r["ok"] == 1 and t["tc"] == 1, (w, nx, ny, prec)
        TX, TY, smem = r["TX"], r["TY"], r["smem"]
        assert smem <= SMEM_MAX
        aw, ah = (TX - 1) * s + w, (TY - 1) * s + w
        nch, ng = aw // 8, (w + 2 * R) // rows
        assert t["cp_lbo"] == 8 * rows * 16 and t["cp_group"] == (nch + 1) * t["cp_lbo"]
        assert t["nbuf"] in (4, 6) and t["cp_bytes"] >= t["nbuf"] * t["cp_group"]
        # every address the copies' MMAs can form: the last slot of the ring, the
        # last window's last K step (chunk nch - 2), every M row (16 slots of 4 rows
        # past it) and both K chunks; it must stay in the ring
        start = t["off_cp"] + (t["nbuf"] - 1) * t["cp_group"] + (nch - 2) * t["cp_lbo"]
        reach = start + 7 * 16 + 15 * 128 + 7 * 2 + t["cp_lbo"] + 2
        assert reach <= t["off_cp"] + t["cp_bytes"], (w, TX, TY)
        # the slabs (two rows): rows 4 g + n of every group, both K chunks of the last window
        assert rows * (ng - 1) + 16 <= t["slab_rows"]
        assert t["off_slab"] + 2 * nch * t["slab_lbo"] <= t["off_cp"]
        assert t["off_cp"] + t["cp_bytes"] <= t["off_ebuf"]
        assert t["off_ebuf"] + 3 * 32 * 20 * 4 <= smem
        # persistent buffers (planes, refit planes) precede the reused region
        nb = (aw // s) * (ah // s)
        assert t["off_p"] + TX * TY * (2 * R + 1) ** 2 * 4 <= t["off_refit"]
        assert t["off_refit"] + nb * 25 * 4 <= t["off_h"] == t["off_slab"] == t["off_c5"]
        assert t["off_red"] + 8 * (1 + 2 * t["nbuf"] + 6) + 16 <= t["off_gst"]
        for k in ("off_p", "off_red", "off_slab", "off_cp", "off_ebuf", "cp_bytes", "slab_lbo", "off_refit"):
            assert t[k] % 16 == 0, k
        cols = t["tmem_cols"]
        assert cols >= max(32, 32 * TX) and cols & (cols - 1) == 0 and cols <= 512
        ctas = min(228 * 1024 // (smem + 1024), 2048 // THREADS)
        assert min(ctas, 512 // cols) >= 1
