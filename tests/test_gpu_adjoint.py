"""The adjoint of the zero-shift correlation score (differentiation pattern).

GPU score and gradient (rpiv_backward, FP32) against the FP64 oracle's
analytic values, against central finite differences of the exact (FP64)
score, through torch.autograd, and the gradient-ascent refinement rule run
on both sides."""
import numpy as np
import pytest
import torch

import oracle
import paper_2504_17987_gb300 as rp
import synth
from synth import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2504_17987_gb300 import build
    build.build()
    oracle.build()


def _case(W, H, seed):
    w = wl.diff_1mp(seed=seed)
    w.spec.W, w.spec.H = W, H
    w.flow.vortices = [(0.5 * W, 0.5 * H, 200.0, 20.0)]
    A, B = w.render()
    win, s = 32, 8
    nx, ny = oracle.grid_n(W, win, s), oracle.grid_n(H, win, s)
    X, Y = np.meshgrid(np.arange(nx) * s + 15.5, np.arange(ny) * s + 15.5)
    tu, tv = w.flow.eval(X, Y)
    r = synth.uniform(seed, 2 * nx * ny).reshape(2, ny, nx)
    gu = (tu + 0.3 * (r[0] - 0.5)).astype(np.float32)
    gv = (tv + 0.3 * (r[1] - 0.5)).astype(np.float32)
    cfg = rp.Config(W, H, windows=(win,), overlaps=(0.75,), radii=(8,), bit_depth=8)
    return A, B, gu, gv, cfg, win, s


def test_score_and_gradient_match_fp64_oracle_at_full_size():
    # 1024 x 1024 u8, 32 px windows at 75 % overlap: 125 x 125 vectors
    A, B, gu, gv, cfg, w, s = _case(1024, 1024, 3003)
    eng = rp.Engine(cfg)
    S, Gu, Gv = eng.score_and_grad(rp.to_device(A), rp.to_device(B), torch.from_numpy(gu).cuda(),
                                   torch.from_numpy(gv).cuda())
    torch.cuda.synchronize()
    So, Ou, Ov = oracle.score_grad(A, B, w, s, gu.astype(np.float64), gv.astype(np.float64))
    assert Gu.shape == (125, 125)
    assert abs(float(S) - So) <= 1e-5 * abs(So)
    g = np.stack([Gu.cpu().numpy(), Gv.cpu().numpy()])
    o = np.stack([Ou, Ov])
    rel = np.linalg.norm(g - o) / np.linalg.norm(o)
    assert rel <= 2e-4, f"relative gradient error {rel:.2e}"
    assert np.max(np.abs(g - o)) <= 1e-3 * np.max(np.abs(o))
    eng.close()


def test_gradient_matches_central_differences_of_the_exact_score():
    # 64 seeded vectors, step 1e-3 px, differences of the FP64 score
    A, B, gu, gv, cfg, w, s = _case(256, 224, 3004)
    eng = rp.Engine(cfg)
    _, Gu, Gv = eng.score_and_grad(rp.to_device(A), rp.to_device(B), torch.from_numpy(gu).cuda(),
                                   torch.from_numpy(gv).cuda())
    Gu, Gv = Gu.cpu().numpy(), Gv.cpu().numpy()
    ny, nx = gu.shape
    h = 1e-3
    picks = synth.uniform(7001, 64)
    base = (gu.astype(np.float64), gv.astype(np.float64))
    errs = []
    for p in picks:
        k = int(p * nx * ny)
        j, i = divmod(k, nx)
        for comp, G in ((0, Gu), (1, Gv)):
            up = [base[0].copy(), base[1].copy()]
            dn = [base[0].copy(), base[1].copy()]
            up[comp][j, i] += h
            dn[comp][j, i] -= h
            fd = (oracle.score_grad(A, B, w, s, *up, grad=False) - oracle.score_grad(A, B, w, s, *dn, grad=False)) / (2 * h)
            errs.append(abs(G[j, i] - fd) / max(1.0, abs(fd)))
    errs = np.array(errs)
    # a step of 1e-3 px crosses a pixel edge (a kink of the bilinear warp) for a
    # few samples; all but those agree tightly
    assert np.percentile(errs, 90) <= 2e-3, f"90th percentile relative error {np.percentile(errs, 90):.2e}"
    assert np.median(errs) <= 5e-4
    eng.close()


def test_autograd_function_routes_through_the_adjoint():
    A, B, gu, gv, cfg, w, s = _case(256, 224, 3005)
    eng = rp.Engine(cfg)
    a, b = rp.to_device(A), rp.to_device(B)
    u = torch.from_numpy(gu).cuda().requires_grad_(True)
    v = torch.from_numpy(gv).cuda().requires_grad_(True)
    S = rp.CorrelationScore.apply(u, v, eng, a, b)
    (2.5 * S).backward()
    _, Gu, Gv = eng.score_and_grad(a, b, u.detach(), v.detach(), grad_score=2.5)
    torch.cuda.synchronize()
    assert torch.equal(u.grad, Gu) and torch.equal(v.grad, Gv)
    eng.close()


def test_refinement_rule_on_gpu_follows_the_oracle():
    A, B, gu, gv, cfg, w, s = _case(256, 224, 3006)
    eng = rp.Engine(cfg)
    u, v, hist = rp.refine(eng, rp.to_device(A), rp.to_device(B), torch.from_numpy(gu).cuda(),
                           torch.from_numpy(gv).cuda(), steps=5)
    ou, ov, ohist = oracle.refine(A, B, w, s, gu.astype(np.float64), gv.astype(np.float64), steps=5)
    assert len(hist) == len(ohist) == 6
    assert all(b >= a - 1e-3 for a, b in zip(hist, hist[1:]))
    assert hist[-1] > hist[0]
    assert np.allclose(hist, ohist, rtol=1e-4)
    assert np.max(np.abs(u.cpu().numpy() - ou)) <= 1e-3 and np.max(np.abs(v.cpu().numpy() - ov)) <= 1e-3
    eng.close()
