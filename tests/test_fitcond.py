"""The fit-conditioning rule the parity tests use (tests/fitcond.py): its fit
equals the oracle's, sharp and edge-of-search stencils are stable, a flat axis
or a value at a branch boundary is not."""
import numpy as np

import oracle
from fitcond import gauss3, well_conditioned


def _stencil(sx, sy, d=(0.2, -0.1)):
    """Sampled Gaussian peak exp(-(k - d)^2 / (2 s^2)) at the five points."""
    g = lambda k, dd, s: np.exp(-(k - dd) ** 2 / (2 * s * s))  # noqa: E731
    return np.array([g(0, d[0], sx) * g(0, d[1], sy), g(-1, d[0], sx) * g(0, d[1], sy), g(1, d[0], sx) * g(0, d[1], sy),
                     g(0, d[0], sx) * g(-1, d[1], sy), g(0, d[0], sx) * g(1, d[1], sy)])


def test_restated_fit_equals_the_oracle():
    oracle.build()
    rng = np.random.default_rng(5)
    trios = np.concatenate([rng.uniform(-0.2, 1.0, (400, 3)), rng.uniform(0.3, 1.0, (400, 3)),
                            [[0.5, 0.5, 0.5], [0.0, 1.0, 0.5], [0.6, 0.5, 0.4], [0.3, 0.5, 0.5]]])
    ref = np.array([oracle.gauss3(*t) for t in trios])
    assert np.allclose(gauss3(trios[:, 0], trios[:, 1], trios[:, 2]), ref, rtol=0, atol=1e-12)


def test_sharp_and_edge_stencils_are_stable():
    for s in (0.6, 1.0, 2.0, 5.0):
        assert well_conditioned(_stencil(s, s))
    # a monotonic stencil (peak beyond the search) clamps at 1: stable
    assert well_conditioned(np.array([0.5, 0.3, 0.7, 0.4, 0.45]))


def test_a_flat_axis_is_ill_conditioned():
    assert not well_conditioned(_stencil(60.0, 1.0))
    c = np.array([0.1282159, 0.1282118, 0.1282164, 0.1206749, 0.0832248])  # a window seen at 4096^2
    assert not well_conditioned(c)


def test_a_value_at_the_branch_boundary_is_ill_conditioned():
    # c- barely positive: the log branch, against the parabola a perturbation away
    assert not well_conditioned(np.array([0.5, 1e-300, 0.3, 0.45, 0.4]))
    c = np.array([0.5, 0.3, 0.3, 0.45, 0.4])
    assert well_conditioned(c)


def test_vectorised_over_leading_axes():
    c = np.stack([_stencil(1.0, 1.0), _stencil(60.0, 1.0)]).reshape(2, 1, 5)
    assert well_conditioned(c).tolist() == [[True], [False]]
