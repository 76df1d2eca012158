"""Conditioning of the three-point Gaussian fit (paper Sec. 2), shared by the
parity tests.

The fit is delta = (ln c- - ln c+) / (2 ln c- - 4 ln c0 + 2 ln c+), with the
parabola (c- - c+) / (2 c- - 4 c0 + 2 c+) when a value is not positive or the
log-curvature is not negative, 0 when neither curvature is negative, clamped
to [-1, 1].  Where the correlation peak is flat along an axis (a tiny
curvature) or a value sits at a branch boundary, an error of the size that
any 32-bit evaluation of the coefficients makes (taken here as a relative
1e-5 plus an absolute 1e-6) moves delta by more than the 1e-3 px tolerance.  The tests assert the
1e-3 px bound on the windows whose fit is stable against that perturbation,
and only validity (finite, rare) on the others."""
import numpy as np

REL = 1e-5    # relative perturbation of a stencil value
ABS = 1e-6    # and absolute (a coefficient near zero carries an absolute error)
TOL = 1e-3    # px the fit may move under it


def gauss3(cm, c0, cp):
    """The fit, vectorised (test restatement of the rule above)."""
    cm, c0, cp = (np.asarray(x, np.float64) for x in (cm, c0, cp))
    pos = (cm > 0) & (c0 > 0) & (cp > 0)
    with np.errstate(divide="ignore", invalid="ignore"):
        lm, l0, lp = (np.log(np.where(pos, x, 1.0)) for x in (cm, c0, cp))
        dl = 2 * lm - 4 * l0 + 2 * lp
        dp = 2 * cm - 4 * c0 + 2 * cp
        use_log = pos & (dl < 0)
        use_par = ~use_log & (dp < 0)
        d = np.where(use_log, (lm - lp) / np.where(use_log, dl, -1.0),
                     np.where(use_par, (cm - cp) / np.where(use_par, dp, -1.0), 0.0))
    return np.clip(d, -1.0, 1.0)


def well_conditioned(c5):
    """c5: (..., 5) stencil values (centre, -x, +x, -y, +y) of the FP64
    oracle; True where no single value perturbed by a relative REL plus an
    absolute ABS (either sign) moves either axis' fit by more than TOL."""
    c5 = np.asarray(c5, np.float64)
    ok = np.ones(c5.shape[:-1], bool)
    for m, p in ((1, 2), (3, 4)):
        trio = [c5[..., m], c5[..., 0], c5[..., p]]
        d0 = gauss3(*trio)
        for k in range(3):
            for sgn in (1.0, -1.0):
                t = list(trio)
                t[k] = t[k] * (1.0 + sgn * REL) + sgn * ABS
                ok &= np.abs(gauss3(*t) - d0) <= TOL
    return ok
