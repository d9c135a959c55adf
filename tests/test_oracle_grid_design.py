"""Pins of the grid re-design oracle (oracle/grid_design.py, Alg. 4)."""
import numpy as np

from oracle import grid_design as GD
from oracle import pmf


def test_design_grid_closed_form():
    """The box around corners mapped by a linear map A = F^{-1} has the closed
    form A c -+ |A| w per axis (c the predictive mean, w the half-widths):
    the grid is the union of that box and the predictive box, for several
    filters the union over filters."""
    rng = np.random.default_rng(3)
    for d in (2, 3, 4):
        F = np.eye(d) + 0.3 * rng.standard_normal((d, d))
        Q = np.diag(rng.uniform(0.05, 0.2, d))
        means = rng.standard_normal((3, d))
        covs = []
        for _ in range(3):
            A = rng.standard_normal((d, d))
            covs.append(A @ A.T / d + 0.1 * np.eye(d))
        covs = np.array(covs)
        kappa = 4.0
        lo, hi = GD.design_grid(F, Q, means, covs, kappa)
        Fi = np.linalg.inv(F)
        elo, ehi = np.full(d, np.inf), np.full(d, -np.inf)
        for m, C in zip(means, covs):
            xp = F @ m
            w = kappa * np.sqrt(np.diag(F @ C @ F.T + Q))
            c = Fi @ xp
            r = np.abs(Fi) @ w
            elo = np.minimum(elo, np.minimum(xp - w, c - r))
            ehi = np.maximum(ehi, np.maximum(xp + w, c + r))
        assert np.allclose(lo, elo, rtol=0, atol=1e-12) and np.allclose(hi, ehi, rtol=0, atol=1e-12)


def test_design_grid_diagonal_model():
    """F = diag(2, 0.5), one filter at the origin with C = I, Q = 0.25 I:
    predictive sd sqrt(4 + 0.25) and sqrt(0.25 + 0.25); kappa = 3."""
    F = np.diag([2.0, 0.5])
    lo, hi = GD.design_grid(F, 0.25 * np.eye(2), np.zeros((1, 2)), np.eye(2)[None], 3.0)
    w = 3.0 * np.sqrt(np.array([4.25, 0.5]))
    box = np.maximum(w, w / np.diag(F))
    assert np.allclose(hi, box) and np.allclose(lo, -box)


def _interp_zero_outside(x, xp, fp):
    """np.interp with the grid continued by one zero-valued point on either
    side (the density is zero at grid points beyond the grid)."""
    D = xp[1] - xp[0]
    xe = np.concatenate([[xp[0] - D], xp, [xp[-1] + D]])
    fe = np.concatenate([[0.0], fp, [0.0]])
    return np.interp(x, xe, fe, left=0.0, right=0.0)


def test_regrid_is_numpy_interp_along_every_axis():
    rng = np.random.default_rng(5)
    g_old = pmf.Grid([-3.0, -2.0], [3.0, 2.5], [17, 12])
    g_new = pmf.Grid([-2.2, -2.6], [3.4, 1.9], [17, 12])
    P = rng.uniform(0.1, 1.0, g_old.shape)
    P, _ = pmf.normalise(P, g_old)
    got = GD.regrid(P, g_old, g_new)
    ref = np.empty((g_new.shape[0], g_old.shape[1]))
    for j in range(g_old.shape[1]):
        ref[:, j] = _interp_zero_outside(g_new.axes[0], g_old.axes[0], P[:, j])
    ref2 = np.empty(g_new.shape)
    for i in range(g_new.shape[0]):
        ref2[i, :] = _interp_zero_outside(g_new.axes[1], g_old.axes[1], ref[i, :])
    ref2, _ = pmf.normalise(ref2, g_new)
    assert np.allclose(got, ref2, rtol=1e-13, atol=1e-15)


def test_regrid_onto_the_same_grid_is_identity():
    g = pmf.Grid([-1.0, 0.0, 2.0], [1.0, 3.0, 5.0], [6, 7, 5])
    P = pmf.prior(g, np.array([0.1, 1.4, 3.3]), np.diag([0.3, 0.5, 0.4]))
    assert np.allclose(GD.regrid(P, g, g), P, rtol=1e-14, atol=0)


def test_regrid_keeps_gaussian_moments():
    """A Gaussian well inside both grids keeps its mean and covariance up to
    the interpolation's O(D^2) error."""
    g_old = pmf.Grid([-6.0, -6.0], [6.0, 6.0], [96, 96])
    g_new = pmf.Grid([-4.3, -5.1], [5.2, 4.4], [96, 96])
    m = np.array([0.4, -0.3])
    C = np.array([[1.0, 0.3], [0.3, 0.6]])
    P = pmf.prior(g_old, m, C)
    mo, co = pmf.moments(GD.regrid(P, g_old, g_new), g_new)
    D = g_old.delta_axis[0]
    assert np.abs(mo - m).max() < 0.2 * D ** 2
    assert np.abs(co - C).max() < 0.5 * D ** 2
