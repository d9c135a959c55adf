"""Grid re-design (Alg. 4) for the point-mass filter, in float64 (test
infrastructure only).

Alg. 4 with linear dynamics x' = F x + w keeps the grid axis-aligned and sized
to the density.
* Step 1: from the filtering moments it forms the predictive moments. For
  linear F they are exact: F m and F C F^T + Q.
* Step 2: it takes the corners of the box around the predictive mean that is
  kappa predictive standard deviations wide on every axis (the sigma-box
  reading of its "Chebyshev inequality / sigma ellipse").
* Step 3: it maps those corners back to the filtering space by F^{-1}.
* Step 4: it designs the smallest axis-aligned grid around the mapped corners.
The re-gridded transition of this repository maps the grid onto itself, so
the grid designed here is the box around both corner sets: the filtering
density lives on it before the step and the predictive density after it. For
a batch that shares one grid, it is the box around every filter's corners.
* Step 5 interpolates the filtering density onto the new grid. The paper does
  it by TT cross of the interpolant. Here it is the separable piecewise-linear
  interpolation of the density values: the value at a new cell centre comes
  from the two old centres around it along each axis, and the density is zero
  at the grid points beyond the old grid, as in the filter's boundary reading.
  The result is then renormalised.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import pmf


def design_grid(F, Q, means, covs, kappa):
    """(lo, hi) of the grid of Alg. 4 steps 1-4 for filtering means
    (batch, d) and covariances (batch, d, d)."""
    F = np.asarray(F, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    means = np.atleast_2d(np.asarray(means, dtype=np.float64))
    d = F.shape[0]
    covs = np.asarray(covs, dtype=np.float64).reshape(means.shape[0], d, d)
    lo = np.full(d, np.inf)
    hi = np.full(d, -np.inf)
    for m, C in zip(means, covs):
        xp = F @ m                      # step 1: predictive mean
        Pp = F @ C @ F.T + Q            # and covariance
        w = kappa * np.sqrt(np.diag(Pp))
        for signs in itertools.product((-1.0, 1.0), repeat=d):
            cpred = xp + np.array(signs) * w          # step 2: corners
            cmeas = np.linalg.solve(F, cpred)         # step 3: F^{-1} corners
            lo = np.minimum(lo, np.minimum(cpred, cmeas))
            hi = np.maximum(hi, np.maximum(cpred, cmeas))
    return lo, hi                                     # step 4: circumscribing box


def interpolation_matrix(old_axis, new_axis) -> np.ndarray:
    """W[j, i]: weight of old point i in the linear interpolant at new point j
    (equidistant old points, zero-valued points beyond them)."""
    old_axis = np.asarray(old_axis, dtype=np.float64)
    D = old_axis[1] - old_axis[0] if old_axis.size > 1 else 1.0
    u = (np.asarray(new_axis, dtype=np.float64)[:, None] - old_axis[None, :]) / D
    return np.maximum(0.0, 1.0 - np.abs(u))


def regrid(P, grid_old: pmf.Grid, grid_new: pmf.Grid) -> np.ndarray:
    """Step 5: the density values onto the new grid's points, renormalised."""
    out = np.asarray(P, dtype=np.float64)
    for m in range(grid_old.d):
        out = pmf.apply_along(out, interpolation_matrix(grid_old.axes[m], grid_new.axes[m]), m)
    return pmf.normalise(out, grid_new)[0]
