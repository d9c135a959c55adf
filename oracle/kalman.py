"""Kalman filter (test infrastructure only).

For a linear-Gaussian model x_{k+1} = F x_k + w_k, z_k = H x_k + v_k (the
linear special case of Eqs. asx/asz) the Bayesian recursion of Sec. 1 has the
closed-form Kalman solution.  The point-mass filter must converge to it as the
grid is refined; the tests use that to pin the dense oracle.  Step order
matches the filter: predict, update with z_k, estimate; no z_0.
"""
from __future__ import annotations

import math

import numpy as np


def kalman(m0, P0, F, Q, H, R, zs):
    """Returns dict(means, covs, log_lik, log_c) where log_c[k] is the log of
    N(z_k; H m_k^-, H P_k^- H^T + R), the exact analogue of log c_k of Eq.
    pmf_filtrace_b."""
    m = np.asarray(m0, dtype=np.float64).copy()
    P = np.asarray(P0, dtype=np.float64).copy()
    F = np.asarray(F, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    H = np.atleast_2d(np.asarray(H, dtype=np.float64))
    R = np.atleast_2d(np.asarray(R, dtype=np.float64))
    means, covs, logc = [], [], []
    for z in zs:
        z = np.atleast_1d(np.asarray(z, dtype=np.float64))
        m = F @ m
        P = F @ P @ F.T + Q
        S = H @ P @ H.T + R
        innov = z - H @ m
        sol = np.linalg.solve(S, innov)
        b = len(z)
        logc.append(-0.5 * (innov @ sol) - 0.5 * np.linalg.slogdet(S)[1] - 0.5 * b * math.log(2 * math.pi))
        K = np.linalg.solve(S, H @ P).T
        m = m + K @ innov
        P = P - K @ S @ K.T
        P = 0.5 * (P + P.T)
        means.append(m.copy())
        covs.append(P.copy())
    return {"means": np.array(means), "covs": np.array(covs),
            "log_c": np.array(logc), "log_lik": float(np.sum(logc))}
