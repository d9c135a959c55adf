"""Pins of the differentiable log-likelihood (oracle/grad.py): its value is the
dense oracle's log-likelihood, and its reverse-mode gradient agrees with
central finite differences of the dense oracle (structurally non-zero
entries of F, the diagonals of Q and R)."""
import numpy as np
import pytest

from oracle import grad, pmf


def _model(d):
    if d == 2:
        g = pmf.Grid([-6.0, -5.0], [6.0, 5.0], [20, 18])
        F = np.array([[0.93, 0.12], [-0.07, 0.88]])
        Q = np.diag([0.09, 0.12])
        comps = [((0,), g.axes[0]), ((1,), np.sin(g.axes[1]))]
        R = np.diag([0.2, 0.1])
        z = [np.array([0.4, 0.2]), np.array([0.1, -0.3]), np.array([-0.2, 0.1])]
    elif d == "bearing":
        # range and bearing (an angle of period 360) on a grid across the
        # negative x axis: the bearing's residual switches branch inside it
        g = pmf.Grid([-15.0, -5.0], [-5.0, 5.0], [20, 18])
        F = np.array([[0.96, 0.05], [-0.04, 0.97]])
        Q = np.diag([0.3, 0.25])
        X, Y = g.axes[0][:, None], g.axes[1][None, :]
        comps = [((0, 1), np.hypot(X, Y)), ((0, 1), np.degrees(np.arctan2(Y, X)), 360.0)]
        R = np.diag([0.5, 9.0])
        z = [np.array([9.6, 178.0]), np.array([9.3, -177.0]), np.array([9.0, 179.5])]
    else:
        g = pmf.Grid([-4.0, -4.0, -3.0], [4.0, 4.0, 3.0], [12, 10, 9])
        F = np.array([[0.95, 0.05, -0.04], [0.03, 0.9, 0.06], [0.0, -0.05, 0.92]])
        Q = np.diag([0.1, 0.15, 0.08])
        comps = [((0, 1), np.hypot(g.axes[0][:, None], g.axes[1][None, :])), ((2,), g.axes[2])]
        R = np.diag([0.3, 0.2])
        z = [np.array([1.1, 0.2]), np.array([0.9, -0.1])]
    m0 = np.array([-10.0, 0.0]) if d == "bearing" else np.zeros(g.d)
    P0 = 2.0 * np.eye(g.d) if d == "bearing" else np.eye(g.d)
    return g, F, Q, R, comps, z, m0, P0


def _dense_ll(g, F, Q, R, comps, z, m0, P0):
    return pmf.run_filter(g, m0, P0, F, Q, comps, R, z)["log_lik"]


@pytest.mark.parametrize("d", [2, 3, "bearing"])
def test_log_likelihood_equals_dense_oracle(d):
    g, F, Q, R, comps, z, m0, P0 = _model(d)
    ll, _, _, _ = grad.gradient(F, Q, R, g, m0, P0, comps, z)
    assert abs(ll - _dense_ll(g, F, Q, R, comps, z, m0, P0)) < 1e-10


@pytest.mark.parametrize("d", [2, 3, "bearing"])
def test_gradient_matches_central_differences(d):
    g, F, Q, R, comps, z, m0, P0 = _model(d)
    d = g.d
    ll, dF, dq, dr = grad.gradient(F, Q, R, g, m0, P0, comps, z)
    h = 1e-6

    def fd(perturb):
        return (_dense_ll(g, *perturb(h), comps, z, m0, P0)
                - _dense_ll(g, *perturb(-h), comps, z, m0, P0)) / (2 * h)

    for i in range(d):
        for j in range(d):
            if F[i, j] == 0.0:
                continue  # structurally zero: a kink of the hat weights
            def pF(e, i=i, j=j):
                F2 = F.copy()
                F2[i, j] += e
                return F2, Q, R
            ref = fd(pF)
            assert abs(dF[i, j] - ref) <= 1e-5 * max(1.0, abs(ref)), (i, j, dF[i, j], ref)
    for m in range(d):
        def pQ(e, m=m):
            Q2 = Q.copy()
            Q2[m, m] += e
            return F, Q2, R
        ref = fd(pQ)
        assert abs(dq[m] - ref) <= 1e-5 * max(1.0, abs(ref)), (m, dq[m], ref)
    for c in range(R.shape[0]):
        def pR(e, c=c):
            R2 = R.copy()
            R2[c, c] += e
            return F, Q, R2
        ref = fd(pR)
        assert abs(dr[c] - ref) <= 1e-5 * max(1.0, abs(ref)), (c, dr[c], ref)
