"""Pins for the dense FP64 oracle (oracle/pmf.py, oracle/kalman.py).

Each test checks the oracle against something other than itself: closed
forms (truncated-normal moments, Gaussian products, Poisson summation of the
kernel), exact moment identities of the discrete operators, exact index
permutations, an independent library convolution, the Kalman filter in the
linear-Gaussian limit and joint-Gaussian conditioning for the Kalman filter.
"""
import math

import numpy as np
import pytest
from scipy import signal, stats

from oracle import kalman, pmf


def _moments_1d(P, x, delta):
    m = float((P * x).sum() * delta)
    v = float((P * (x - m) ** 2).sum() * delta)
    return m, v


# ------------------------------------------------------------------ grid
def test_grid_cell_centres():
    g = pmf.Grid([-10.0, -8.0], [10.0, 8.0], [64, 128])
    assert g.delta_axis[0] == pytest.approx(0.3125)
    assert g.delta_axis[1] == pytest.approx(0.125)
    assert g.axes[0][0] == pytest.approx(-10.0 + 0.15625)
    assert g.axes[0][-1] == pytest.approx(10.0 - 0.15625)
    np.testing.assert_allclose(g.axes[1], -g.axes[1][::-1], atol=1e-15)
    assert g.delta == pytest.approx(0.3125 * 0.125)
    assert g.points().shape == (64 * 128, 2)
    # C order: the last mode runs fastest.
    assert g.points()[1, 1] == pytest.approx(g.axes[1][1])


def test_prior_truncated_normal_moments():
    # 1-D Gaussian cut by the grid: moments are those of the truncated normal.
    mu, var, lo, hi = 0.7, 1.3, -1.5, 3.0
    g = pmf.Grid([lo], [hi], [4000])
    P = pmf.prior(g, [mu], [[var]])
    m, v = _moments_1d(P, g.axes[0], g.delta)
    sd = math.sqrt(var)
    tn = stats.truncnorm((lo - mu) / sd, (hi - mu) / sd, loc=mu, scale=sd)
    assert m == pytest.approx(tn.mean(), abs=2e-7)
    assert v == pytest.approx(tn.var(), abs=2e-7)
    assert float(P.sum() * g.delta) == pytest.approx(1.0, abs=1e-14)


def test_prior_correlated_moments_are_exact():
    # A resolved Gaussian far from the boundary: lattice sums of Gaussians
    # reproduce the continuous moments to exp(-2 pi^2 sigma^2/D^2) ~ 0.
    mean = np.array([0.6, -1.1])
    cov = np.array([[1.2, 0.5], [0.5, 0.9]])
    g = pmf.Grid([-12, -12], [12, 12], [96, 96])
    m, c = pmf.moments(pmf.prior(g, mean, cov), g)
    np.testing.assert_allclose(m, mean, atol=1e-10)
    np.testing.assert_allclose(c, cov, atol=1e-10)


def test_moments_three_modes_cross_terms():
    mean = np.array([0.3, -0.2, 0.5])
    cov = np.array([[1.0, 0.3, -0.2], [0.3, 0.8, 0.25], [-0.2, 0.25, 1.1]])
    g = pmf.Grid([-9, -8, -10], [9, 8, 10], [48, 40, 52])
    m, c = pmf.moments(pmf.prior(g, mean, cov), g)
    np.testing.assert_allclose(m, mean, atol=1e-8)
    np.testing.assert_allclose(c, cov, atol=1e-8)


# ------------------------------------------------------------ LDU / order
def test_ldu_reconstructs():
    rng = np.random.default_rng(5)
    for d in (2, 3, 4, 6):
        F = rng.standard_normal((d, d)) + 3 * np.eye(d)
        L, D, U = pmf.ldu(F)
        np.testing.assert_allclose(L @ np.diag(D) @ U, F, atol=1e-12)
        assert np.allclose(np.triu(L, 1), 0) and np.allclose(np.diag(L), 1)
        assert np.allclose(np.tril(U, -1), 0) and np.allclose(np.diag(U), 1)
    with pytest.raises(np.linalg.LinAlgError):
        pmf.ldu(np.array([[0.0, 1.0], [1.0, 0.0]]))


def test_elementary_ops_compose_to_F():
    rng = np.random.default_rng(6)
    for d in (2, 3, 4, 5):
        F = rng.standard_normal((d, d)) * 0.3 + np.eye(d)
        M = np.eye(d)
        for op in pmf.elementary_ops(F):
            E = np.eye(d)
            if op[0] == "shear":
                E[op[1], op[2]] = op[3]
            else:
                E[op[1], op[1]] = op[2]
            M = E @ M          # ops act in list order on x
        np.testing.assert_allclose(M, F, atol=1e-12)


# ------------------------------------------------------------------ shear
def test_shear_integer_shift_is_permutation():
    # N odd, equal spacing: a * xi_n / D_m = a * (i_n - (N-1)/2) is an integer
    # for integer a, so the shear moves whole cells.
    N = 21
    g = pmf.Grid([-5.25, -5.25], [5.25, 5.25], [N, N])
    rng = np.random.default_rng(1)
    P = rng.random((N, N))
    for a in (1, -2):
        for (m, n) in ((0, 1), (1, 0)):
            out = pmf.shear(P, g, m, n, float(a))
            ref = np.zeros_like(P)
            for im in range(N):
                for inn in range(N):
                    jm = im + a * (inn - (N - 1) // 2)
                    if 0 <= jm < N:
                        if m == 0:
                            ref[jm, inn] = P[im, inn]
                        else:
                            ref[inn, jm] = P[inn, im]
            np.testing.assert_allclose(out, ref, atol=1e-14)


def _exact_cic_moments(P, g, axis_moved, frac_of_cell, A):
    """Moments after moving each cell's mass with the linear map A and
    splitting it between the two neighbouring cells: the mean maps exactly,
    the covariance gains sum(mass * f (1 - f)) D^2 on the moved axis."""
    m0, c0 = pmf.moments(P, g)
    mass = P * g.delta
    extra = float((mass * frac_of_cell * (1 - frac_of_cell)).sum()) * g.delta_axis[axis_moved] ** 2
    c = A @ c0 @ A.T
    c[axis_moved, axis_moved] += extra
    return A @ m0, c


@pytest.mark.parametrize("m,n,a", [(0, 1, 0.37), (1, 0, -0.23), (0, 2, 0.11), (2, 1, 0.29)])
def test_shear_moments_exact(m, n, a):
    g = pmf.Grid([-10, -9, -8], [10, 9, 8], [40, 36, 32])
    P = pmf.prior(g, [0.4, -0.3, 0.2], [[1.0, 0.2, 0.1], [0.2, 0.8, -0.1], [0.1, -0.1, 0.7]])
    out = pmf.shear(P, g, m, n, a)
    assert float(out.sum()) == pytest.approx(float(P.sum()), rel=1e-13)
    s = a * g.axes[n] / g.delta_axis[m]
    f = s - np.floor(s)
    shape = [1, 1, 1]
    shape[n] = -1
    frac = np.broadcast_to(f.reshape(shape), P.shape)
    A = np.eye(3)
    A[m, n] = a
    em, ec = _exact_cic_moments(P, g, m, frac, A)
    gm, gc = pmf.moments(out, g)
    np.testing.assert_allclose(gm, em, atol=1e-9)
    np.testing.assert_allclose(gc, ec, atol=1e-9)


@pytest.mark.parametrize("m,lam", [(0, 0.93), (1, 1.07), (1, 0.5)])
def test_scale_moments_exact(m, lam):
    g = pmf.Grid([-10, -9], [10, 9], [50, 44])
    P = pmf.prior(g, [0.4, -0.3], [[1.1, 0.3], [0.3, 0.9]])
    out = pmf.scale_axis(P, g, m, lam)
    assert float(out.sum()) == pytest.approx(float(P.sum()), rel=1e-13)
    u = (lam * g.axes[m] - g.lo[m]) / g.delta_axis[m] - 0.5
    f = u - np.floor(u)
    shape = [1, 1]
    shape[m] = -1
    frac = np.broadcast_to(f.reshape(shape), P.shape)
    A = np.eye(2)
    A[m, m] = lam
    em, ec = _exact_cic_moments(P, g, m, frac, A)
    gm, gc = pmf.moments(out, g)
    np.testing.assert_allclose(gm, em, atol=1e-9)
    np.testing.assert_allclose(gc, ec, atol=1e-9)


def test_scale_identity():
    g = pmf.Grid([-3, -2], [3, 2], [12, 9])
    P = np.random.default_rng(2).random(g.shape)
    np.testing.assert_allclose(pmf.scale_axis(P, g, 1, 1.0), P, atol=1e-15)
    np.testing.assert_allclose(pmf.regrid(P, g, np.eye(2)), P, atol=1e-15)


# ------------------------------------------------------------ convolution
def test_kernel_sum_poisson_closed_form():
    # sum_t D N(D t; 0, q) = 1 + 2 sum_l exp(-2 pi^2 q l^2 / D^2)  (Poisson).
    for D, q in ((1.0, 0.25), (0.125, 0.05 * 0.03), (0.3125, 0.1)):
        k = pmf.gauss_kernel(D, q, 400)
        closed = 1 + 2 * sum(math.exp(-2 * math.pi ** 2 * q * l * l / D ** 2) for l in range(1, 50))
        assert float(k.sum()) == pytest.approx(closed, rel=1e-13)


def test_convolution_matches_scipy():
    g = pmf.Grid([-4, -3], [4, 3], [24, 19])
    P = np.random.default_rng(3).random(g.shape)
    out = pmf.convolve_axis(pmf.convolve_axis(P, g, 0, 0.3), g, 1, 0.07)
    k0 = pmf.gauss_kernel(g.delta_axis[0], 0.3, 24)
    k1 = pmf.gauss_kernel(g.delta_axis[1], 0.07, 19)
    full = signal.convolve(P, np.outer(k0, k1), mode="full", method="direct")
    ref = full[23:23 + 24, 18:18 + 19]
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-15)


def test_convolution_adds_q():
    g = pmf.Grid([-12, -12], [12, 12], [120, 120])
    P = pmf.prior(g, [0.5, -0.5], [[1.0, 0.4], [0.4, 1.5]])
    q = (0.3, 0.7)
    out = P
    for m in range(2):
        out = pmf.convolve_axis(out, g, m, q[m])
    out, _ = pmf.normalise(out, g)
    m1, c1 = pmf.moments(out, g)
    np.testing.assert_allclose(m1, [0.5, -0.5], atol=1e-10)
    np.testing.assert_allclose(c1, [[1.3, 0.4], [0.4, 2.2]], atol=1e-9)


# --------------------------------------------------------------- predict
def test_predict_textbook_matches_gaussian_pushforward():
    # Riemann sums of Gaussians are exact to exp(-2 pi^2 s^2/D^2): one step of
    # the direct sum maps N(m, P) to N(F m, F P F^T + Q) at the grid points.
    g = pmf.Grid([-10, -10], [10, 10], [64, 64])
    m0 = np.array([1.0, -0.5])
    P0 = np.array([[2.0, 0.3], [0.3, 1.5]])
    F = np.array([[0.9, 0.1], [0.0, 0.9]])
    Q = 0.1 * np.eye(2)
    P = pmf.prior(g, m0, P0)
    out, mass = pmf.predict_textbook(P, g, F, Q)
    ref = pmf.prior(g, F @ m0, F @ P0 @ F.T + Q)
    assert np.max(np.abs(out - ref)) <= 1e-7 * np.max(ref)
    assert mass == pytest.approx(1.0, abs=1e-5)
    # non-triangular F and non-diagonal Q
    F2 = np.array([[0.8, 0.2], [-0.3, 0.95]])
    Q2 = np.array([[0.2, 0.05], [0.05, 0.15]])
    out2, _ = pmf.predict_textbook(P, g, F2, Q2)
    ref2 = pmf.prior(g, F2 @ m0, F2 @ P0 @ F2.T + Q2)
    assert np.max(np.abs(out2 - ref2)) <= 1e-7 * np.max(ref2)


def test_predict_rg_mean_exact_and_cov_converges():
    m0 = np.array([0.8, -0.6])
    P0 = np.array([[1.5, 0.2], [0.2, 1.0]])
    F = np.array([[0.9, 0.1], [-0.05, 0.9]])
    Q = np.diag([0.1, 0.2])
    exact_c = F @ P0 @ F.T + Q
    errs = []
    for N in (32, 64, 128):
        g = pmf.Grid([-10, -10], [10, 10], [N, N])
        out, _ = pmf.predict_rg(pmf.prior(g, m0, P0), g, F, Q)
        m, c = pmf.moments(out, g)
        np.testing.assert_allclose(m, F @ m0, atol=1e-9)
        errs.append(np.abs(c - exact_c).max())
    # numerical diffusion of the hat interpolation is O(D^2): at most D^2/4
    # per elementary op, three ops here (shear, two scalings, shear)
    assert errs[0] > 2.5 * errs[1] > 2.5 * 2.5 * errs[2]
    assert errs[2] < 4 * (20.0 / 128) ** 2 / 4


def test_predict_rg_identity_F_is_pure_convolution():
    g = pmf.Grid([-6, -6], [6, 6], [30, 30])
    P = pmf.prior(g, [0.2, 0.1], [[1.0, 0.2], [0.2, 0.6]])
    out, _ = pmf.predict_rg(P, g, np.eye(2), np.diag([0.05, 0.08]))
    ref = pmf.convolve_axis(pmf.convolve_axis(P, g, 0, 0.05), g, 1, 0.08)
    np.testing.assert_allclose(out, pmf.normalise(ref, g)[0], rtol=1e-13, atol=1e-16)


def test_predict_rg_vanishing_noise_and_identity():
    g = pmf.Grid([-6, -6], [6, 6], [24, 24])
    P = np.random.default_rng(4).random(g.shape)
    P, _ = pmf.normalise(P, g)
    q = (0.001 * g.delta_axis[0]) ** 2
    out, _ = pmf.predict_rg(P, g, np.eye(2), q * np.eye(2))
    np.testing.assert_allclose(out, P, rtol=1e-12)


def test_predict_rejects_non_diagonal_Q():
    g = pmf.Grid([-1, -1], [1, 1], [4, 4])
    with pytest.raises(ValueError):
        pmf.predict_rg(np.ones(g.shape), g, np.eye(2), np.array([[1.0, 0.1], [0.1, 1.0]]))


# ---------------------------------------------------------------- update
def test_update_gaussian_product_closed_form():
    g = pmf.Grid([-10, -10], [10, 10], [128, 128])
    m0 = np.array([0.5, -0.2])
    P0 = np.array([[1.4, 0.35], [0.35, 1.0]])
    P = pmf.prior(g, m0, P0)
    H = np.array([[1.0, 2.0]])
    R = np.array([[0.3]])
    z = np.array([0.9])
    comps = [((0, 1), g.axes[0][:, None] + 2.0 * g.axes[1][None, :])]
    out, logc = pmf.update(P, g, pmf.likelihood(g, comps, z, R))
    S = H @ P0 @ H.T + R
    K = P0 @ H.T @ np.linalg.inv(S)
    mpost = m0 + (K @ (z - H @ m0))
    cpost = P0 - K @ S @ K.T
    m, c = pmf.moments(out, g)
    np.testing.assert_allclose(m, mpost, atol=1e-9)
    np.testing.assert_allclose(c, cpost, atol=1e-9)
    ref = stats.norm(loc=float((H @ m0)[0]), scale=math.sqrt(float(S[0, 0]))).logpdf(0.9)
    assert logc == pytest.approx(ref, abs=1e-9)


def test_likelihood_mode_order_and_one_mode():
    g = pmf.Grid([-2, -3, -1], [2, 3, 1], [5, 7, 4])
    tab = np.random.default_rng(8).random((7, 4))
    L1 = pmf.likelihood(g, [((1, 2), tab)], [0.3], [[0.5]])
    L2 = pmf.likelihood(g, [((2, 1), tab.T)], [0.3], [[0.5]])
    np.testing.assert_allclose(L1, L2, atol=0)
    for i0 in range(5):
        for i1 in range(7):
            for i2 in range(4):
                v = stats.norm(loc=tab[i1, i2], scale=math.sqrt(0.5)).pdf(0.3)
                assert L1[i0, i1, i2] == pytest.approx(v, rel=1e-13)
    tab1 = np.linspace(-1, 1, 5)
    L3 = pmf.likelihood(g, [((0,), tab1), ((2,), np.sin(g.axes[2]))], [0.1, 0.2], np.diag([0.4, 0.6]))
    for i0 in range(5):
        for i2 in range(4):
            v = stats.norm(tab1[i0], math.sqrt(0.4)).pdf(0.1) * stats.norm(
                math.sin(g.axes[2][i2]), math.sqrt(0.6)).pdf(0.2)
            np.testing.assert_allclose(L3[i0, :, i2], v, rtol=1e-13)


def test_angle_residual_is_the_nearest_branch():
    """Brute force: the wrapped residual is, among z - h + 360 k, the one of
    smallest magnitude (either one at a tie, where the squares agree)."""
    rng = np.random.default_rng([11, 0])
    z, h = rng.uniform(-400, 400, 500), rng.uniform(-400, 400, 500)
    r = pmf.residual(z, h, 360.0)
    cand = (z - h)[:, None] + 360.0 * np.arange(-4, 5)[None, :]
    best = cand[np.arange(500), np.argmin(np.abs(cand), axis=1)]
    np.testing.assert_allclose(r * r, best * best, rtol=1e-12, atol=1e-9)
    k = (r - (z - h)) / 360.0
    np.testing.assert_allclose(k, np.round(k), atol=1e-12)
    assert (np.abs(r) <= 180.0 + 1e-9).all()
    np.testing.assert_array_equal(pmf.residual(z, h), z - h)


def test_bearing_likelihood_across_the_cut():
    """A bearing component on a grid across the negative x axis: every
    point's factor is the normal density of its angular distance to z."""
    g = pmf.Grid([-30.0, -10.0], [-10.0, 10.0], [9, 8])
    b = np.degrees(np.arctan2(g.axes[1][None, :], g.axes[0][:, None]))
    L = pmf.likelihood(g, [((0, 1), b, 360.0)], [179.0], [[0.5]])
    for i0 in range(9):
        for i1 in range(8):
            dist = min(abs(179.0 - b[i0, i1]), 360.0 - abs(179.0 - b[i0, i1]))
            assert L[i0, i1] == pytest.approx(stats.norm(0.0, math.sqrt(0.5)).pdf(dist), rel=1e-12)
    assert (b.max() > 150.0) and (b.min() < -150.0)  # the grid spans the cut


# ----------------------------------------------------------- full filter
def test_filter_matches_kalman_textbook_and_rg():
    # Linear-Gaussian variant of config 1: the point-mass filter converges to
    # the Kalman filter as the grid is refined (R = 0.05 is under-resolved at
    # N = 64, D = 0.3125, so agreement there is to discretisation error).
    import synth
    model = synth.config1_linear()
    x, z = synth.simulate(model, 0, steps=8)
    kf = kalman.kalman(model.m0, model.P0, model.F, model.Q, np.eye(2), model.R, z)
    g = pmf.Grid(model.lo, model.hi, model.n)
    masses = []
    out_t = pmf.run_filter(g, model.m0, model.P0, model.F, model.Q, model.tables(g.axes),
                           model.R, z, transition="textbook",
                           callback=lambda k, P: masses.append((P.sum() * g.delta, P.min())))
    for mass, pmin in masses:
        assert mass == pytest.approx(1.0, abs=1e-12) and pmin >= 0.0
    np.testing.assert_allclose(out_t["means"], kf["means"], atol=5e-3)
    np.testing.assert_allclose(out_t["covs"], kf["covs"], atol=5e-3)
    np.testing.assert_allclose(out_t["log_c"], kf["log_c"], atol=3e-2)
    errs = []
    for N in (64, 128, 256):
        g = pmf.Grid(model.lo, model.hi, [N, N])
        o = pmf.run_filter(g, model.m0, model.P0, model.F, model.Q, model.tables(g.axes),
                           model.R, z)
        errs.append((np.abs(o["means"] - kf["means"]).max(), np.abs(o["covs"] - kf["covs"]).max(),
                     np.abs(o["log_c"] - kf["log_c"]).max()))
    for e0, e1 in zip(errs[:-1], errs[1:]):
        assert e0[0] > 2.5 * e1[0] and e0[1] > 2.5 * e1[1] and e0[2] > 2.5 * e1[2]
    assert errs[-1][0] < 5e-3 and errs[-1][1] < 5e-4 and errs[-1][2] < 5e-2


def test_kalman_matches_joint_gaussian_conditioning():
    # Batch form: stack x_1..x_K and z_1..z_K as one Gaussian and condition.
    rng = np.random.default_rng(11)
    d, b, K = 2, 1, 5
    F = np.array([[0.95, 0.2], [-0.1, 0.9]])
    Q = np.array([[0.2, 0.05], [0.05, 0.1]])
    H = np.array([[1.0, -0.5]])
    R = np.array([[0.3]])
    m0 = np.array([0.5, 1.0])
    P0 = np.array([[1.0, 0.2], [0.2, 0.5]])
    zs = rng.standard_normal((K, b))
    # x_k = F^k x_0 + sum_j F^(k-j) w_{j-1}
    Fp = [np.linalg.matrix_power(F, k) for k in range(K + 1)]
    mx = np.concatenate([Fp[k] @ m0 for k in range(1, K + 1)])
    Cx = np.zeros((K * d, K * d))
    for i in range(1, K + 1):
        for j in range(1, K + 1):
            c = Fp[i] @ P0 @ Fp[j].T
            for l in range(1, min(i, j) + 1):
                c = c + Fp[i - l] @ Q @ Fp[j - l].T
            Cx[(i - 1) * d:i * d, (j - 1) * d:j * d] = c
    Hb = np.kron(np.eye(K), H)
    Cz = Hb @ Cx @ Hb.T + np.kron(np.eye(K), R)
    zf = zs.ravel()
    gain = Cx @ Hb.T @ np.linalg.inv(Cz)
    post_m = mx + gain @ (zf - Hb @ mx)
    post_C = Cx - gain @ Hb @ Cx
    kf = kalman.kalman(m0, P0, F, Q, H, R, zs)
    np.testing.assert_allclose(kf["means"][-1], post_m[-d:], atol=1e-12)
    np.testing.assert_allclose(kf["covs"][-1], post_C[-d:, -d:], atol=1e-12)
    ll = stats.multivariate_normal(mean=Hb @ mx, cov=Cz).logpdf(zf)
    assert kf["log_lik"] == pytest.approx(ll, abs=1e-10)


def test_config1_golden_regression():
    """The committed fixture (written by tests/golden/make_golden.py from the
    oracle) still matches: guards against unintended oracle changes."""
    import json
    import os
    import synth
    path = os.path.join(os.path.dirname(__file__), "golden", "config1_oracle.json")
    with open(path) as f:
        gold = json.load(f)
    model = synth.config1()
    x, z = synth.simulate(model, 0)
    np.testing.assert_allclose(z, gold["z"], rtol=0, atol=0)
    g = pmf.Grid(model.lo, model.hi, model.n)
    r = pmf.run_filter(g, model.m0, model.P0, model.F, model.Q, model.tables(g.axes), model.R, z,
                       transition="rg")
    np.testing.assert_allclose(r["means"], gold["rg"]["means"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(r["log_c"], gold["rg"]["log_c"], rtol=1e-12, atol=1e-12)


def test_block_diagonal_model_factors_over_pairs():
    """For a block-diagonal F, diagonal Q, a separable prior and one-mode
    measurements (the d = 6, 8 constant-velocity workload), the re-gridded
    filter's density stays the tensor product of the pairs' 2-D densities:
    every shear couples modes inside one pair, the kernel and the likelihood
    are separable.  This is what the GPU tests at N = 128 and 256 compare the
    TT density against."""
    import synth
    model = synth.config3(d=4, n=12)
    g = pmf.Grid(model.lo, model.hi, model.n)
    oc = model.tables(g.axes)
    z = synth.simulate(model, 0, steps=2)[1]
    P = pmf.prior(g, model.m0, model.P0)
    pairs = []
    for i in range(2):
        s = slice(2 * i, 2 * i + 2)
        gi = pmf.Grid(model.lo[s], model.hi[s], model.n[s])
        pairs.append((gi, model.F[s, s], model.Q[s, s], model.R[i:i + 1, i:i + 1],
                      pmf.prior(gi, model.m0[s], model.P0[s, s])))
    for k in range(2):
        P, _ = pmf.predict_rg(P, g, model.F, model.Q)
        P, logc = pmf.update(P, g, pmf.likelihood(g, oc, z[k], model.R))
        logc_pairs = 0.0
        dens = []
        for i, (gi, Fi, Qi, Ri, Pi) in enumerate(pairs):
            Pi, _ = pmf.predict_rg(Pi, gi, Fi, Qi)
            Pi, lci = pmf.update(Pi, gi, pmf.likelihood(gi, [((0,), oc[i][1])], z[k][i:i + 1], Ri))
            pairs[i] = (gi, Fi, Qi, Ri, Pi)
            dens.append(Pi)
            logc_pairs += lci
        prod = np.einsum("ab,cd->abcd", dens[0], dens[1])
        assert np.abs(P - prod).max() <= 1e-12 * np.abs(P).max()
        assert abs(logc - logc_pairs) < 1e-10
