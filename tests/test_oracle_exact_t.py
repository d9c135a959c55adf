"""Pins of the TT predictive step with the textbook transition
(oracle/ttfilter.predict_exact: the mode factors of Eq. TPMmat for an upper
bidiagonal F, coupled factors on 2-site blocks): against the dense textbook
transition (pmf.predict_textbook), the Gaussian closed form, and the
re-gridded transition's interpolation smear."""
import numpy as np
import pytest

import synth
from oracle import cross as X
from oracle import pmf, tt
from oracle import ttfilter as T


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _state(g, seed):
    G = synth.random_index_bumps_tt(g.n, 3, seed=seed)
    G[-1] = G[-1] / (tt.full_sum(G) * g.delta)
    P = tt.densify(G)
    return G, P / (P.sum() * g.delta)


@pytest.mark.parametrize("case", ["d3 two couplings", "d4 constant-velocity pairs", "d2 diagonal"])
def test_exact_equals_dense_textbook(case):
    if case == "d3 two couplings":
        g = pmf.Grid([-3.0, -2.5, -2.0], [3.0, 2.5, 2.0], [12, 10, 9])
        F = np.array([[1.0, 0.3, 0.0], [0.0, 0.95, -0.2], [0.0, 0.0, 1.1]])
        Q = np.diag([0.1, 0.2, 0.15])
    elif case == "d4 constant-velocity pairs":
        g = pmf.Grid([-4.0, -2.0, -4.0, -2.0], [4.0, 2.0, 4.0, 2.0], [8, 6, 7, 5])
        F = np.array([[1.0, 0.5, 0, 0], [0, 1.0, 0, 0], [0, 0, 1.0, 0.5], [0, 0, 0, 1.0]])
        Q = np.diag([0.05, 0.1, 0.08, 0.12])
    else:
        g = pmf.Grid([-3.0, -3.0], [3.0, 3.0], [14, 13])
        F = np.diag([0.9, 1.05])
        Q = np.diag([0.2, 0.1])
    G, P = _state(g, 7)
    Pt, mt = pmf.predict_textbook(P, g, F, Q)
    Ge, _, me = T.predict_exact(G, g, F, Q, 0.0, None)
    assert rel(tt.densify(Ge), Pt) < 1e-12
    assert abs(me - mt) < 1e-12
    # the cross at full rank interpolates the 2-site blocks exactly
    Gc, _, mc = T.predict_exact(G, g, F, Q, 0.0, None, cross={"s": 64})
    assert rel(tt.densify(Gc), Pt) < 1e-11


def test_truncated_exact_step_within_its_tails_and_cross_matches():
    """With eps and a rank cap the step's error against the untruncated step
    (equal to the dense textbook transition, pinned above on grids the dense
    matrix fits) is within 10 (eps + tails) (the roundings' discarded norms),
    and the cross at rank cap + 8 gives the exact block's truncation."""
    g = pmf.Grid([-4.0, -2.0, -4.0, -2.0], [4.0, 2.0, 4.0, 2.0], [24, 20, 24, 20])
    F = np.array([[1.0, 0.4, 0, 0], [0, 1.0, 0, 0], [0, 0, 1.0, 0.4], [0, 0, 0, 1.0]])
    Q = np.diag([0.02, 0.05, 0.03, 0.04])
    G, P = _state(g, 11)
    Pt = tt.densify(T.predict_exact(G, g, F, Q, 0.0, None)[0])
    Ge, te, _ = T.predict_exact(G, g, F, Q, 1e-6, 8)
    Gc, tc, _ = T.predict_exact(G, g, F, Q, 1e-6, 8, cross={"s": 16})
    e, ec = rel(tt.densify(Ge), Pt), rel(tt.densify(Gc), Pt)
    assert e <= 10 * (1e-6 + sum(te)), (e, te)
    assert ec <= 10 * (1e-6 + sum(te)), (ec, te)
    assert tt.ranks(Gc) == tt.ranks(Ge)


def test_exact_transition_keeps_the_gaussian_pushforward():
    """A constant-velocity pair: the exact step maps N(m, P) to
    N(F m, F P F^T + Q) up to the grid's point-mass moment error, which
    shrinks with the grid; the re-gridded transition adds its shear's
    interpolation smear (about D^2 / 6 per shift step) to the position
    variance, and so lands farther from the closed form."""
    F = np.array([[1.0, 0.5], [0.0, 1.0]])
    Q = np.diag([0.01, 0.02])
    m0, P0 = np.array([0.3, -0.2]), np.array([[0.3, 0.05], [0.05, 0.2]])
    g = pmf.Grid([-4.0, -3.0], [4.0, 3.0], [64, 48])
    P = pmf.prior(g, m0, P0)
    X0 = [np.asarray(c) for c in tt.from_dense(P, 0.0)]
    Ge, _, _ = T.predict_exact(X0, g, F, Q, 1e-12, None)
    me, ce = pmf.moments(tt.densify(Ge), g)
    Prg, _ = pmf.predict_rg(P, g, F, Q)
    mr, cr = pmf.moments(Prg, g)
    mp, cp = pmf.moments(P, g)  # the gridded prior's own moments
    c_ref = F @ cp @ F.T + Q
    np.testing.assert_allclose(me, F @ mp, atol=1e-6)
    assert abs(ce[0, 0] - c_ref[0, 0]) < 1e-4
    assert abs(cr[0, 0] - c_ref[0, 0]) > 5 * abs(ce[0, 0] - c_ref[0, 0])


def test_rejects_other_couplings():
    g = pmf.Grid([-1.0] * 3, [1.0] * 3, [4] * 3)
    G, _ = _state(g, 1)
    with pytest.raises(ValueError):
        T.predict_exact(G, g, np.array([[1, 0, 0.2], [0, 1, 0], [0, 0, 1.0]]), np.eye(3), 0.0, None)
    with pytest.raises(ValueError):
        T.predict_exact(G, g, np.array([[1, 0, 0], [0.1, 1, 0], [0, 0, 1.0]]), np.eye(3), 0.0, None)
    with pytest.raises(ValueError):
        T.predict_exact(G, g, np.eye(3), np.ones((3, 3)) + np.eye(3), 0.0, None)


def test_transition_block_value_is_the_2site_sum():
    """TransitionBlock's entries by brute force over i for random cores."""
    rng = np.random.default_rng([41])
    G0, G1 = rng.standard_normal((2, 5, 3)), rng.standard_normal((3, 4, 2))
    K = rng.standard_normal((5, 5, 4))
    blk = X.TransitionBlock([G0, G1], K)
    for a in range(2):
        for j in range(5):
            for i1 in range(4):
                for b in range(2):
                    ref = sum(K[j, i, i1] * float(G0[a, i, :] @ G1[:, i1, b]) for i in range(5))
                    assert blk.value((a * 5 + j, i1 * 2 + b)) == pytest.approx(ref, rel=1e-12, abs=1e-12)
