"""Pins of the float64 TT filter step (oracle/ttfilter.py) against what the
dense oracle and the mathematics fix:

* without truncation (eps = 0, no cap) every TT step is the dense step of
  oracle/pmf.py exactly (to float64 rounding): shears, scalings, the kernel,
  the update and log c, for upper and lower shears, scalings, one- and
  two-mode likelihood factors, and shears applied in pieces;
* with truncation, a rounding's error is exactly the root sum of squares of
  its reported link tails (the links of a left-to-right TT-SVD sweep carry
  orthogonal errors), and stays within eps where the cap does not bind;
* on two modes the rounding is the Eckart-Young truncated SVD;
* the TT moments equal the dense moments of the densified TT."""
import math

import numpy as np
import pytest

import synth
from oracle import pmf, tt
from oracle import ttfilter as T


def rank1_prior(grid, mean, var):
    """Separable Gaussian prior as rank-1 cores, normalised."""
    cores = []
    for m in range(grid.d):
        f = np.exp(-0.5 * (grid.axes[m] - mean[m]) ** 2 / var[m])
        cores.append(f.reshape(1, -1, 1))
    c = tt.full_sum(cores) * grid.delta
    cores[-1] = cores[-1] / c
    return cores


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_exact_predict_and_update_equal_dense_config2():
    model = synth.config2(n=12)
    g = pmf.Grid(model.lo, model.hi, model.n)
    comps = model.tables(g.axes)
    G = rank1_prior(g, model.m0, np.diag(model.P0))
    P = pmf.prior(g, model.m0, model.P0)
    assert rel(tt.densify(G), P) < 1e-13
    _, z = synth.simulate(model, 4, steps=2)
    for k in range(2):
        G, tp, mp = T.predict(G, g, model.F, model.Q, 0.0, None)
        P, mass = pmf.predict_rg(P, g, model.F, model.Q)
        assert rel(tt.densify(G), P) < 1e-12
        assert abs(mp - mass) < 1e-12 * mass
        G, tu, logc = T.update(G, g, comps, z[k], model.R, 0.0, None)
        P, logc_d = pmf.update(P, g, pmf.likelihood(g, comps, z[k], model.R))
        assert rel(tt.densify(G), P) < 1e-12
        assert abs(logc - logc_d) < 1e-12
        assert max(tp + tu) < 1e-13


def test_exact_step_with_lower_shears_scalings_and_pieces():
    # a general F (upper and lower shears, scalings), one-mode likelihoods,
    # and shears spanning more shifts than a piece holds
    d, N = 3, 10
    g = pmf.Grid(np.full(d, -4.0), np.full(d, 4.0), np.full(d, N))
    F = np.array([[0.9, 0.3, -0.2], [0.25, 1.1, 0.4], [-0.3, 0.2, 0.8]])
    L, D, U = pmf.ldu(F)
    assert np.abs(np.tril(L, -1)).max() > 0 and np.any(D != 1.0)
    Q = np.diag([0.2, 0.3, 0.25])
    comps = [((0,), g.axes[0]), ((2,), np.sin(g.axes[2]))]
    R = np.diag([0.5, 0.2])
    z = np.array([0.4, -0.3])
    G = rank1_prior(g, np.zeros(d), np.ones(d))
    P = tt.densify(G)
    for smax in (10, 2):
        Gs, tp, _ = T.predict(G, g, F, Q, 0.0, None, smax=smax)
        Pp, _ = pmf.predict_rg(P, g, F, Q)
        assert rel(tt.densify(Gs), Pp) < 1e-12, smax
        Gu, _, logc = T.update(Gs, g, comps, z, R, 0.0, None)
        Pu, logc_d = pmf.update(Pp, g, pmf.likelihood(g, comps, z, R))
        assert rel(tt.densify(Gu), Pu) < 1e-12
        assert abs(logc - logc_d) < 1e-12


def test_pieces_sum_to_the_whole_shear():
    g = pmf.Grid(np.full(3, -4.0), np.full(3, 4.0), np.full(3, 16))
    G = synth.random_index_bumps_tt(g.n, 3, seed=5)
    s, ts = T.shear_shifts(g, 0, 2, 0.7)
    assert len(ts) > 4
    whole = tt.shear_operator(G, 0, 2, s, ts)
    pieces = [tt.shear_operator(G, 0, 2, s, ts[a:b]) for a, b in ((0, 2), (2, 4), (4, len(ts)))]
    assert rel(tt.densify(T.add_block(pieces, 0, 2)), tt.densify(whole)) < 1e-14


@pytest.mark.parametrize("rmax", [None, 6, 3])
def test_rounding_error_is_the_root_sum_of_tails(rmax):
    # a shear expands ranks; rounding the block: ||A - round(A)|| / ||A|| is
    # sqrt(sum tau^2) (orthogonal link errors), <= eps without a cap
    model = synth.config2(n=16)
    g = pmf.Grid(model.lo, model.hi, model.n)
    G = synth.random_index_bumps_tt(g.n, 5, seed=2)
    T.canonical(G, 1, 3)
    s, ts = T.shear_shifts(g, 1, 3, 0.9)
    A = tt.shear_operator(G, 1, 3, s, ts)
    B = [c.copy() for c in A]
    eps = 1e-3
    tails = T.round_block(B, 1, 3, eps, rmax)
    err = rel(tt.densify(B), tt.densify(A))
    assert abs(err - math.sqrt(sum(t * t for t in tails))) < 1e-9
    if rmax is None:
        assert err <= eps * (1 + 1e-9)
    else:
        assert max(tt.ranks(B)[2:4]) <= rmax  # links 1 and 2, inside the block
        assert tt.ranks(B)[1] == tt.ranks(A)[1]  # link 0 is outside the block
        assert err > eps  # the cap binds at these ranks


def test_update_rounding_error_is_the_root_sum_of_tails():
    model = synth.config2(n=16)
    g = pmf.Grid(model.lo, model.hi, model.n)
    comps = model.tables(g.axes)
    G = synth.random_index_bumps_tt(g.n, 4, seed=9)
    z = np.array([1.3])
    exact, _, logc0 = T.update(G, g, comps, z, model.R, 0.0, None)
    for rmax in (None, 4):
        Gt, tails, logc = T.update(G, g, comps, z, model.R, 1e-3, rmax)
        assert abs(logc - logc0) < 1e-12  # log c is taken before rounding
        # both are normalised by their own mass: compare up to that scale
        A, B = tt.densify(exact), tt.densify(Gt)
        B = B * (np.vdot(A, B) / np.vdot(B, B))
        err = rel(B, A)
        bound = math.sqrt(sum(t * t for t in tails))
        assert err <= bound * (1 + 1e-6) + 1e-12
        if rmax is None:
            assert bound <= 1e-3 * (1 + 1e-9)


def test_two_mode_rounding_is_eckart_young():
    rng = np.random.default_rng([7, 1, 0])
    A = rng.standard_normal((30, 20)) @ np.diag(0.7 ** np.arange(20)) @ rng.standard_normal((20, 25))
    cores = [A.reshape(1, 30, 25), np.eye(25).reshape(25, 25, 1)]
    for r in (1, 4, 9):
        G, tails = T.round_full(cores, 0.0, r)
        U, s, Vt = np.linalg.svd(A, full_matrices=False)
        best = (U[:, :r] * s[:r]) @ Vt[:r]
        assert rel(tt.densify(G), best) < 1e-12
        assert abs(tails[0] - np.sqrt((s[r:] ** 2).sum()) / np.linalg.norm(A)) < 1e-12


def test_tt_moments_equal_dense_moments():
    g = pmf.Grid(np.array([-3.0, -2.0, -4.0]), np.array([5.0, 2.0, 1.0]), np.array([9, 11, 8]))
    G = synth.random_index_bumps_tt(g.n, 3, seed=4)
    G[-1] = G[-1] / (tt.full_sum(G) * g.delta)
    m_tt, c_tt = T.moments(G, g)
    m_d, c_d = pmf.moments(tt.densify(G), g)
    np.testing.assert_allclose(m_tt, m_d, rtol=0, atol=1e-12)
    np.testing.assert_allclose(c_tt, c_d, rtol=0, atol=1e-12)


def test_rel_distance_by_inner_products():
    g = pmf.Grid(np.full(3, -1.0), np.full(3, 1.0), np.full(3, 7))
    a = synth.random_index_bumps_tt(g.n, 2, seed=1)
    b = synth.random_index_bumps_tt(g.n, 3, seed=3)
    assert abs(T.rel_distance(a, b) - rel(tt.densify(a), tt.densify(b))) < 1e-7


def test_rank_is_borderline():
    # singular values 1, 0.1, 0.01, 1e-3, 1e-4; threshold 1.02e-3 keeps rank 3
    # (tail of rank 3 is 1.005e-3 <= thr, tail of rank 2 is 1.0e-2 > thr)
    s = np.array([1.0, 0.1, 0.01, 1e-3, 1e-4])
    rec = {"s": s, "thr": 1.02e-3, "rank": 3, "rmax": None}
    assert T._rank_and_tail(s, rec["thr"], None)[0] == 3
    assert T.rank_is_borderline(rec, 3, 0.0)
    assert T.rank_is_borderline(rec, 4, 0.25)       # tail of rank 3 is 0.985 thr: at the threshold
    assert not T.rank_is_borderline(rec, 4, 0.01)
    assert not T.rank_is_borderline(rec, 2, 0.25)   # tail of rank 2 is 9.8 thr
    assert not T.rank_is_borderline(rec, 5, 0.25)   # tail of rank 4 is 0.1 thr
    capped = dict(rec, rmax=3)
    assert not T.rank_is_borderline(capped, 4, 0.25)  # above the cap


@pytest.mark.parametrize("where", ["first quadrant", "across the cut"])
def test_two_two_mode_components_equal_dense_update(where):
    """Range and bearing on modes (0, 1) (the radar measurement of Sec. 5):
    without truncation the TT update equals the dense update, log c included;
    on a grid across the negative x axis the bearing's residual is taken on
    its nearer branch by both."""
    if where == "first quadrant":
        g = pmf.Grid([5.0, 6.0, -2.0], [15.0, 14.0, 2.0], [14, 12, 6])
        z = np.array([13.5, 41.0, 0.2])
    else:
        g = pmf.Grid([-15.0, -4.0, -2.0], [-5.0, 4.0, 2.0], [14, 12, 6])
        z = np.array([10.5, 178.5, 0.2])
    X, Y = g.axes[0][:, None], g.axes[1][None, :]
    comps = [((0, 1), np.hypot(X, Y)), ((0, 1), np.degrees(np.arctan2(Y, X)), 360.0), ((2,), g.axes[2])]
    R = np.diag([1.0, 0.1, 0.3])
    G = synth.random_index_bumps_tt(g.n, 3, seed=4)
    P = tt.densify(G)
    P = P / (P.sum() * g.delta)
    G[-1] = G[-1] / (tt.full_sum(G) * g.delta)
    Gt, _, logc = T.update(G, g, comps, z, R, 0.0, None)
    Pd, logc_d = pmf.update(P, g, pmf.likelihood(g, comps, z, R))
    assert rel(tt.densify(Gt), Pd) < 1e-12
    assert abs(logc - logc_d) < 1e-12
