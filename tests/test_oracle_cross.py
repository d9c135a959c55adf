"""Pins of the deterministic TT cross (oracle/cross.py) and of the block
update of the oracle TT filter that uses it (oracle/ttfilter.update_block):
against brute force, exactness properties of skeleton decompositions and the
dense filter."""
import itertools
import math

import numpy as np
import pytest

import synth
from oracle import cross as X
from oracle import pmf, tt
from oracle import ttfilter as T


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ------------------------------------------------------------------ maxvol
def test_lu_rows_hand_example():
    """By hand: column 0's largest magnitude is row 2 (1.0).  Eliminating it,
    column 1 becomes col1 + 0.2 col0 = [0.4, 0.12, 0, -0.34], whose largest
    free entry is row 0; without the elimination it would be row 3 (0.4 >
    0.3)."""
    Q = np.array([[0.5, 0.3], [0.1, 0.1], [-1.0, 0.2], [0.3, -0.4]])
    assert X.lu_rows(Q) == [2, 0]


@pytest.mark.parametrize("seed", range(6))
def test_maxvol_is_dominant_and_near_max_volume(seed):
    """Brute force over every row subset: B[rows] = I, every |B_ij| <= 1 +
    delta, and so (Hadamard's bound on det B[S]) the volume is within a
    factor (sqrt(n) (1 + delta))^n of the largest."""
    rng = np.random.default_rng([21, seed])
    M, n = 9, 3
    Q = X.orth(rng.standard_normal((M, n)) * rng.uniform(0.1, 3.0, (M, 1)))
    delta = 0.05
    rows, B = X.maxvol(Q, delta)
    assert len(set(rows)) == n
    np.testing.assert_allclose(B[rows], np.eye(n), atol=1e-12)
    np.testing.assert_allclose(B, Q @ np.linalg.inv(Q[rows]), atol=1e-10)
    assert np.abs(B).max() <= 1 + delta + 1e-12
    vol = abs(np.linalg.det(Q[rows]))
    best = max(abs(np.linalg.det(Q[list(S)])) for S in itertools.combinations(range(M), n))
    assert vol >= best / (math.sqrt(n) * (1 + delta)) ** n
    # with delta = 0 exchanges continue to a dominant submatrix of (locally) maximal volume
    rows0, B0 = X.maxvol(Q, 0.0, max_iter=1000)
    assert np.abs(B0).max() <= 1 + 1e-10


def test_select_rows_pads_by_row_norm():
    Y = np.zeros((6, 1))
    Y[:, 0] = [0.1, 3.0, -0.5, 2.0, 0.0, -2.5]
    rows, _ = X.select_rows(Y, 3)
    assert rows == [1, 5, 3]  # maxvol of one column: its largest entry; then by |row|


# ------------------------------------------------------------------ cross
def _random_block(N, ranks, seed):
    rng = np.random.default_rng([22, seed])
    return [rng.standard_normal((ranks[q], N[q], ranks[q + 1])) for q in range(len(N))]


@pytest.mark.parametrize("k", [2, 3, 4])
def test_cross_is_exact_at_sufficient_rank(k):
    """A block whose likelihood-weighted tensor has TT ranks <= s (random
    cores of rank 2 inside, boundary ranks 3 and 2, and a separable positive
    likelihood, which keeps the ranks) is reproduced exactly: a skeleton
    decomposition is exact when the rank of the intersection equals the rank
    of the matrix."""
    N = [5, 4, 6, 3][:k]
    cores = _random_block(N, [3] + [2] * (k - 1) + [2], k)
    rng = np.random.default_rng([23, k])
    lik = np.ones(N)
    for q in range(k):
        sh = [1] * k
        sh[q] = N[q]
        lik = lik * rng.uniform(0.5, 2.0, N[q]).reshape(sh)
    blk = X.Block(cores, lik)
    out, sets = X.block_cross(cores, lik, s=6, sweeps=1)
    ref = X.Block(out, np.ones(N)).dense()
    assert rel(ref, blk.dense()) < 1e-11


def test_cross_at_full_rank_is_exact_for_any_tensor():
    """s at least the size of every unfolding: the cross interpolates every
    entry (random cores and a random positive likelihood of full rank)."""
    N = [4, 3, 5]
    cores = _random_block(N, [2, 3, 3, 2], 7)
    lik = np.random.default_rng([24]).uniform(0.1, 1.0, N)
    out, _ = X.block_cross(cores, lik, s=40, sweeps=1)
    assert rel(X.Block(out, np.ones(N)).dense(), X.Block(cores, lik).dense()) < 1e-11


def test_cross_interpolates_its_last_fibers():
    """At the final left index set the approximation equals the tensor on
    the whole last mode (nested rows with B[rows] = I make every left part a
    unit vector), here with a rank well below the tensor's."""
    N = [6, 5, 6]
    cores = _random_block(N, [1, 4, 4, 1], 9)
    lik = np.random.default_rng([25]).uniform(0.1, 1.0, N)
    out, sets = X.block_cross(cores, lik, s=3, sweeps=1)
    blk = X.Block(cores, lik)
    approx = X.Block(out, np.ones(N))
    for alpha in sets["I"][2]:
        for v in range(N[2]):
            assert approx.value(alpha + (v,)) == pytest.approx(blk.value(alpha + (v,)), rel=1e-10, abs=1e-12)


# --------------------------------------------------------- filter update
def _prior_tt(g, m0, var):
    G = [np.exp(-0.5 * (g.axes[m] - m0[m]) ** 2 / var[m]).reshape(1, -1, 1) for m in range(g.d)]
    T.normalise(G, g)
    return G


@pytest.mark.parametrize("case", ["three modes", "two modes (3, 1)", "angle on (1, 2)"])
def test_block_update_exact_equals_dense(case):
    """Without truncation the TT update with a block component (formed
    exactly) equals the dense update, log c included; also together with a
    one-mode and a (0, 1) component, and for a factor given on modes in
    decreasing order."""
    g = pmf.Grid([-3.0, -3.0, -2.5, -2.0], [3.0, 3.0, 2.5, 2.0], [8, 7, 6, 5])
    G = synth.random_index_bumps_tt(g.n, 3, seed=31)
    G[-1] = G[-1] / (tt.full_sum(G) * g.delta)
    P = tt.densify(G)
    P = P / (P.sum() * g.delta)
    ax = g.axes
    if case == "three modes":
        tab = np.sqrt(ax[0][:, None, None] ** 2 + ax[1][None, :, None] ** 2 + ax[2][None, None, :] ** 2)
        comps = [((3,), ax[3]), ((0, 1, 2), tab)]
        z = np.array([0.2, 2.1])
    elif case == "two modes (3, 1)":
        tab = ax[3][:, None] * np.cos(ax[1][None, :])
        comps = [((0, 1), np.hypot(ax[0][:, None], ax[1][None, :])), ((3, 1), tab)]
        z = np.array([1.5, 0.3])
    else:
        tab = np.degrees(np.arctan2(ax[2][None, :], ax[1][:, None]))
        comps = [((1, 2), tab, 360.0)]
        z = np.array([175.0])
    R = np.diag([0.4, 0.3][:len(comps)])
    Gt, _, logc = T.update(G, g, comps, z, R, 0.0, None)
    Pd, logc_d = pmf.update(P, g, pmf.likelihood(g, comps, z, R))
    assert rel(tt.densify(Gt), Pd) < 1e-12
    assert abs(logc - logc_d) < 1e-12


def test_block_update_by_cross_matches_exact_truncation():
    """A 3-D range (||x[0:3]||, R = 0.05) on a 32^4 grid with a Gaussian
    prior: the cross (s = rank cap + 8, one refinement sweep) and the exact
    block product, both rounded with eps 1e-6 and rank cap 16, are within
    1e-6 of each other and of the dense update, log c within 1e-8."""
    n = 32
    g = pmf.Grid([-4.0] * 4, [4.0] * 4, [n] * 4)
    m0, var = np.array([1.5, 1.0, 0.5, 0.0]), np.ones(4)
    G = _prior_tt(g, m0, var)
    P = pmf.prior(g, m0, np.diag(var))
    ax = g.axes
    tab = np.sqrt(ax[0][:, None, None] ** 2 + ax[1][None, :, None] ** 2 + ax[2][None, None, :] ** 2)
    comps = [((0, 1, 2), tab)]
    R, z = np.array([[0.05]]), np.array([2.2])
    Pd, logc_d = pmf.update(P, g, pmf.likelihood(g, comps, z, R))
    Ge, te, lce = T.update(G, g, comps, z, R, 1e-6, 16)
    Gc, tc, lcc = T.update(G, g, comps, z, R, 1e-6, 16, cross={"s": 24, "sweeps": 1})
    e_exact, e_cross = rel(tt.densify(Ge), Pd), rel(tt.densify(Gc), Pd)
    assert e_exact < 1e-6 and e_cross < 1e-6, (e_exact, e_cross)
    assert rel(tt.densify(Gc), tt.densify(Ge)) < 1e-6
    assert abs(lcc - logc_d) < 1e-8 and abs(lce - logc_d) < 1e-12
    assert tt.ranks(Gc) == tt.ranks(Ge)
