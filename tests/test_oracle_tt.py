"""Pins for the FP64 tensor-train helpers (oracle/tt.py): the TT definition of
Eq. ttd_exact written as one einsum, Eckart-Young for d = 2, exact recovery of
tensors with known TT ranks, and the rounding error bound."""
import numpy as np
import pytest

from oracle import tt


def _random_tt(n, r, seed):
    rng = np.random.default_rng(seed)
    ranks = [1] + list(r) + [1]
    return [rng.standard_normal((ranks[k], n[k], ranks[k + 1])) for k in range(len(n))]


def test_densify_matches_einsum_definition():
    cores = _random_tt([3, 4, 5, 2], [2, 3, 2], 0)
    full = np.einsum("aib,bjc,ckd,dle->ijkl", *cores)
    np.testing.assert_allclose(tt.densify(cores), full, rtol=1e-13, atol=1e-13)


def test_rank_one_is_outer_product():
    rng = np.random.default_rng(1)
    vs = [rng.random(n) for n in (4, 3, 5)]
    cores = [v.reshape(1, -1, 1) for v in vs]
    np.testing.assert_allclose(tt.densify(cores), np.multiply.outer(np.multiply.outer(*vs[:2]), vs[2]))


def test_inner_and_sum():
    a = _random_tt([4, 3, 5], [2, 3], 2)
    b = _random_tt([4, 3, 5], [3, 2], 3)
    A, B = tt.densify(a), tt.densify(b)
    assert tt.inner(a, b) == pytest.approx(float((A * B).sum()), rel=1e-12)
    assert tt.full_sum(a) == pytest.approx(float(A.sum()), rel=1e-12)


def test_round_two_modes_is_truncated_svd():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((12, 9))
    s = np.linalg.svd(A, compute_uv=False)
    for r in (1, 3, 6):
        out, tails = tt.round_tt(tt.from_dense(A), eps=0.0, rmax=r)
        err = np.linalg.norm(tt.densify(out) - A)
        assert err == pytest.approx(np.sqrt((s[r:] ** 2).sum()), rel=1e-10)
        assert tails[0] == pytest.approx(err / np.linalg.norm(A), rel=1e-10)


def test_round_recovers_exact_ranks():
    cores = _random_tt([5, 6, 4, 5], [3, 4, 2], 5)
    A = tt.densify(cores)
    out, tails = tt.round_tt(cores, eps=1e-12)
    assert tt.ranks(out) == [1, 3, 4, 2, 1]
    np.testing.assert_allclose(tt.densify(out), A, atol=1e-10 * np.abs(A).max())
    # padding with redundant rank is removed
    padded = [np.concatenate([c, np.zeros_like(c)], axis=2) if k < 3 else c for k, c in enumerate(cores)]
    padded = [np.concatenate([c, np.zeros_like(c)], axis=0) if k > 0 else c for k, c in enumerate(padded)]
    out2, _ = tt.round_tt(padded, eps=1e-12)
    assert tt.ranks(out2) == [1, 3, 4, 2, 1]


@pytest.mark.parametrize("eps", [0.3, 0.1, 0.01, 1e-4])
def test_round_error_bound(eps):
    rng = np.random.default_rng(6)
    A = rng.standard_normal((6, 5, 6, 4))
    cores = tt.from_dense(A)
    out, tails = tt.round_tt(cores, eps=eps)
    err = np.linalg.norm(tt.densify(out) - A) / np.linalg.norm(A)
    assert err <= eps * (1 + 1e-10)
    assert err ** 2 <= sum(t * t for t in tails) * (1 + 1e-9) + 1e-24
    # the rank cap overrides eps; the reported tails still bound the error
    out_c, tails_c = tt.round_tt(cores, eps=eps, rmax=2)
    assert max(tt.ranks(out_c)) <= 2
    err_c = np.linalg.norm(tt.densify(out_c) - A) / np.linalg.norm(A)
    assert err_c ** 2 <= sum(t * t for t in tails_c) * (1 + 1e-10)


def test_from_dense_roundtrip():
    A = np.random.default_rng(7).random((3, 4, 5))
    np.testing.assert_allclose(tt.densify(tt.from_dense(A)), A, atol=1e-13)


def test_add_is_elementwise_sum():
    rng = np.random.default_rng(41)
    a = [rng.standard_normal(s) for s in [(1, 5, 2), (2, 4, 3), (3, 6, 1)]]
    b = [rng.standard_normal(s) for s in [(1, 5, 3), (3, 4, 2), (2, 6, 1)]]
    np.testing.assert_allclose(tt.densify(tt.add(a, b)), tt.densify(a) + tt.densify(b),
                               rtol=0, atol=1e-12)
    assert tt.ranks(tt.add(a, b)) == [1, 5, 5, 1]


SHEAR_CASES = [(0, 1, 0.3), (0, 2, -0.45), (2, 0, 0.3), (1, 2, 1.2), (2, 1, -0.2)]


@pytest.mark.parametrize("m,n,a", SHEAR_CASES)
def test_shear_operator_equals_dense_shear(m, n, a):
    """The TT form of the hat shear reproduces the dense push-forward
    (an independent implementation, slice by slice) exactly."""
    from oracle import pmf
    g = pmf.Grid([-5.0, -4.0, -3.0], [5.0, 4.0, 3.0], [20, 16, 12])
    rng = np.random.default_rng(7)
    cores = [rng.random(sh) for sh in [(1, 20, 2), (2, 16, 3), (3, 12, 1)]]
    s = a * g.axes[n] / g.delta_axis[m]
    ref = pmf.shear(tt.densify(cores), g, m, n, a)
    got = tt.densify(tt.shear_operator(cores, m, n, s))
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("m,n,a", SHEAR_CASES)
def test_shear_in_pieces_is_the_sum_of_pieces(m, n, a):
    """The shear as a TT sum of pieces of consecutive shifts is exactly the
    whole operator; rounding every piece and then the sum stays within
    eps (sum of the pieces' norms + the norm of the result)."""
    from oracle import pmf
    g = pmf.Grid([-5.0, -4.0, -3.0], [5.0, 4.0, 3.0], [20, 16, 12])
    rng = np.random.default_rng(8)
    cores = [rng.random(sh) for sh in [(1, 20, 2), (2, 16, 3), (3, 12, 1)]]
    s = a * g.axes[n] / g.delta_axis[m]
    ts = list(range(int(np.floor(s.min())), int(np.floor(s.max())) + 2))
    cuts = [0, len(ts) // 3, 2 * len(ts) // 3, len(ts)]
    pieces = [tt.shear_operator(cores, m, n, s, ts[c0:c1])
              for c0, c1 in zip(cuts[:-1], cuts[1:]) if c1 > c0]
    whole = tt.densify(tt.shear_operator(cores, m, n, s))
    total = pieces[0]
    for p in pieces[1:]:
        total = tt.add(total, p)
    np.testing.assert_allclose(tt.densify(total), whole, rtol=0, atol=1e-12 * np.abs(whole).max())
    eps = 1e-3
    rounded = [tt.round_tt(p, eps)[0] for p in pieces]
    acc = rounded[0]
    for p in rounded[1:]:
        acc = tt.add(acc, p)
    out = tt.densify(tt.round_tt(acc, eps)[0])
    nw = np.linalg.norm(whole)
    bound = eps * (sum(np.linalg.norm(tt.densify(p)) for p in pieces) + nw) / nw
    assert np.linalg.norm(out - whole) / nw <= bound * (1 + 1e-9) + 1e-12
