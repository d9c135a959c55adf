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
