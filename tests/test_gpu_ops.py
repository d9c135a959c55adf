"""GPU parity of every TT operation of the step against the dense FP64 oracle,
element by element on the densified TT (C ABI through the Python binding).

Inputs are seeded: random positive index-space bump TTs (synth) or oracle
densities; no input or expected value comes from the CUDA path.  Where an
operation rounds, the bound 10 (eps + tau) + 1e-5 takes tau from the float64
TT filter of oracle/ttfilter.py on the same cores, and the GPU's ranks must
equal that oracle's."""
import numpy as np
import pytest

import synth
from oracle import pmf, tt
from oracle import ttfilter as T

from gpu_util import lib_module, rel, tt_tol

pytestmark = pytest.mark.gpu

LO = [-5.0, -4.0, -3.0, -4.0]
HI = [5.0, 4.0, 3.0, 4.0]
N = [20, 16, 12, 14]
EPS = 1e-6


@pytest.fixture(scope="module")
def G():
    return lib_module()


def bumps_filter(G, d=3, terms=3, seed=0, cap=16, smax=10, batch=1, n=None, conv="auto"):
    n = N[:d] if n is None else n
    f = G.TTFilter(LO[:d], HI[:d], n, np.zeros(d), np.ones(d), batch=batch, rank_cap=cap, eps=EPS,
                   max_shift_span=smax, conv=conv)
    cores = [c.astype(np.float32) for c in synth.random_index_bumps_tt(n, terms, seed)]
    for b in range(batch):
        f.import_cores(b, cores)
    g = pmf.Grid(LO[:d], HI[:d], n)
    return f, g, tt.densify([c.astype(np.float64) for c in cores])


def bumps_cores(d=3, terms=3, seed=0, n=None):
    """The float32 input cores of bumps_filter, as the oracle sees them."""
    n = N[:d] if n is None else n
    return [c.astype(np.float32).astype(np.float64)
            for c in synth.random_index_bumps_tt(n, terms, seed)]


def test_prior_matches_oracle(G):
    mean, var = [0.3, -0.2, 0.1], [1.0, 0.8, 0.5]
    f = G.TTFilter(LO[:3], HI[:3], N[:3], mean, var, batch=2)
    g = pmf.Grid(LO[:3], HI[:3], N[:3])
    ref = pmf.prior(g, mean, np.diag(var))
    for b in range(2):
        assert rel(tt.densify(f.export_cores(b)), ref) < 1e-6
    assert (f.ranks() == 1).all()
    m, c, lc, ll = f.estimate()
    mo, co = pmf.moments(ref, g)
    np.testing.assert_allclose(m[0], mo, atol=1e-6)
    np.testing.assert_allclose(c[0], co, atol=1e-6)


@pytest.mark.parametrize("m,n,a", [(0, 1, 0.3), (0, 2, -0.25), (2, 0, 0.2), (1, 2, 0.15), (2, 1, -0.1)])
def test_shear_unrounded_is_exact(G, m, n, a):
    f, g, P = bumps_filter(G)
    f.shear(m, n, a, do_round=False)
    ref = pmf.shear(P, g, m, n, a)
    assert rel(tt.densify(f.export_cores(0)), ref) < 1e-6
    S = f.ranks()[0]
    lo, hi = min(m, n), max(m, n)
    assert all(S[l] > 3 for l in range(lo + 1, hi + 1))


@pytest.mark.parametrize("m,n,a", [(0, 1, 0.3), (0, 2, -0.25), (2, 0, 0.2)])
def test_shear_rounded_within_eps(G, m, n, a):
    f, g, P = bumps_filter(G)
    f.shear(m, n, a, do_round=True)
    X, tails = T.shear_round(bumps_cores(), g, m, n, a, EPS, 16)
    ref = pmf.shear(P, g, m, n, a)
    assert rel(tt.densify(f.export_cores(0)), ref) <= tt_tol(EPS, sum(tails))
    assert f.ranks()[0].tolist() == tt.ranks(X)


@pytest.mark.parametrize("m,n,a,smax", [(0, 1, 0.3, 3), (0, 2, -0.45, 3), (2, 0, 0.3, 4),
                                         (1, 2, 1.2, 4), (2, 1, -0.2, 3)])
def test_wide_shear_in_pieces_within_eps(G, m, n, a, smax):
    """Shears spanning 5-15 shifts with an expansion capacity of 3-4 shifts:
    2-4 rounded pieces (adjacent and non-adjacent couplings, both triangles)
    whose TT sum is rounded again."""
    f, g, P = bumps_filter(G, smax=smax)
    f.shear(m, n, a, do_round=True)
    X, tails = T.shear_round(bumps_cores(), g, m, n, a, EPS, 16, smax)
    ref = pmf.shear(P, g, m, n, a)
    assert rel(tt.densify(f.export_cores(0)), ref) <= tt_tol(EPS, sum(tails))
    assert f.ranks()[0].tolist() == tt.ranks(X)


@pytest.mark.parametrize("conv", ["dense", "fft"])
def test_scale_and_convolve_are_exact(G, conv):
    """The kernel as the dense Toeplitz product or as zero-padded FFT
    convolutions (float32 transforms: relative error a few u log2 M)."""
    f, g, P = bumps_filter(G, conv=conv)
    f.scale(1, 0.93)
    assert rel(tt.densify(f.export_cores(0)), pmf.scale_axis(P, g, 1, 0.93)) < 1e-6
    f, g, P = bumps_filter(G, conv=conv)
    q = [0.05, 0.1, 0.02]
    f.convolve(q)
    ref = P
    for k in range(3):
        ref = pmf.convolve_axis(ref, g, k, q[k])
    assert rel(tt.densify(f.export_cores(0)), ref) < 1e-6


def test_round_recovers_rank_and_bound(G):
    # a rank-3 TT represented with ranks 9: rounding returns rank 3, same tensor
    f, g, P = bumps_filter(G, terms=3)
    f.shear(0, 1, 0.0, do_round=False)   # zero shear: rank x S representation of the same tensor
    assert f.ranks()[0][1] > 3
    f.round()
    assert f.ranks()[0].tolist() == [1, 3, 3, 1]
    assert rel(tt.densify(f.export_cores(0)), P) < 1e-5
    # eps-truncation of a full-rank tensor: error within eps * ||A|| (+ fp32)
    rng = np.random.default_rng(3)
    A = np.exp(-rng.random((12, 10, 11)) * 4.0)
    cores = tt.from_dense(A)
    f2 = G.TTFilter([-1, -1, -1], [1, 1, 1], [12, 10, 11], [0, 0, 0], [1, 1, 1], rank_cap=16,
                    eps=1e-3)
    f2.import_cores(0, [c.astype(np.float32) for c in cores])
    f2.round()
    err = rel(tt.densify(f2.export_cores(0)), A)
    assert err <= 1e-3 + 1e-5
    ref_cores, _ = tt.round_tt(cores, 1e-3, 16)
    assert abs(err - rel(tt.densify(ref_cores), A)) < 2e-4


@pytest.mark.parametrize("scale", [1e-16, 1e-8, 1e8, 1e16])
def test_round_scale_invariant_at_extreme_magnitudes(G, scale):
    """Rounding commutes with scaling: a core of magnitude 1e-16 or 1e16
    (sums of squares outside [1e-30, 1e30], so the QR reflectors take their
    rescaled path) gives the scaled result of the unit-scale rounding."""
    f, g, P = bumps_filter(G, terms=3)
    f.shear(0, 1, 0.0, do_round=False)
    f.round()
    ref = tt.densify(f.export_cores(0))
    f2, _, _ = bumps_filter(G, terms=3)
    cores = f2.export_cores(0)
    cores[1] = cores[1] * np.float32(scale)
    f2.import_cores(0, cores)
    f2.shear(0, 1, 0.0, do_round=False)
    f2.round()
    out = f2.export_cores(0)
    assert all(np.isfinite(c).all() for c in out)
    assert f2.ranks()[0].tolist() == f.ranks()[0].tolist()
    assert rel(tt.densify([c.astype(np.float64) for c in out]) / scale, ref) < 1e-5


@pytest.mark.parametrize("conv", ["dense", "fft"])
def test_predict_one_step(G, conv):
    """Upper-triangular F (scalings fused into the kernel: the FFT path
    gathers them while loading) and a general F (L shears after the
    scalings, which then run as their own pass)."""
    F = np.array([[0.95, 0.04, -0.03], [0.0, 0.97, 0.05], [0.0, 0.0, 0.92]])
    Q = np.diag([0.05, 0.08, 0.03])
    f, g, P = bumps_filter(G, conv=conv)
    f.predict(F, Q)
    X, tails, _ = T.predict(bumps_cores(), g, F, Q, EPS, 16)
    ref, mass = pmf.predict_rg(P / (P.sum() * g.delta), g, F, Q)
    assert rel(tt.densify(f.export_cores(0)), ref) <= tt_tol(EPS, sum(tails))
    assert f.ranks()[0].tolist() == tt.ranks(X)
    # non-triangular F: L shears follow the scalings
    F2 = np.array([[0.95, 0.04, 0.0], [-0.05, 0.97, 0.02], [0.03, 0.0, 0.92]])
    f, g, P = bumps_filter(G, conv=conv)
    f.predict(F2, Q)
    X, tails, _ = T.predict(bumps_cores(), g, F2, Q, EPS, 16)
    ref, _ = pmf.predict_rg(P / (P.sum() * g.delta), g, F2, Q)
    assert rel(tt.densify(f.export_cores(0)), ref) <= tt_tol(EPS, sum(tails))
    assert f.ranks()[0].tolist() == tt.ranks(X)


def test_update_one_and_two_mode_components(G):
    import torch
    f, g, P = bumps_filter(G, batch=2)
    Pn = P / (P.sum() * g.delta)
    f.normalise()
    axes = f.grid_axes()
    hr = np.sqrt(axes[0][:, None] ** 2 + axes[1][None, :] ** 2)
    hs = np.sin(axes[2])
    comps = [((0, 1), torch.tensor(hr, dtype=torch.float32, device="cuda")),
             ((2,), torch.tensor(hs, dtype=torch.float32, device="cuda"))]
    R = np.diag([0.05, 0.1])
    z = np.array([[1.5, 0.3], [2.0, -0.5]])
    f.update(comps, R, z)
    m, c, lc, ll = f.estimate()
    ocomps = [((0, 1), np.sqrt(g.axes[0][:, None] ** 2 + g.axes[1][None, :] ** 2)),
              ((2,), np.sin(g.axes[2]))]
    X0 = bumps_cores()
    X0[-1] = X0[-1] / (tt.full_sum(X0) * g.delta)
    for b in range(2):
        ref, logc = pmf.update(Pn, g, pmf.likelihood(g, ocomps, z[b], R))
        X, tails, _ = T.update(X0, g, ocomps, z[b], R, EPS, 16)
        assert rel(tt.densify(f.export_cores(b)), ref) <= tt_tol(EPS, sum(tails))
        assert f.ranks()[b].tolist() == tt.ranks(X)
        assert abs(lc[b] - logc) < 1e-5
        assert abs(ll[b] - logc) < 1e-5
        mo, co = pmf.moments(ref, g)
        assert np.abs(m[b] - mo).max() < 1e-3 * g.delta_axis.min()
        np.testing.assert_allclose(c[b], co, atol=1e-5)


def test_update_dev_matches_host_update(G):
    import torch
    f1, g, P = bumps_filter(G, batch=3)
    f2, _, _ = bumps_filter(G, batch=3)
    axes = f1.grid_axes()
    comps = [((1,), torch.tensor(axes[1], dtype=torch.float32, device="cuda"))]
    z = np.array([[0.3], [-0.7], [0.3]])
    f1.update(comps, [[0.2]], z)
    f2.update_dev(comps, [[0.2]], torch.tensor(z, dtype=torch.float32, device="cuda"))
    m1 = f1.estimate()
    mean = torch.zeros(3, 3, dtype=torch.float64, device="cuda")
    cov = torch.zeros(3, 3, 3, dtype=torch.float64, device="cuda")
    lc = torch.zeros(3, dtype=torch.float64, device="cuda")
    ll = torch.zeros(3, dtype=torch.float64, device="cuda")
    f2.estimate_dev(mean, cov, lc, ll)
    torch.cuda.synchronize()
    np.testing.assert_allclose(mean.cpu().numpy(), m1[0], atol=1e-12)
    np.testing.assert_allclose(lc.cpu().numpy(), m1[2], atol=1e-12)
    # equal measurements give identical filters
    np.testing.assert_array_equal(f1.export_cores(0)[0], f1.export_cores(2)[0])


def test_invalid_arguments_leave_state(G):
    f, g, P = bumps_filter(G)
    before = tt.densify(f.export_cores(0))
    with pytest.raises(G.TTGBFError) as e:
        f.predict(np.eye(3), np.array([[1.0, 0.1, 0], [0.1, 1.0, 0], [0, 0, 1.0]]))
    assert e.value.code == -1
    with pytest.raises(G.TTGBFError) as e:
        f.predict(np.array([[0.0, 1.0, 0], [1.0, 0.0, 0], [0, 0, 1.0]]), np.eye(3))
    assert e.value.code == -6
    with pytest.raises(G.TTGBFError) as e:
        f.predict(np.full((3, 3), np.nan), np.eye(3))
    assert e.value.code == -2
    with pytest.raises(G.TTGBFError) as e:
        f.shear(0, 1, 10.0)       # 152 shifts: beyond max_shift_span^2 even in pieces
    assert e.value.code == -5
    with pytest.raises(G.TTGBFError) as e:
        f.shear(0, 1, 5.0, do_round=False)  # 77 shifts unrounded: beyond max_shift_span
    assert e.value.code == -5
    with pytest.raises(G.TTGBFError) as e:
        f.shear(1, 1, 0.1)
    assert e.value.code == -1
    np.testing.assert_array_equal(tt.densify(f.export_cores(0)), before)


def test_one_dimensional_and_tiny_grid(G):
    f = G.TTFilter([-3.0], [3.0], [2], [0.0], [1.0])
    f.predict([[0.9]], [[0.1]])
    g = pmf.Grid([-3.0], [3.0], [2])
    ref, _ = pmf.predict_rg(pmf.prior(g, [0.0], [[1.0]]), g, [[0.9]], [[0.1]])
    assert rel(tt.densify(f.export_cores(0)), ref) < 1e-6
    f = G.TTFilter([-3.0, -2.0], [3.0, 2.0], [5, 3], [0.1, 0.0], [1.0, 0.5], rank_cap=8)
    F = np.array([[0.9, 0.2], [0.0, 0.8]])
    f.predict(F, 0.1 * np.eye(2))
    g = pmf.Grid([-3.0, -2.0], [3.0, 2.0], [5, 3])
    P0 = pmf.prior(g, [0.1, 0.0], np.diag([1.0, 0.5]))
    ref, _ = pmf.predict_rg(P0, g, F, 0.1 * np.eye(2))
    X0 = [np.exp(-0.5 * (g.axes[m] - [0.1, 0.0][m]) ** 2 / [1.0, 0.5][m]).reshape(1, -1, 1)
          for m in range(2)]
    X, tails, _ = T.predict(X0, g, F, 0.1 * np.eye(2), 1e-6, 8)
    assert rel(tt.densify(f.export_cores(0)), ref) <= tt_tol(1e-6, sum(tails))


@pytest.mark.parametrize("terms", [17, 40])
def test_mass_and_moments_at_ranks_above_16(G, terms):
    """Ranks 17 and 40 on the inner links (more (alpha, beta) pairs per core
    than a moments pass takes at once): the normalised TT has unit mass by
    the oracle's sum, and the moments equal the oracle's of the densified TT."""
    n = [12, 10, 9]
    f = G.TTFilter(LO[:3], HI[:3], n, np.zeros(3), np.ones(3), rank_cap=40, eps=EPS,
                   max_shift_span=4)
    cores = [c.astype(np.float32) for c in synth.random_index_bumps_tt(n, terms, 7)]
    f.import_cores(0, cores)
    assert f.ranks()[0].tolist() == [1, terms, terms, 1]
    f.normalise()
    g = pmf.Grid(LO[:3], HI[:3], n)
    out = f.export_cores(0)
    assert abs(tt.full_sum([c.astype(np.float64) for c in out]) * g.delta - 1.0) < 1e-5
    m, c, lc, ll = f.estimate()
    P = tt.densify([x.astype(np.float64) for x in cores])
    mo, co = pmf.moments(P / (P.sum() * g.delta), g)
    np.testing.assert_allclose(m[0], mo, rtol=0, atol=1e-6)
    np.testing.assert_allclose(c[0], co, rtol=0, atol=1e-5)
