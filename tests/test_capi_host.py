"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every function that include/ttgbf.h declares, and validates
arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2501_07942_gb300 as G
from paper_2501_07942_gb300 import build as B

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ttgbf.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return G.load()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(ttgbf_\w+)\s*\(", text, flags=re.M)))


def test_header_functions_exported(lib):
    names = declared_functions()
    assert len(names) >= 19
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(G.EXPORTED) == names


def test_strerror(lib):
    assert G.strerror(0) == "ok"
    for code in range(-1, -8, -1):
        assert G.strerror(code) != "unknown error"
    assert G.strerror(-99) == "unknown error"


def test_workspace_bytes(lib):
    small = G.workspace_bytes([-8] * 4, [8] * 4, [32] * 4, batch=1)
    big = G.workspace_bytes([-8] * 4, [8] * 4, [128] * 4, batch=100)
    assert 0 < small < big
    assert big % 256 == 0 or big > 0
    # rank_cap * max_shift_span beyond the 160-column limit of one SVD problem
    assert G.workspace_bytes([-8] * 4, [8] * 4, [32] * 4, rank_cap=17) == 0
    assert G.workspace_bytes([-8] * 4, [8] * 4, [32] * 4, rank_cap=32, max_shift_span=5) > 0
    # float64 rounding: the TSQR stacks hold float64 slice factors (twice the words)
    fp64 = G.workspace_bytes([-8] * 4, [8] * 4, [128] * 4, batch=100, precision="fp64")
    assert fp64 > big
    # the cross's scratch: 2 s^2 N_max fiber floats, row norms, masks, index sets per filter
    cross = G.workspace_bytes([-8] * 4, [8] * 4, [128] * 4, batch=100, cross_rank=24)
    assert cross - big >= 100 * (2 * 24 * 24 * 128 + 2 * 5 * 24 * 24) * 4
    # invalid grids
    assert G.workspace_bytes([0.0], [0.0], [8]) == 0
    assert G.workspace_bytes([0.0], [1.0], [1]) == 0
    assert G.workspace_bytes([np.nan], [1.0], [8]) == 0


def _init(lib, lo, hi, n, mean, var, **kw):
    g, keep = G._grid(lo, hi, n)
    o = G.Opts(kw.get("batch", 1), kw.get("rank_cap", 16), kw.get("eps", 1e-6),
               kw.get("smax", 0), None, None, 0, kw.get("precision", 0), kw.get("conv", 0),
               0, 0, 0, kw.get("cross_rank", 0), kw.get("cross_sweeps", 0), kw.get("contraction", 0))
    m, v = G._f64(mean), G._f64(var)
    p = G.Prior(G._dptr(m), G._dptr(v))
    ctx = ctypes.c_void_p()
    rc = lib.ttgbf_init(ctypes.byref(ctx), ctypes.byref(g), ctypes.byref(p), ctypes.byref(o))
    return rc, ctx


def test_init_validates_before_device(lib):
    # every case below must be rejected on the host, before any CUDA call
    assert _init(lib, [0.0], [1.0], [8], [0.0], [1.0], batch=0)[0] == -1
    assert _init(lib, [0.0], [1.0], [8], [0.0], [1.0], rank_cap=0)[0] == -1
    assert _init(lib, [0.0], [1.0], [8], [0.0], [1.0], eps=float("nan"))[0] == -2
    assert _init(lib, [0.0], [1.0], [8], [0.0], [1.0], eps=-1.0)[0] == -1
    assert _init(lib, [0.0], [1.0], [8], [0.0], [1.0], rank_cap=40)[0] == -5
    assert _init(lib, [0.0], [1.0], [8], [np.inf], [1.0])[0] == -2
    assert _init(lib, [0.0], [1.0], [8], [0.0], [0.0])[0] == -1
    assert _init(lib, [1.0], [0.0], [8], [0.0], [1.0])[0] == -1
    assert _init(lib, [0.0] * 17, [1.0] * 17, [4] * 17, [0.0] * 17, [1.0] * 17)[0] == -1
    assert _init(lib, [0.0], [1.0], [8], [0.0], [1.0], precision=2)[0] == -1
    assert _init(lib, [0.0], [1.0], [8], [0.0], [1.0], precision=-1)[0] == -1
    assert _init(lib, [0.0], [1.0], [8], [0.0], [1.0], conv=3)[0] == -1
    assert _init(lib, [0.0], [1.0], [8], [0.0], [1.0], contraction=3)[0] == -1
    assert _init(lib, [0.0], [1.0], [8], [0.0], [1.0], contraction=-1)[0] == -1
    # the cross rank: at least the rank cap, at most 64 and the rank capacity
    assert _init(lib, [0.0], [1.0], [8], [0.0], [1.0], cross_rank=8)[0] == -1
    assert _init(lib, [0.0], [1.0], [8], [0.0], [1.0], cross_rank=65)[0] == -1
    assert _init(lib, [0.0], [1.0], [8], [0.0], [1.0], rank_cap=8, smax=2, cross_rank=24)[0] == -1
    assert _init(lib, [0.0], [1.0], [8], [0.0], [1.0], cross_rank=-1)[0] == -1
    assert _init(lib, [0.0], [1.0], [8], [0.0], [1.0], cross_rank=24, cross_sweeps=-1)[0] == -1


def test_null_context_calls(lib):
    assert lib.ttgbf_free(None) == 0
    assert lib.ttgbf_predict(None, None, None) == -1
    assert lib.ttgbf_round(None) == -1
    assert lib.ttgbf_normalise(None) == -1
    assert lib.ttgbf_grid_axes(None, None) == -1
    assert lib.ttgbf_densify(None, 0, None, 0) == -1


def test_filter_reports_capacity_before_device(lib):
    # the size query fails; the binding names the reason from ttgbf_init's
    # host-side validation (no workspace is allocated, nothing is launched)
    import types
    null_stream = types.SimpleNamespace(cuda_stream=0)
    with pytest.raises(G.TTGBFError) as ei:
        G.TTFilter([-40.0, -10.0], [40.0, 10.0], [256, 256], [0.0, 0.0], [4.0, 1.0],
                   rank_cap=32, eps=1e-5, stream=null_stream)
    assert ei.value.code == -5
    with pytest.raises(G.TTGBFError) as ei:
        G.TTFilter([0.0], [0.0], [8], [0.0], [1.0], stream=null_stream)
    assert ei.value.code == -1


def test_injected_alloc_failure(lib, monkeypatch):
    # TTGBF_FAULT=alloc: init validates, then reports the allocation failure
    monkeypatch.setenv("TTGBF_FAULT", "alloc")
    rc, ctx = _init(lib, [0.0], [1.0], [8], [0.0], [1.0])
    assert rc == -3 and not ctx.value
    # invalid arguments are still reported as such
    assert _init(lib, [0.0], [1.0], [8], [0.0], [1.0], batch=0)[0] == -1


@pytest.mark.parametrize("d,seed", [(2, 0), (4, 1), (6, 2)])
def test_ldu_adjoint_matches_central_differences(lib, d, seed):
    """ttgbf_ldu_adjoint (host code of the reverse pass): the gradient of
    f(F) = <GL, L> + <GD, D> + <GU, U> over F = L D U equals central
    differences of f through the oracle's Doolittle factorisation."""
    from oracle import pmf
    rng = np.random.default_rng(seed)
    F = np.eye(d) * 1.5 + 0.3 * rng.standard_normal((d, d))
    GL = np.tril(rng.standard_normal((d, d)), -1)
    GU = np.triu(rng.standard_normal((d, d)), 1)
    GD = rng.standard_normal(d)

    def f(X):
        L, D, U = pmf.ldu(X)
        return float((GL * L).sum() + (GD * D).sum() + (GU * U).sum())

    h = 1e-6
    fd = np.zeros((d, d))
    for i in range(d):
        for j in range(d):
            E = np.zeros((d, d))
            E[i, j] = h
            fd[i, j] = (f(F + E) - f(F - E)) / (2 * h)
    got = G.ldu_adjoint(F, GL, GD, GU)
    assert np.abs(got - fd).max() <= 1e-6 * max(1.0, np.abs(fd).max()), (got, fd)


def test_ldu_adjoint_rejects_singular_leading_minor(lib):
    F = np.array([[0.0, 1.0], [1.0, 0.0]])
    with pytest.raises(G.TTGBFError) as e:
        G.ldu_adjoint(F, np.zeros((2, 2)), np.zeros(2), np.zeros((2, 2)))
    assert e.value.code == -6


def test_design_grid_matches_oracle(lib):
    """ttgbf_design_grid (host code, Alg. 4 steps 1-4) equals the oracle's
    design rule on random models and batches."""
    from oracle import grid_design as GD
    rng = np.random.default_rng(11)
    for d, B in [(2, 1), (3, 4), (4, 2)]:
        F = np.eye(d) * 0.9 + 0.2 * rng.standard_normal((d, d))
        Q = np.diag(rng.uniform(0.01, 0.1, d))
        means = rng.standard_normal((B, d))
        covs = np.array([(lambda A: A @ A.T / d + 0.05 * np.eye(d))(rng.standard_normal((d, d)))
                         for _ in range(B)])
        lo, hi = G.design_grid(F, Q, means, covs, kappa=4.5)
        elo, ehi = GD.design_grid(F, Q, means, covs, 4.5)
        assert np.allclose(lo, elo, rtol=0, atol=1e-12) and np.allclose(hi, ehi, rtol=0, atol=1e-12)
    with pytest.raises(G.TTGBFError) as e:
        G.design_grid(np.zeros((2, 2)), np.eye(2), np.zeros((1, 2)), np.eye(2)[None], 3.0)
    assert e.value.code == -6
