"""GPU parity of the plain full-grid point-mass filter (ttgbf_fg_*) against
the dense FP64 oracle: float64 mode to 1e-12 relative L1 of the density,
float32 mode to 1e-5 relative L1 (the bound the full-grid filter is held to),
on config 1 (textbook direct sum and re-gridded transition) and on config 2
at a reduced grid."""
import numpy as np
import pytest

import synth
from oracle import pmf

from gpu_util import bearing_cut_model, lib_module

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    return lib_module()


def rel_l1(a, b):
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def tables(model, axes, dtype):
    import torch
    return [(m, torch.tensor(np.asarray(t), dtype=dtype, device="cuda"), *p) for m, t, *p in model.tables(axes)]


@pytest.mark.parametrize("transition", ["textbook", "rg"])
def test_config1_float64(G, transition):
    import torch
    model = synth.config1()
    x, z = synth.simulate(model, 2, steps=6)
    f = G.FullGridFilter(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), precision=64)
    g = pmf.Grid(model.lo, model.hi, model.n)
    comps = tables(model, g.axes, torch.float64)
    oc = model.tables(g.axes)
    P = pmf.prior(g, model.m0, model.P0)
    assert rel_l1(f.density(), P) < 1e-13
    ll = 0.0
    for k in range(6):
        if transition == "textbook":
            f.predict_direct(model.F, model.Q)
            P, _ = pmf.predict_textbook(P, g, model.F, model.Q)
        else:
            f.predict(model.F, model.Q)
            P, _ = pmf.predict_rg(P, g, model.F, model.Q)
        assert rel_l1(f.density(), P) < 1e-12
        f.update(comps, model.R, z[k])
        P, logc = pmf.update(P, g, pmf.likelihood(g, oc, z[k], model.R))
        ll += logc
        assert rel_l1(f.density(), P) < 1e-12
        m, c, lc, lls = f.estimate()
        mo, co = pmf.moments(P, g)
        np.testing.assert_allclose(m, mo, atol=1e-11)
        np.testing.assert_allclose(c, co, atol=1e-11)
        assert abs(lc - logc) < 1e-10 and abs(lls - ll) < 1e-9


def test_config2_float32_reduced_grid(G):
    import torch
    model = synth.config2(n=24)
    x, z = synth.simulate(model, 4, steps=4)
    f = G.FullGridFilter(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), precision=32)
    g = pmf.Grid(model.lo, model.hi, model.n)
    comps = tables(model, g.axes, torch.float32)
    oc = model.tables(g.axes)
    P = pmf.prior(g, model.m0, model.P0)
    for k in range(4):
        f.predict(model.F, model.Q)
        f.update(comps, model.R, z[k])
        P, _ = pmf.predict_rg(P, g, model.F, model.Q)
        P, logc = pmf.update(P, g, pmf.likelihood(g, oc, z[k], model.R))
        assert rel_l1(f.density(), P) < 1e-5
        m, c, lc, _ = f.estimate()
        mo, co = pmf.moments(P, g)
        np.testing.assert_allclose(m, mo, atol=1e-5)
        assert abs(lc - logc) < 1e-4


def test_general_F_and_two_mode_any_order(G):
    # non-triangular F (L shears after the scalings) and a two-mode component
    # on modes (2, 0) in float64
    import torch
    lo, hi, n = [-4.0, -3.0, -3.5], [4.0, 3.0, 3.5], [20, 16, 24]
    F = np.array([[0.95, 0.04, 0.0], [-0.05, 0.97, 0.02], [0.03, 0.0, 0.92]])
    Q = np.diag([0.05, 0.08, 0.03])
    f = G.FullGridFilter(lo, hi, n, [0.2, -0.1, 0.0], [1.0, 0.8, 0.6], precision=64)
    g = pmf.Grid(lo, hi, n)
    P = pmf.prior(g, [0.2, -0.1, 0.0], np.diag([1.0, 0.8, 0.6]))
    f.predict(F, Q)
    P, _ = pmf.predict_rg(P, g, F, Q)
    assert rel_l1(f.density(), P) < 1e-12
    tab = np.sqrt(g.axes[2][:, None] ** 2 + 0.5 * g.axes[0][None, :] ** 2)
    f.update([((2, 0), torch.tensor(tab, dtype=torch.float64, device="cuda"))], [[0.05]], [1.2])
    P, _ = pmf.update(P, g, pmf.likelihood(g, [((2, 0), tab)], [1.2], [[0.05]]))
    assert rel_l1(f.density(), P) < 1e-12


def test_config2_float32_at_64(G):
    """The benchmark's model on a 64^4 grid in float32 (one fused pass per
    axis, likelihood and moments in one pass) against the oracle."""
    import torch
    model = synth.config2(n=64)
    x, z = synth.simulate(model, 6, steps=2)
    f = G.FullGridFilter(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), precision=32)
    g = pmf.Grid(model.lo, model.hi, model.n)
    comps = tables(model, g.axes, torch.float32)
    oc = model.tables(g.axes)
    P = pmf.prior(g, model.m0, model.P0)
    for k in range(2):
        f.predict(model.F, model.Q)
        f.update(comps, model.R, z[k])
        P, _ = pmf.predict_rg(P, g, model.F, model.Q)
        P, logc = pmf.update(P, g, pmf.likelihood(g, oc, z[k], model.R))
        m, c, lc, _ = f.estimate()
        mo, co = pmf.moments(P, g)
        np.testing.assert_allclose(m, mo, atol=1e-5)
        np.testing.assert_allclose(c, co, atol=1e-5)
        assert abs(lc - logc) < 1e-4
    assert rel_l1(f.density(), P) < 1e-5


def test_pending_normalisations_in_any_call_order(G):
    """predict twice in a row, estimate after a predict, estimate after an
    update, density in between: every path that applies or carries the
    deferred normalisations gives the oracle's densities and moments."""
    import torch
    model = synth.config2(n=12)
    x, z = synth.simulate(model, 1, steps=2)
    f = G.FullGridFilter(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), precision=64)
    g = pmf.Grid(model.lo, model.hi, model.n)
    comps = tables(model, g.axes, torch.float64)
    oc = model.tables(g.axes)
    P = pmf.prior(g, model.m0, model.P0)
    for _ in range(2):
        f.predict(model.F, model.Q)
        P, _ = pmf.predict_rg(P, g, model.F, model.Q)
    m, c, _, _ = f.estimate()
    mo, co = pmf.moments(P, g)
    np.testing.assert_allclose(m, mo, atol=1e-11)
    f.update(comps, model.R, z[0])
    P, logc = pmf.update(P, g, pmf.likelihood(g, oc, z[0], model.R))
    m, c, lc, _ = f.estimate()
    mo, co = pmf.moments(P, g)
    np.testing.assert_allclose(m, mo, atol=1e-11)
    np.testing.assert_allclose(c, co, atol=1e-11)
    assert abs(lc - logc) < 1e-10
    f.predict(model.F, model.Q)
    P, _ = pmf.predict_rg(P, g, model.F, model.Q)
    f.update(comps, model.R, z[1])
    P, _ = pmf.update(P, g, pmf.likelihood(g, oc, z[1], model.R))
    assert rel_l1(f.density(), P) < 1e-12


def test_bearing_across_the_cut_float64(G):
    """Range and a bearing whose residual wraps inside the grid (period 360):
    float64 full-grid filter against the dense oracle to 1e-12."""
    import torch
    model, zs = bearing_cut_model((40, 36))
    f = G.FullGridFilter(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), precision=64)
    g = pmf.Grid(model.lo, model.hi, model.n)
    comps = tables(model, g.axes, torch.float64)
    oc = model.tables(g.axes)
    P = pmf.prior(g, model.m0, model.P0)
    for z in zs:
        f.predict(model.F, model.Q)
        P, _ = pmf.predict_rg(P, g, model.F, model.Q)
        f.update(comps, model.R, z)
        P, logc = pmf.update(P, g, pmf.likelihood(g, oc, z, model.R))
        assert rel_l1(f.density(), P) < 1e-12
        assert abs(f.estimate()[2] - logc) < 1e-10


def test_three_mode_and_other_pairs_float64(G):
    """Components on three consecutive modes, on a non-adjacent pair in
    decreasing order and on one mode: float64 full-grid filter against the
    dense oracle to 1e-12."""
    import torch
    g = pmf.Grid([-3.0, -3.0, -2.5, -2.0], [3.0, 3.0, 2.5, 2.0], [16, 12, 12, 8])  # multiples of 4
    a = g.axes
    r3 = np.sqrt(a[1][:, None, None] ** 2 + a[2][None, :, None] ** 2 + a[3][None, None, :] ** 2)
    t31 = a[3][:, None] + 0.5 * np.sin(a[1][None, :])
    oc = [((1, 2, 3), r3), ((3, 1), t31), ((0,), a[0])]
    comps = [(m, torch.tensor(t, dtype=torch.float64, device="cuda")) for m, t in oc]
    F = 0.95 * np.eye(4) + 0.05 * np.triu(np.ones((4, 4)), 1)
    Q = 0.05 * np.eye(4)
    R = np.diag([0.1, 0.2, 0.3])
    m0, P0 = np.array([0.5, -0.3, 0.2, 0.1]), np.eye(4)
    f = G.FullGridFilter(g.lo, g.hi, g.shape, m0, np.diag(P0), precision=64)
    P = pmf.prior(g, m0, P0)
    for z in (np.array([1.2, 0.4, 0.3]), np.array([0.9, -0.2, 0.6])):
        f.predict(F, Q)
        P, _ = pmf.predict_rg(P, g, F, Q)
        f.update(comps, R, z)
        P, logc = pmf.update(P, g, pmf.likelihood(g, oc, z, R))
        assert rel_l1(f.density(), P) < 1e-12
        assert abs(f.estimate()[2] - logc) < 1e-10
