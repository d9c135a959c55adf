"""Grid re-design on the GPU (Alg. 4: ttgbf_design_grid, ttgbf_regrid) against
the oracle (oracle/grid_design.py).

* ttgbf_regrid: the TT cores of a stepped batch, moved onto a shifted and
  rescaled grid, equal the oracle's interpolation of the same densified
  cores, to float32 rounding (relative L2 1e-5).
* A filter that re-designs its grid after every update, on models small
  enough that no rank cap binds (the general models of the gradient tests:
  lower couplings, one-mode and two-mode components), equals the dense oracle
  filter re-gridded onto the same grids (the grids the GPU run chose, given
  to the oracle), to float32 rounding and eps-level truncation (relative L2
  1e-4 per step); means within 1e-3 grid spacings."""
import numpy as np
import pytest

import synth
from oracle import grid_design as GD
from oracle import pmf, tt

from gpu_util import device_tables, lib_module, oracle_grid, rel

pytestmark = pytest.mark.gpu

REGRID_TOL = 1e-5
STEP_TOL = 1e-4


@pytest.fixture(scope="module")
def G():
    return lib_module()


def test_regrid_matches_oracle_interpolation(G):
    import torch
    model = synth.config2(n=24)
    f = G.TTFilter(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), batch=2, rank_cap=16,
                   eps=model.eps, max_shift_span=10)
    comps = device_tables(model, f.grid_axes())
    z = np.stack([synth.simulate(model, b, steps=1)[1][0] for b in range(2)])
    f.predict(model.F, model.Q)
    f.update(comps, model.R, z)
    g_old = oracle_grid(model)
    before = [tt.densify(f.export_cores(b)) for b in range(2)]
    lo = np.array(model.lo) + np.array([0.7, -0.4, 0.3, -0.9])
    hi = np.array(model.hi) * np.array([0.8, 1.1, 0.9, 1.05])
    f.regrid(lo, hi)
    g_new = pmf.Grid(lo, hi, model.n)
    axes = f.grid_axes()
    for k in range(model.d):
        assert np.allclose(axes[k], g_new.axes[k], rtol=0, atol=1e-12)
    for b in range(2):
        got = tt.densify(f.export_cores(b))
        ref = GD.regrid(before[b], g_old, g_new)
        e = rel(got, ref)
        print(f"filter {b}: rel L2 {e:.2e}")
        assert e <= REGRID_TOL, e
    torch.cuda.synchronize()


def _general_model(d):
    if d == 2:
        g = pmf.Grid([-6.0, -5.0], [6.0, 5.0], [20, 18])
        F = np.array([[0.93, 0.12], [-0.07, 0.88]])
        Q = np.diag([0.09, 0.12])
        comps = [((0,), synth.workloads.h_identity), ((1,), synth.workloads.h_sin)]
        R = np.diag([0.2, 0.1])
        z = np.array([[0.4, 0.2], [0.1, -0.3], [-0.2, 0.1], [0.3, 0.0]])
    else:
        g = pmf.Grid([-4.0, -4.0, -3.0], [4.0, 4.0, 3.0], [12, 10, 9])
        F = np.array([[0.95, 0.05, -0.04], [0.03, 0.9, 0.06], [0.0, -0.05, 0.92]])
        Q = np.diag([0.1, 0.15, 0.08])
        comps = [((0, 1), synth.workloads.h_range), ((2,), synth.workloads.h_identity)]
        R = np.diag([0.3, 0.2])
        z = np.array([[1.1, 0.2], [0.9, -0.1], [1.0, 0.1]])
    m = synth.Model(name=f"design-d{d}", lo=np.array(g.lo), hi=np.array(g.hi), n=np.array(g.shape),
                    m0=np.zeros(d), P0=np.eye(d), F=F, Q=Q, R=R, comps=comps, eps=1e-6, rank_cap=32)
    return m, g, z


@pytest.mark.parametrize("d", [2, 3])
def test_filter_with_grid_redesign_matches_oracle(G, d):
    model, g, zs = _general_model(d)
    f = G.TTFilter(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), batch=1, rank_cap=32,
                   eps=model.eps, max_shift_span=5)
    P = pmf.prior(g, model.m0, model.P0)
    for k, z in enumerate(zs):
        comps = device_tables(model, f.grid_axes())
        f.predict(model.F, model.Q)
        f.update(comps, model.R, z[None, :])
        mean, cov, lc, ll = f.estimate()
        P, _ = pmf.predict_rg(P, g, model.F, model.Q)
        P, logc = pmf.update(P, g, pmf.likelihood(g, model.tables(g.axes), z, model.R))
        e = rel(tt.densify(f.export_cores(0)), P)
        mo, _ = pmf.moments(P, g)
        print(f"d={d} step {k}: rel L2 {e:.2e}, |log c diff| {abs(lc[0] - logc):.1e}, grid lo {g.lo}")
        assert e <= STEP_TOL, (k, e)
        assert (np.abs(mean[0] - mo) <= 1e-3 * g.delta_axis).all(), (k, mean[0], mo)
        # re-design the grid from the GPU's posterior moments; the oracle follows
        lo, hi = G.design_grid(model.F, model.Q, mean, cov, kappa=4.0)
        elo, ehi = GD.design_grid(model.F, model.Q, mean, cov, 4.0)
        assert np.allclose(lo, elo, atol=1e-12) and np.allclose(hi, ehi, atol=1e-12)
        f.regrid(lo, hi)
        g_new = pmf.Grid(lo, hi, model.n)
        P = GD.regrid(P, g, g_new)
        g = g_new
