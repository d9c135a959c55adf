"""The core contractions on the tensor cores (ttgbf_opts.contraction: tcgen05
TF32 MMAs, float32 accumulation in tensor memory) against the float64 oracle.

TF32X3 splits each operand into a TF32 part and a TF32-rounded remainder;
its products are float32-level, so it is held to the bounds of the float32
path.  Plain TF32 rounds every operand to 10 mantissa bits (round to nearest:
relative error at most 2^-11 per operand, so at most about 2^-10 per product
term).  A filter step chains at most 3d + 1 contraction stages (the predictive
step's d per-mode operators, the 2d - 1 stages of a rounding sweep, the 2-site
merge of the update), and a stage's relative error is at most that of its
terms, so a step adds at most (3d + 1) 2^-10 relative error to the float32
path's bound.  The convolution hook runs one stage per mode."""
import numpy as np
import pytest

import synth
from oracle import pmf, tt
from oracle import ttfilter as T

from gpu_util import (device_tables, lib_module, mean_tol, oracle_grid, oracle_tt_prior, rel,
                      tt_tol)

pytestmark = pytest.mark.gpu

TF32_TERM = 2.0 ** -10  # relative error of a product of two TF32-rounded operands


@pytest.fixture(scope="module")
def G():
    return lib_module()


def _bumps(G, contraction, n=(40, 36, 44), terms=3, seed=0):
    lo, hi = [-5.0, -4.0, -3.0], [5.0, 4.0, 3.0]
    f = G.TTFilter(lo, hi, list(n), np.zeros(3), np.ones(3), rank_cap=16, eps=1e-6, conv="dense",
                   contraction=contraction)
    cores = [c.astype(np.float32) for c in synth.random_index_bumps_tt(list(n), terms, seed)]
    f.import_cores(0, cores)
    g = pmf.Grid(lo, hi, list(n))
    return f, g, tt.densify([c.astype(np.float64) for c in cores])


@pytest.mark.parametrize("contraction", ["fp32", "tf32x3", "tf32"])
def test_convolution_on_tensor_cores(G, contraction):
    """The dense Toeplitz kernel applied to every core's grid index (one
    grouped product per mode: N x N by N x r fibres, N not a multiple of the
    128 x 32 tile or of the 16-wide k chunks).  TF32 must show its rounding
    (an error above the float32 path's): that is the evidence that the
    tensor-core path ran."""
    f, g, P = _bumps(G, contraction)
    q = [0.05, 0.1, 0.02]
    f.convolve(q)
    ref = P
    for k in range(3):
        ref = pmf.convolve_axis(ref, g, k, q[k])
    e = rel(tt.densify(f.export_cores(0)), ref)
    print(f"{contraction}: convolution rel err {e:.3e}")
    if contraction == "tf32":
        assert 1e-5 < e <= 3 * TF32_TERM, e
    else:
        assert e < 1e-6, e


@pytest.mark.parametrize("contraction", ["tf32x3", "tf32"])
def test_filter_steps_on_tensor_cores(G, contraction):
    """Config 2 at 24^4 (ranks 16 x spans up to 9: products of 384 x 144 by
    144 x 16 and their transposes), three filters, four steps, against the
    dense float64 oracle: TF32X3 at the float32 path's bound (summed
    10 (eps + tau) + 1e-5 with tau from the oracle TT filter, means within
    1e-3 grid spacings + 2 tau sigma), TF32 with (3d + 1) 2^-10 per step
    added to the density bound and the same added relative error times sigma
    to the means'."""
    model = synth.config2(n=24)
    mcs = [0, 1, 2]
    steps = 4
    f = G.TTFilter(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), batch=len(mcs),
                   rank_cap=model.rank_cap, eps=model.eps, contraction=contraction)
    comps = device_tables(model, f.grid_axes())
    g = oracle_grid(model)
    oc = model.tables(g.axes)
    zs = [synth.simulate(model, mc, steps=steps)[1] for mc in mcs]
    Ps = [pmf.prior(g, model.m0, model.P0) for _ in mcs]
    X = [oracle_tt_prior(model) for _ in mcs]
    bound = [0.0] * len(mcs)
    tacc = [0.0] * len(mcs)
    extra = (3 * model.d + 1) * TF32_TERM if contraction == "tf32" else 0.0
    for k in range(steps):
        f.predict(model.F, model.Q)
        f.update(comps, model.R, np.stack([z[k] for z in zs]))
        m, c, lc, ll = f.estimate()
        st = f.stats()
        for i in range(len(mcs)):
            Ps[i], _ = pmf.predict_rg(Ps[i], g, model.F, model.Q)
            Ps[i], logc = pmf.update(Ps[i], g, pmf.likelihood(g, oc, zs[i][k], model.R))
            X[i], info = T.step(X[i], g, model.F, model.Q, oc, zs[i][k], model.R, model.eps,
                                model.rank_cap)
            bound[i] += tt_tol(model.eps, info["tail_sum"]) + extra
            tacc[i] += info["tail_sum"]
            e = rel(f.densify(i), Ps[i])
            mo, co = pmf.moments(Ps[i], g)
            mt = mean_tol(g.delta_axis, co, tacc[i] + (k + 1) * extra)
            merr = float((np.abs(m[i] - mo) / mt).max())
            print(f"{contraction} step {k} filter {i}: rel err {e:.3e} (bound {bound[i]:.3e}), "
                  f"mean err / tol {merr:.2f}, |log c diff| {abs(lc[i] - logc):.2e}, "
                  f"max rank {st[i]['max_rank']}")
            assert e <= bound[i], (k, i, e, bound[i])
            assert merr <= 1.0, (k, i, merr)
            assert np.isfinite(c[i]).all()


def test_tensor_core_products_in_a_split_batch(G, monkeypatch):
    """A batch split into concurrent parts (their tensor-core products on
    several streams at once) gives each filter what the unsplit batch gives
    it on the same contraction path (TF32X3)."""
    model = synth.config2(n=24)
    B = 6
    zs = np.stack([synth.simulate(model, mc, steps=2)[1] for mc in range(B)], axis=1)
    outs = []
    for parts in ("1", "3"):
        monkeypatch.setenv("TTGBF_PARTS", parts)
        f = G.TTFilter(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), batch=B,
                       rank_cap=model.rank_cap, eps=model.eps, contraction="tf32x3")
        comps = device_tables(model, f.grid_axes())
        for k in range(2):
            f.predict(model.F, model.Q)
            f.update(comps, model.R, zs[k])
        m, c, lc, ll = f.estimate()
        outs.append((f.ranks(), [f.densify(b) for b in range(B)], m))
        f.free()
    (r1, d1, m1), (r3, d3, m3) = outs
    np.testing.assert_array_equal(r1, r3)
    for b in range(B):
        assert rel(d3[b], d1[b]) < 1e-4
    np.testing.assert_allclose(m3, m1, rtol=0, atol=1e-5)
