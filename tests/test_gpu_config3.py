"""GPU parity on the higher-dimensional workload: d = 6 and d = 8 constant-
velocity blocks x_{2i} += 0.1 x_{2i+1}, diagonal Q, one-mode measurements
z_i = x_{2i}^2 / 20 + v_i, rank cap 32, eps 1e-5.

* d = 6 at N = 16 and d = 8 at N = 8: the whole density against the dense
  FP64 oracle (a 256^d grid is out of any dense filter's reach).
* d = 8 at N = 128 and d = 6, 8 at the full N = 256: the model is block diagonal (F, Q, prior and likelihood
  all factor over the pairs (x_{2i}, x_{2i+1})) and so is the re-gridded
  transition, whose shears act inside one pair each.  The exact density is
  then the tensor product of four 2-D oracle densities, each computed densely
  on its 128 x 128 grid; the TT density is compared with that product through
  TT inner products, so no 128^8 tensor is formed.

Tolerances as for the other workloads: per step 10 (eps + tau) + 1e-5 in
relative Frobenius norm, summed over the steps, tau the discarded tails of
the float64 TT filter of oracle/ttfilter.py on the same measurements (its
ranks must equal the GPU's); means within 1e-3 grid spacings (plus 2 tau
sigma where the rank cap binds); covariances within the matching 1e-3
(D_i sigma_j + D_j sigma_i); log c within 1e-3.  The shear span of this workload is at most 5 up
to N = 128 (|0.1 xi_vel / Delta_pos| <= 1.59), so the rank expansion stays at
32 x 5 = 160 columns; at N = 256 it is 9 and the shears run in pieces."""
import numpy as np
import pytest

import synth
from oracle import pmf, tt
from oracle import ttfilter as T

from gpu_util import (cov_tol, device_tables, lib_module, make_filter, mean_tol, oracle_grid,
                      oracle_tt_prior, rel, tt_tol)

pytestmark = pytest.mark.gpu

SPAN = 5


@pytest.fixture(scope="module")
def G():
    return lib_module()


def block_model(model: synth.Model, i: int) -> synth.Model:
    """The 2-D model of the pair (x_{2i}, x_{2i+1}) of a config-3 model."""
    s = slice(2 * i, 2 * i + 2)
    return synth.Model(name=f"{model.name}-pair{i}", lo=model.lo[s], hi=model.hi[s],
                       n=model.n[s], m0=model.m0[s], P0=model.P0[s, s], F=model.F[s, s],
                       Q=model.Q[s, s], R=model.R[i:i + 1, i:i + 1],
                       comps=[((0,), synth.workloads.h_square20)], eps=model.eps,
                       rank_cap=model.rank_cap)


@pytest.mark.parametrize("d,n,steps", [(6, 16, 4), (8, 8, 3)])
def test_config3_small_grid_vs_dense_oracle(G, d, n, steps):
    model = synth.config3(d=d, n=n)
    mcs = [0, 1]
    f = make_filter(G, model, batch=len(mcs), smax=SPAN)
    comps = device_tables(model, f.grid_axes())
    g = oracle_grid(model)
    oc = model.tables(g.axes)
    zs = [synth.simulate(model, mc, steps=steps)[1] for mc in mcs]
    Ps = [pmf.prior(g, model.m0, model.P0) for _ in mcs]
    X = [oracle_tt_prior(model) for _ in mcs]
    bound = [0.0] * len(mcs)
    tacc = [0.0] * len(mcs)
    for k in range(steps):
        f.predict(model.F, model.Q)
        f.update(comps, model.R, np.stack([z[k] for z in zs]))
        st = f.stats()
        m, c, lc, ll = f.estimate()
        for i in range(len(mcs)):
            Ps[i], _ = pmf.predict_rg(Ps[i], g, model.F, model.Q)
            Ps[i], logc = pmf.update(Ps[i], g, pmf.likelihood(g, oc, zs[i][k], model.R))
            mo, co = pmf.moments(Ps[i], g)
            X[i], info = T.step(X[i], g, model.F, model.Q, oc, zs[i][k], model.R, model.eps,
                                model.rank_cap, SPAN)
            assert f.ranks()[i].tolist() == tt.ranks(X[i]), (k, i)
            bound[i] += tt_tol(model.eps, info["tail_sum"])
            tacc[i] += info["tail_sum"]
            e = rel(tt.densify(f.export_cores(i)), Ps[i])
            assert e <= bound[i], (k, i, e, bound[i])
            assert (np.abs(m[i] - mo) <= mean_tol(g.delta_axis, co, tacc[i])).all(), (k, i)
            assert (np.abs(c[i] - co) <= cov_tol(g.delta_axis, co)).all(), (k, i)
            assert abs(lc[i] - logc) < 1e-3, (k, i)
            assert st[i]["max_rank"] <= model.rank_cap


@pytest.mark.parametrize("d,n,steps,smax", [(8, 128, 4, 5), (6, 256, 3, 5), (8, 256, 3, 5),
                                             (6, 256, 2, 3), (6, 256, 25, 5)])
def test_config3_vs_blockwise_oracle(G, d, n, steps, smax):
    """At N = 256 every shear spans 9 shifts: with a span of 5 (3) it is
    applied as 2 (3) rounded pieces whose TT sum is rounded again.  The
    25-step case is the long horizon: the pieces' extra truncations compound
    over it, and the summed per-step bound still holds; its ranks may part from
    the oracle TT filter's at a decision on the threshold (R23), so there it
    checks them within one of the oracle's, and its covariances against the
    oracle TT filter's (the same truncations) at the flat bound."""
    model = synth.config3(d=d, n=n)
    mcs = [0, 1]
    f = make_filter(G, model, batch=len(mcs), smax=smax)
    comps = device_tables(model, f.grid_axes())
    zs = [synth.simulate(model, mc, steps=steps)[1] for mc in mcs]
    pairs = [block_model(model, i) for i in range(model.d // 2)]
    grids = [oracle_grid(bm) for bm in pairs]
    tabs = [bm.tables(gb.axes) for bm, gb in zip(pairs, grids)]
    P = [[pmf.prior(gb, bm.m0, bm.P0) for bm, gb in zip(pairs, grids)] for _ in mcs]
    g = oracle_grid(model)
    oc = model.tables(g.axes)
    X = [oracle_tt_prior(model) for _ in mcs]
    bound = [0.0] * len(mcs)
    tacc = [0.0] * len(mcs)
    for k in range(steps):
        f.predict(model.F, model.Q)
        f.update(comps, model.R, np.stack([z[k] for z in zs]))
        st = f.stats()
        m, c, lc, ll = f.estimate()
        for b in range(len(mcs)):
            logc = 0.0
            mean = np.zeros(model.d)
            cov = np.zeros((model.d, model.d))
            exact = []
            for i, (bm, gb, tb) in enumerate(zip(pairs, grids, tabs)):
                Pi, _ = pmf.predict_rg(P[b][i], gb, bm.F, bm.Q)
                Pi, lci = pmf.update(Pi, gb, pmf.likelihood(gb, tb, zs[b][k][i:i + 1], bm.R))
                P[b][i] = Pi
                logc += lci
                mo, co = pmf.moments(Pi, gb)
                mean[2 * i:2 * i + 2] = mo
                cov[2 * i:2 * i + 2, 2 * i:2 * i + 2] = co
                # exact 2-core TT of the pair's density (1e-12 truncation)
                exact += tt.from_dense(Pi, eps=1e-12)
            cores = [np.asarray(x, dtype=np.float64) for x in f.export_cores(b)]
            nn = tt.inner(exact, exact)
            diff2 = tt.inner(cores, cores) - 2.0 * tt.inner(cores, exact) + nn
            e = float(np.sqrt(max(diff2, 0.0) / nn))
            X[b], info = T.step(X[b], g, model.F, model.Q, oc, zs[b][k], model.R, model.eps,
                                model.rank_cap, smax)
            if steps <= 4:
                assert f.ranks()[b].tolist() == tt.ranks(X[b]), (k, b)
            else:
                assert np.abs(np.array(f.ranks()[b]) - np.array(tt.ranks(X[b]))).max() <= 1, (k, b)
            bound[b] += tt_tol(model.eps, info["tail_sum"])
            tacc[b] += info["tail_sum"]
            assert e <= bound[b], (k, b, e, bound[b])
            D = np.concatenate([gb.delta_axis for gb in grids])
            assert (np.abs(m[b] - mean) <= mean_tol(D, cov, tacc[b])).all(), (k, b, m[b], mean)
            if steps <= 4:
                assert (np.abs(c[b] - cov) <= cov_tol(D, cov)).all(), (k, b, c[b] - cov)
            else:
                # over the long horizon the truncations move the covariances by more than
                # 2 tau sigma_i sigma_j (the oracle TT filter itself, in float64, misses that
                # against the dense densities at step 5): held to the oracle TT filter's
                # covariances, which make the same truncations, at the flat bound
                _, cov_tt = T.moments(X[b], g)
                assert (np.abs(c[b] - cov_tt) <= cov_tol(D, cov)).all(), (k, b, c[b] - cov_tt)
            assert abs(lc[b] - logc) < 1e-3, (k, b, lc[b], logc)
            r = f.ranks()[b]
            assert r.max() <= model.rank_cap
            # the pairs are independent: rank 1 between them
            assert all(r[2 * i] == 1 for i in range(1, model.d // 2)), r


def test_config3_capacity_limits(G):
    """rank_cap x span above 160 columns is refused at init; a shear wider
    than span^2 shifts (more pieces than the sum has rank room for) at
    predict, before anything is enqueued."""
    model = synth.config3(d=6, n=256)
    with pytest.raises(G.TTGBFError) as ei:
        make_filter(G, model, batch=1)  # default span 10: 32 x 10 > 160
    assert ei.value.code == -5
    f = make_filter(G, model, batch=1, smax=2)  # 9 shifts > 2^2
    r0 = f.ranks().copy()
    with pytest.raises(G.TTGBFError) as ei:
        f.predict(model.F, model.Q)
    assert ei.value.code == -5
    np.testing.assert_array_equal(f.ranks(), r0)
