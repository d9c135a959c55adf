"""The predictive step with the textbook transition (ttgbf_predict_exact: mode
factors of the transition matrix for an upper bidiagonal F, coupled factors
on 2-site blocks by the cross of csrc/cross.cu) against the oracle.

* One step from a shared input (the oracle TT filter's state loaded into the
  GPU filter): constant-velocity pairs (config 3's model form, d = 4) and a
  chain with non-unit diagonal (d = 3), against the untruncated oracle step
  (oracle/ttfilter.predict_exact, itself equal to the dense textbook
  transition, tests/test_oracle_exact_t.py) within 10 (eps + tau) + 1e-5, tau
  the tails of the oracle's truncated step; the predictive mass within 1e-5.
* A filter of predict_exact + update over several steps against the dense
  oracle filter with the textbook transition (pmf.run_filter), per-step
  bounds summed; means within the cap-aware tolerance.
* Config 3's model at its full size (d = 6, N = 256) against the tensor
  product of its pairs' exact 2-D densities.
* Other couplings, a non-diagonal Q and cross_rank 0 are TTGBF_EINVAL."""
import numpy as np
import pytest

import synth
from oracle import pmf, tt
from oracle import ttfilter as T

from gpu_util import device_tables, lib_module, mean_tol, rel, tt_tol

pytestmark = pytest.mark.gpu

S = 24


@pytest.fixture(scope="module")
def G():
    return lib_module()


def _state(g, seed):
    X = synth.random_index_bumps_tt(g.n, 3, seed=seed)
    X[-1] = X[-1] / (tt.full_sum(X) * g.delta)
    return X


def _filter(G, g, B=1, cap=16, eps=1e-6, cross_rank=S):
    return G.TTFilter(g.lo, g.hi, g.shape, np.zeros(g.d), np.ones(g.d), batch=B, rank_cap=cap, eps=eps,
                      max_shift_span=10, cross_rank=cross_rank)


@pytest.mark.parametrize("case", ["cv pairs d4", "chain d3"])
def test_one_exact_step(G, case):
    if case == "cv pairs d4":
        g = pmf.Grid([-4.0, -2.0, -4.0, -2.0], [4.0, 2.0, 4.0, 2.0], [32, 24, 32, 24])
        F = np.array([[1.0, 0.4, 0, 0], [0, 1.0, 0, 0], [0, 0, 1.0, 0.4], [0, 0, 0, 1.0]])
        Q = np.diag([0.02, 0.05, 0.03, 0.04])
    else:
        g = pmf.Grid([-3.0, -2.5, -2.0], [3.0, 2.5, 2.0], [40, 32, 24])
        F = np.array([[0.95, 0.3, 0.0], [0.0, 1.05, -0.2], [0.0, 0.0, 0.9]])
        Q = np.diag([0.05, 0.08, 0.06])
    cap, eps = 16, 1e-6
    X = _state(g, 5)
    f = _filter(G, g, cap=cap, eps=eps)
    f.import_cores(0, [np.asarray(c, dtype=np.float32) for c in X], 0.0)
    f.predict_exact(F, Q)
    ref, _, mass = T.predict_exact(X, g, F, Q, 0.0, None)
    Xt, tails, _ = T.predict_exact(X, g, F, Q, eps, cap)
    P = tt.densify(ref)
    e = rel(tt.densify(f.export_cores(0)), P)
    bound = tt_tol(eps, sum(tails))
    st = f.stats()[0]
    print(f"{case}: GPU {e:.2e}, oracle truncated {rel(tt.densify(Xt), P):.2e}, bound {bound:.1e}; "
          f"mass {st['mass_pred']:.8f} vs {mass:.8f}; ranks {f.ranks()[0].tolist()} oracle {tt.ranks(Xt)}")
    assert e <= bound, (e, bound)
    assert abs(st["mass_pred"] - mass) < 1e-5
    f.free()


def test_filter_with_exact_transition(G):
    """Constant-velocity pair with a range-like measurement of the position
    and the velocity, 48 x 40 cells, 5 steps: predict_exact + update against
    the dense oracle filter with the textbook transition."""
    g = pmf.Grid([-6.0, -3.0], [6.0, 3.0], [48, 40])
    F = np.array([[1.0, 0.5], [0.0, 1.0]])
    Q = np.diag([0.02, 0.05])
    comps = [((0,), synth.workloads.h_identity), ((1,), synth.workloads.h_sin)]
    model = synth.Model(name="cv-exact", lo=np.array(g.lo), hi=np.array(g.hi), n=np.array(g.shape),
                        m0=np.array([0.5, 0.2]), P0=np.diag([0.5, 0.3]), F=F, Q=Q, R=np.diag([0.1, 0.05]),
                        comps=comps, steps=5, eps=1e-6, rank_cap=16, config_id=8)
    x, zs = synth.simulate(model, 0)
    f = G.TTFilter(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), batch=1, rank_cap=16,
                   eps=model.eps, max_shift_span=10, cross_rank=S)
    dcomps = device_tables(model, f.grid_axes())
    oc = model.tables(g.axes)
    P = pmf.prior(g, model.m0, model.P0)
    X = [np.exp(-0.5 * (g.axes[m] - model.m0[m]) ** 2 / model.P0[m, m]).reshape(1, -1, 1) for m in range(2)]
    T.normalise(X, g)
    bound, tails_acc = 0.0, 0.0
    for k, z in enumerate(zs):
        f.predict_exact(F, Q)
        f.update(dcomps, model.R, z[None, :])
        mean, cov, lc, ll = f.estimate()
        P, _ = pmf.predict_textbook(P, g, F, Q)
        P, logc = pmf.update(P, g, pmf.likelihood(g, oc, z, model.R))
        X, tp, _ = T.predict_exact(X, g, F, Q, model.eps, 16)
        X, tu, _ = T.update(X, g, oc, z, model.R, model.eps, 16)
        tails_acc += sum(tp) + sum(tu)
        bound += tt_tol(model.eps, sum(tp) + sum(tu))
        e = rel(tt.densify(f.export_cores(0)), P)
        mo, co = pmf.moments(P, g)
        print(f"step {k}: rel L2 {e:.2e} (bound {bound:.1e}), |log c diff| {abs(lc[0] - logc):.1e}")
        assert e <= bound, (k, e, bound)
        assert abs(lc[0] - logc) < 1e-4
        assert (np.abs(mean[0] - mo) <= mean_tol(g.delta_axis, co, tails_acc)).all(), (k, mean[0], mo)
    f.free()


def test_exact_step_rejects_other_models(G):
    g = pmf.Grid([-2.0] * 3, [2.0] * 3, [12] * 3)
    f = _filter(G, g)
    for F, Q in ((np.array([[1, 0, 0.2], [0, 1, 0], [0, 0, 1.0]]), np.eye(3) * 0.1),
                 (np.array([[1, 0, 0], [0.2, 1, 0], [0, 0, 1.0]]), np.eye(3) * 0.1),
                 (np.eye(3), np.full((3, 3), 0.01) + np.eye(3) * 0.1)):
        with pytest.raises(G.TTGBFError) as ei:
            f.predict_exact(F, Q)
        assert ei.value.code == -1
    f.free()
    f = _filter(G, g, cross_rank=0)
    with pytest.raises(G.TTGBFError) as ei:
        f.predict_exact(np.eye(3), np.eye(3) * 0.1)
    assert ei.value.code == -1
    f.free()


def test_config3_exact_transition_full_size(G):
    """Config 3's model (d = 6 constant-velocity pairs, N = 256, rank cap 32,
    eps 1e-5) with the textbook transition: F is upper bidiagonal (each pair's
    coupling x_{2i} += 0.1 x_{2i+1} is the only one), so every coupled factor
    is the 2-site block of one pair, between links of rank 1.  The exact
    density is the tensor product of the three pairs' 2-D densities, each
    stepped by the oracle's untruncated exact transition and the dense
    update; the GPU density is compared with that product through TT inner
    products.  Per-step bounds 10 (eps + tau) + 1e-5 summed, tau the tails of
    the oracle TT filter with the same transition; its ranks equal the GPU's."""
    model = synth.config3(d=6, n=256)
    mcs, steps, cap = [0, 1], 3, model.rank_cap
    f = G.TTFilter(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), batch=len(mcs), rank_cap=cap,
                   eps=model.eps, max_shift_span=5, cross_rank=cap + 8)
    comps = device_tables(model, f.grid_axes())
    zs = [synth.simulate(model, mc, steps=steps)[1] for mc in mcs]
    g = pmf.Grid(model.lo, model.hi, model.n)
    oc = model.tables(g.axes)
    npair = model.d // 2
    pg = [pmf.Grid(model.lo[2 * i:2 * i + 2], model.hi[2 * i:2 * i + 2], model.n[2 * i:2 * i + 2])
          for i in range(npair)]
    P = [[pmf.prior(pg[i], model.m0[2 * i:2 * i + 2], model.P0[2 * i:2 * i + 2, 2 * i:2 * i + 2])
          for i in range(npair)] for _ in mcs]
    X = []
    for _ in mcs:
        Xb = [np.exp(-0.5 * (g.axes[m] - model.m0[m]) ** 2 / model.P0[m, m]).reshape(1, -1, 1)
              for m in range(model.d)]
        T.normalise(Xb, g)
        X.append(Xb)
    bound = [0.0] * len(mcs)
    for k in range(steps):
        f.predict_exact(model.F, model.Q)
        f.update(comps, model.R, np.stack([z[k] for z in zs]))
        for b in range(len(mcs)):
            exact = []
            for i in range(npair):
                s = slice(2 * i, 2 * i + 2)
                Xi, _, _ = T.predict_exact(tt.from_dense(P[b][i], eps=1e-14), pg[i], model.F[s, s],
                                           model.Q[s, s], 0.0, None)
                Pi = tt.densify(Xi)
                tab = [((0,), synth.workloads.h_square20(pg[i].axes[0]))]
                Pi, _ = pmf.update(Pi, pg[i], pmf.likelihood(pg[i], tab, zs[b][k][i:i + 1],
                                                               model.R[i:i + 1, i:i + 1]))
                P[b][i] = Pi
                exact += tt.from_dense(Pi, eps=1e-12)
            cores = [np.asarray(x, dtype=np.float64) for x in f.export_cores(b)]
            nn = tt.inner(exact, exact)
            e = float(np.sqrt(max(tt.inner(cores, cores) - 2.0 * tt.inner(cores, exact) + nn, 0.0) / nn))
            X[b], tp, _ = T.predict_exact(X[b], g, model.F, model.Q, model.eps, cap)
            X[b], tu, _ = T.update(X[b], g, oc, zs[b][k], model.R, model.eps, cap)
            bound[b] += tt_tol(model.eps, sum(tp) + sum(tu))
            print(f"step {k} filter {b}: rel L2 {e:.2e} (bound {bound[b]:.1e}), ranks {f.ranks()[b].tolist()}")
            assert f.ranks()[b].tolist() == tt.ranks(X[b]), (k, b)
            assert e <= bound[b], (k, b, e, bound[b])
    f.free()


def test_split_batch_exact_step(G):
    """26 filters (two concurrent parts): one textbook step of each from its
    own state, four of them against the untruncated oracle step."""
    g = pmf.Grid([-4.0, -2.0, -4.0, -2.0], [4.0, 2.0, 4.0, 2.0], [24, 20, 24, 20])
    F = np.array([[1.0, 0.4, 0, 0], [0, 1.0, 0, 0], [0, 0, 1.0, 0.4], [0, 0, 0, 1.0]])
    Q = np.diag([0.02, 0.05, 0.03, 0.04])
    B = 26
    Xs = [_state(g, 100 + b) for b in range(B)]
    f = _filter(G, g, B=B)
    for b in range(B):
        f.import_cores(b, [np.asarray(c, dtype=np.float32) for c in Xs[b]], 0.0)
    f.predict_exact(F, Q)
    for b in (0, 12, 13, B - 1):
        ref = tt.densify(T.predict_exact(Xs[b], g, F, Q, 0.0, None)[0])
        _, tails, _ = T.predict_exact(Xs[b], g, F, Q, 1e-6, 16)
        e = rel(tt.densify(f.export_cores(b)), ref)
        print(f"filter {b}: GPU {e:.2e}, bound {tt_tol(1e-6, sum(tails)):.1e}")
        assert e <= tt_tol(1e-6, sum(tails)), (b, e)
    f.free()
