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
