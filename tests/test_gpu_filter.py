"""GPU parity of whole filter steps (predict -> update -> estimate) on the
benchmark workloads against the dense FP64 oracle.

Tolerances: per step the TT density may deviate from the oracle by
10 * (eps + tau) + 1e-5 in relative Frobenius norm, tau being the discarded
relative tails of the float64 TT filter of oracle/ttfilter.py run on the same
measurements with the same rank cap (tau is at the eps level when the cap
does not bind; no bound uses a tail the GPU reports).  Over several steps the
bounds of the steps add.  Posterior means agree within 1e-3 grid spacings,
plus 2 tau sigma_m where the rank cap binds (tau the oracle's summed tails,
sigma_m the oracle's marginal standard deviation)."""
import numpy as np
import pytest

import synth
from oracle import pmf, tt
from oracle import ttfilter as T

from gpu_util import (cov_tol, device_tables, lib_module, make_filter, mean_tol, oracle_grid,
                      oracle_tt_prior, rel, tt_tol)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    return lib_module()


def run_compare(G, model, mcs, steps, batch_extra=0):
    """Run len(mcs) filters on the GPU, and the dense oracle and the oracle TT
    filter (for the tails) on each; return per-step errors (density rel,
    mean err / tolerance, |log c diff|) and the bounds."""
    B = len(mcs) + batch_extra
    f = make_filter(G, model, batch=B)
    X = [oracle_tt_prior(model) for _ in mcs]
    comps = device_tables(model, f.grid_axes())
    g = oracle_grid(model)
    oc = model.tables(g.axes)
    zs = [synth.simulate(model, mc, steps=steps)[1] for mc in mcs]
    zs += [zs[0]] * batch_extra
    Ps = [pmf.prior(g, model.m0, model.P0) for _ in mcs]
    bound = [0.0] * len(mcs)
    tacc = [0.0] * len(mcs)
    out = []
    for k in range(steps):
        f.predict(model.F, model.Q)
        f.update(comps, model.R, np.stack([z[k] for z in zs]))
        st = f.stats()
        m, c, lc, ll = f.estimate()
        row = []
        for i in range(len(mcs)):
            Ps[i], _ = pmf.predict_rg(Ps[i], g, model.F, model.Q)
            Ps[i], logc = pmf.update(Ps[i], g, pmf.likelihood(g, oc, zs[i][k], model.R))
            mo, co = pmf.moments(Ps[i], g)
            X[i], info = T.step(X[i], g, model.F, model.Q, oc, zs[i][k], model.R, model.eps,
                                model.rank_cap)
            bound[i] += tt_tol(model.eps, info["tail_sum"])  # the oracle's predict + update tails
            tacc[i] += info["tail_sum"]
            e = rel(tt.densify(f.export_cores(i)), Ps[i])
            # mean error in units of its tolerance (< 1 passes)
            merr = float((np.abs(m[i] - mo) / mean_tol(g.delta_axis, co, tacc[i])).max())
            row.append((e, bound[i], merr, abs(lc[i] - logc), st[i]["max_rank"]))
        out.append(row)
    return out, f


def test_config1_vs_oracle(G):
    model = synth.config1()
    out, f = run_compare(G, model, [0, 1], model.steps)
    for k, row in enumerate(out):
        for e, bound, merr, dlc, mr in row:
            assert e <= bound, (k, e, bound)
            assert merr < 1.0, (k, merr)
            assert dlc < 1e-3 + bound, (k, dlc)
            assert mr <= model.rank_cap


def test_config1_linear_tracks_kalman(G):
    from oracle import kalman
    model = synth.config1_linear()
    x, z = synth.simulate(model, 3, steps=10)
    f = make_filter(G, model)
    comps = device_tables(model, f.grid_axes())
    kf = kalman.kalman(model.m0, model.P0, model.F, model.Q, np.eye(2), model.R, z)
    for k in range(10):
        f.predict(model.F, model.Q)
        f.update(comps, model.R, z[k][None, :])
    m, c, lc, ll = f.estimate()
    # discretisation error of the re-gridded transition at N = 64 (the oracle's
    # own distance to the Kalman filter is of the same size)
    assert np.abs(m[0] - kf["means"][-1]).max() < 0.05
    assert np.abs(c[0] - kf["covs"][-1]).max() < 0.01


def test_config2_small_grid_multi_step(G):
    model = synth.config2(n=32)
    out, f = run_compare(G, model, [0, 1], 6)
    for k, row in enumerate(out):
        for e, bound, merr, dlc, mr in row:
            assert e <= bound, (k, e, bound)
            assert merr < 1.0, (k, merr)
            assert mr <= 16


def test_config2_one_step_from_oracle_posterior(G):
    # shared input: the oracle's posterior after 3 steps, compressed by the
    # oracle's TT rounding; both sides take one predict + update from it
    model = synth.config2(n=32)
    g = oracle_grid(model)
    oc = model.tables(g.axes)
    x, z = synth.simulate(model, 5, steps=4)
    P = pmf.prior(g, model.m0, model.P0)
    for k in range(3):
        P, _ = pmf.predict_rg(P, g, model.F, model.Q)
        P, _ = pmf.update(P, g, pmf.likelihood(g, oc, z[k], model.R))
    cores, _ = tt.round_tt(tt.from_dense(P), 1e-7, 16)
    cores = [c.astype(np.float32) for c in cores]
    P_in = tt.densify([c.astype(np.float64) for c in cores])
    P_in, _ = pmf.normalise(P_in, g)
    f = make_filter(G, model)
    f.import_cores(0, cores)
    f.normalise()
    comps = device_tables(model, f.grid_axes())
    f.predict(model.F, model.Q)
    Xp, tp, _ = T.predict([c.astype(np.float64) for c in cores], g, model.F, model.Q, model.eps, 16)
    t_pred = sum(tp)
    Pp, _ = pmf.predict_rg(P_in, g, model.F, model.Q)
    assert rel(tt.densify(f.export_cores(0)), Pp) <= tt_tol(model.eps, t_pred)
    f.update(comps, model.R, z[3][None, :])
    _, tu, _ = T.update(Xp, g, oc, z[3], model.R, model.eps, 16)
    t_step = t_pred + sum(tu)  # the oracle's predict + update tails of this step
    Pu, logc = pmf.update(Pp, g, pmf.likelihood(g, oc, z[3], model.R))
    assert rel(tt.densify(f.export_cores(0)), Pu) <= tt_tol(model.eps, t_step)
    m, c, lc, ll = f.estimate()
    mo, co = pmf.moments(Pu, g)
    assert (np.abs(m[0] - mo) <= mean_tol(g.delta_axis, co, t_step)).all()
    assert abs(lc[0] - logc) < 1e-3


def test_batch_filters_are_independent(G):
    model = synth.config2(n=24)
    out, f = run_compare(G, model, [7, 8, 9], 3, batch_extra=2)
    for row in out:
        for e, bound, merr, dlc, mr in row:
            assert e <= bound and merr < 1.0
    # the two extra filters saw filter 0's measurements
    a = tt.densify(f.export_cores(0))
    np.testing.assert_allclose(tt.densify(f.export_cores(3)), a, rtol=0, atol=0)
    np.testing.assert_allclose(tt.densify(f.export_cores(4)), a, rtol=0, atol=0)


@pytest.mark.slow
def test_config2_full_size_bench_launch(G):
    """The bench's launch configuration (100 filters, 128^4 grid, rank cap 16,
    eps 1e-6): filter 0 is compared with the oracle over two steps on the full
    grid; every filter is checked for unit mass, finite moments and ranks."""
    model = synth.config2(n=128)
    B = 100
    f = make_filter(G, model, batch=B)
    comps = device_tables(model, f.grid_axes())
    zs = np.stack([synth.simulate(model, mc, steps=2)[1] for mc in range(B)], axis=1)
    g = oracle_grid(model)
    oc = model.tables(g.axes)
    P = pmf.prior(g, model.m0, model.P0)
    X = oracle_tt_prior(model)
    bound = 0.0
    tacc = 0.0
    for k in range(2):
        f.predict(model.F, model.Q)
        f.update(comps, model.R, zs[k])
        st = f.stats()
        X, info = T.step(X, g, model.F, model.Q, oc, zs[k][0], model.R, model.eps, model.rank_cap)
        bound += tt_tol(model.eps, info["tail_sum"])
        tacc += info["tail_sum"]
        P, _ = pmf.predict_rg(P, g, model.F, model.Q)
        P, logc = pmf.update(P, g, pmf.likelihood(g, oc, zs[k][0], model.R))
        m, c, lc, ll = f.estimate()
        e = rel(tt.densify(f.export_cores(0)), P)
        assert e <= bound, (k, e, bound)
        mo, co = pmf.moments(P, g)
        assert (np.abs(m[0] - mo) <= mean_tol(g.delta_axis, co, tacc)).all()
        assert abs(lc[0] - logc) < 1e-3
        assert np.isfinite(m).all() and np.isfinite(c).all() and np.isfinite(lc).all()
        assert (np.abs(m) < 8).all()
        assert (f.ranks() <= 16).all()
        assert all(s["max_rank"] <= 16 for s in st)


def test_batch_split_into_concurrent_parts(G, monkeypatch):
    """A batch split into parts on their own streams (the library's default
    for large batches) gives each filter what the unsplit batch gives it:
    same ranks, densities and moments up to FP32 rounding (the QR's row
    slicing depends on the batch size)."""
    model = synth.config2(n=24)
    B = 8
    zs = np.stack([synth.simulate(model, mc, steps=3)[1] for mc in range(B)], axis=1)
    outs = []
    for parts in ("1", "3"):
        monkeypatch.setenv("TTGBF_PARTS", parts)
        f = make_filter(G, model, batch=B)
        comps = device_tables(model, f.grid_axes())
        for k in range(3):
            f.predict(model.F, model.Q)
            f.update(comps, model.R, zs[k])
        m, c, lc, ll = f.estimate()
        outs.append((f.ranks(), [tt.densify(f.export_cores(b)) for b in range(B)], m, lc, ll,
                     [s["tail_sum"] for s in f.stats()]))
        f.free()
    (r1, d1, m1, lc1, ll1, t1), (r3, d3, m3, lc3, ll3, t3) = outs
    np.testing.assert_array_equal(r1, r3)
    for b in range(B):
        assert rel(d3[b], d1[b]) < 1e-4
    np.testing.assert_allclose(m3, m1, rtol=0, atol=1e-5)
    np.testing.assert_allclose(lc3, lc1, rtol=0, atol=1e-5)
    np.testing.assert_allclose(ll3, ll1, rtol=0, atol=1e-4)
    np.testing.assert_allclose(t3, t1, rtol=1e-3, atol=1e-6)


@pytest.mark.parametrize("parts", ["1", "3"])
def test_densify_on_device(G, monkeypatch, parts):
    """ttgbf_densify contracts a filter's cores into the full grid on the
    device: the same tensor as the host contraction of the exported cores
    (both in float64 from the same float32 cores, so equal up to the order of
    the sums), normalised to 1 / cell volume after a step, and within one
    step's parity bound of the dense oracle; too small a buffer and a filter
    index out of range are refused."""
    monkeypatch.setenv("TTGBF_PARTS", parts)
    model = synth.config2(n=24)
    B = 4
    zs = np.stack([synth.simulate(model, mc, steps=1)[1] for mc in range(B)], axis=1)
    f = make_filter(G, model, batch=B)
    comps = device_tables(model, f.grid_axes())
    f.predict(model.F, model.Q)
    f.update(comps, model.R, zs[0])
    g = oracle_grid(model)
    oc = model.tables(g.axes)
    X0 = oracle_tt_prior(model)
    for b in range(B):
        D = f.densify(b)
        assert D.shape == tuple(model.n)
        H = tt.densify(f.export_cores(b))
        assert float(np.abs(D - H).max()) <= 1e-12 * float(np.abs(H).max())
        assert abs(D.sum() * g.delta - 1.0) < 1e-5
        P, _ = pmf.predict_rg(pmf.prior(g, model.m0, model.P0), g, model.F, model.Q)
        P, _ = pmf.update(P, g, pmf.likelihood(g, oc, zs[0][b], model.R))
        _, info = T.step(X0, g, model.F, model.Q, oc, zs[0][b], model.R, model.eps, model.rank_cap)
        assert rel(D, P) <= tt_tol(model.eps, info["tail_sum"])
    total = int(np.prod(model.n))
    with pytest.raises(G.TTGBFError) as ei:
        f.densify(0, cap=total - 1)
    assert ei.value.code == -3
    with pytest.raises(G.TTGBFError) as ei:
        f.densify(B)
    assert ei.value.code == -1
    f.free()


def test_shears_in_pieces_small_grid(G):
    """Every shear of the 32^4 workload spans 3 shifts; with a span of 2 each
    runs as two rounded pieces (both triangles' couplings, including the
    non-adjacent ones with block-diagonal middle cores) whose TT sum is
    rounded again.  Same tolerance against the oracle as the whole
    expansion."""
    model = synth.config2(n=32)
    mcs = [3, 4]
    steps = 3
    f = make_filter(G, model, batch=len(mcs), smax=2)
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
                                model.rank_cap, 2)
            bound[i] += tt_tol(model.eps, info["tail_sum"])
            tacc[i] += info["tail_sum"]
            e = rel(tt.densify(f.export_cores(i)), Ps[i])
            assert e <= bound[i], (k, i, e, bound[i])
            assert (np.abs(m[i] - mo) <= mean_tol(g.delta_axis, co, tacc[i])).all(), (k, i)
            assert (np.abs(c[i] - co) <= cov_tol(g.delta_axis, co)).all(), (k, i)
            assert abs(lc[i] - logc) < 1e-3, (k, i)
            assert st[i]["max_rank"] <= model.rank_cap


@pytest.mark.parametrize("batch", [2, 24])
def test_injected_cuda_error_poisons_context(G, monkeypatch, batch):
    """Failure detection without a GPU fault: TTGBF_FAULT=cuda:2 makes the
    second status check after init report a CUDA error.  That call returns
    TTGBF_ECUDA, every later call TTGBF_EPOISONED (for a batch split into
    parts as well), and the context is still freed cleanly."""
    monkeypatch.setenv("TTGBF_FAULT", "cuda:2")
    model = synth.config2(n=16)
    f = make_filter(G, model, batch=batch)
    monkeypatch.delenv("TTGBF_FAULT")
    comps = device_tables(model, f.grid_axes())
    z = np.stack([synth.simulate(model, mc, steps=1)[1][0] for mc in range(batch)])
    f.predict(model.F, model.Q)  # first check: fine
    with pytest.raises(G.TTGBFError) as ei:
        f.update(comps, model.R, z)  # second check: the injected error
    assert ei.value.code == -4
    for call in (lambda: f.estimate(), lambda: f.predict(model.F, model.Q),
                 lambda: f.update(comps, model.R, z)):
        with pytest.raises(G.TTGBFError) as ei:
            call()
        assert ei.value.code == -7
    f.free()
    # a fresh context is unaffected
    g = make_filter(G, model, batch=batch)
    g.predict(model.F, model.Q)
    g.update(comps, model.R, z)
    m, c, lc, ll = g.estimate()
    assert np.isfinite(m).all() and np.isfinite(lc).all()
