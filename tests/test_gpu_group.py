"""Groups of uneven batches (ttgbf_group_*), their CUDA graphs and the launch
autotuner, through the C ABI.

* A group of batches of different d, N, rank cap and model steps every filter
  exactly as stepping each batch on its own does (the group only interleaves
  the enqueue order across streams): bitwise equal densities and estimates;
  and every filter matches the dense oracle within 10 (eps + tau) + 1e-5 per
  step (tau the oracle TT filter's tails), means within 1e-3 grid spacings
  plus 2 tau sigma.
* A recorded horizon (CUDA graph) of two steps, launched, gives what two more
  group steps give, bitwise; per-step, per-batch times come from global-timer
  stamps recorded in the graph.
* ttgbf_autotune returns a valid launch configuration and, from its cache file,
  the same one again."""
import numpy as np
import pytest

import synth
from oracle import pmf, tt
from oracle import ttfilter as T

from gpu_util import device_tables, lib_module, mean_tol, oracle_grid, oracle_tt_prior, rel, tt_tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    return lib_module()


def small_models():
    """Three uneven shapes with config 4's kind of model (factored random
    stable F, range measurement), on grids the dense oracle handles."""
    out = []
    for (d, n, cap, k) in [(3, 16, 8, 0), (4, 10, 16, 13), (3, 20, 8, 29)]:
        src = synth.config4()[k][0]
        m = synth.Model(name=f"small-d{d}-N{n}", lo=np.full(d, -8.0), hi=np.full(d, 8.0),
                        n=np.full(d, n), m0=np.zeros(d), P0=4.0 * np.eye(d),
                        F=src.F[:d, :d] if src.d >= d else np.eye(d) * 0.9, Q=src.Q[:d, :d],
                        R=src.R, comps=[((0, 1), synth.workloads.h_range)], eps=1e-6, rank_cap=cap)
        out.append(m)
    return out


def make(G, model, batch, stream):
    return G.TTFilter(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), batch=batch,
                      rank_cap=model.rank_cap, eps=model.eps, max_shift_span=min(10, 160 // model.rank_cap),
                      stream=stream)


class Run:
    """Filters, device measurements and estimate buffers of every batch."""

    def __init__(self, G, models, batches, steps):
        import torch
        self.models = models
        self.streams = [torch.cuda.Stream() for _ in models]
        self.f = [make(G, m, B, s) for m, B, s in zip(models, batches, self.streams)]
        self.comps = [device_tables(m, f.grid_axes()) for m, f in zip(models, self.f)]
        self.z = [np.stack([synth.simulate(m, 100 * i + b, steps=steps)[1] for b in range(B)], axis=1)
                  for i, (m, B) in enumerate(zip(models, batches))]
        self.zd = [torch.tensor(z, dtype=torch.float32, device="cuda") for z in self.z]
        self.out = [[torch.zeros(steps, B, m.d, dtype=torch.float64, device="cuda"),
                     torch.zeros(steps, B, m.d, m.d, dtype=torch.float64, device="cuda"),
                     torch.zeros(steps, B, dtype=torch.float64, device="cuda"),
                     torch.zeros(steps, B, dtype=torch.float64, device="cuda")]
                    for m, B in zip(models, batches)]

    def args(self, k, horizon=False):
        """Step k's arguments (the horizon's start when horizon=True)."""
        res = []
        for i, m in enumerate(self.models):
            mean, cov, lc, ll = self.out[i]
            res.append((m.F, m.Q, self.comps[i], m.R, self.zd[i][k], mean[k], cov[k], lc[k], ll[k]))
        return res


def test_group_equals_separate_batches_and_oracle(G):
    import torch
    models = small_models()
    batches = [2, 3, 2]
    steps = 3
    a = Run(G, models, batches, steps)
    b = Run(G, models, batches, steps)
    grp = G.TTFilterGroup(a.f)
    for k in range(steps):
        grp.step(a.args(k))
        for i, (f, m) in enumerate(zip(b.f, models)):
            f.predict(m.F, m.Q)
            f.update_dev(b.comps[i], m.R, b.zd[i][k])
            f.estimate_dev(*[t[k] for t in b.out[i]])
    torch.cuda.synchronize()
    assert len(grp.times()) == len(models)
    for i in range(len(models)):
        for t_a, t_b in zip(a.out[i], b.out[i]):
            assert torch.equal(t_a, t_b)
        for bb in range(batches[i]):
            ca, cb = a.f[i].export_cores(bb), b.f[i].export_cores(bb)
            assert all(np.array_equal(x, y) for x, y in zip(ca, cb))
    # every filter against the dense oracle (tails from the oracle TT filter)
    for i, m in enumerate(models):
        g = oracle_grid(m)
        oc = m.tables(g.axes)
        for bb in range(batches[i]):
            P = pmf.prior(g, m.m0, m.P0)
            X = oracle_tt_prior(m)
            bound = tacc = 0.0
            for k in range(steps):
                P, _ = pmf.predict_rg(P, g, m.F, m.Q)
                P, _ = pmf.update(P, g, pmf.likelihood(g, oc, a.z[i][k][bb], m.R))
                X, info = T.step(X, g, m.F, m.Q, oc, a.z[i][k][bb], m.R, m.eps, m.rank_cap,
                                 min(10, 160 // m.rank_cap))
                bound += tt_tol(m.eps, info["tail_sum"])
                tacc += info["tail_sum"]
            e = rel(tt.densify(a.f[i].export_cores(bb)), P)
            assert e <= bound, (m.name, bb, e, bound)
            mo, co = pmf.moments(P, g)
            mean = a.out[i][0][steps - 1, bb].cpu().numpy()
            assert (np.abs(mean - mo) <= mean_tol(g.delta_axis, co, tacc)).all(), (m.name, bb)


def test_group_graph_replays_steps(G):
    import torch
    models = small_models()
    batches = [2, 3, 2]
    steps = 5
    a = Run(G, models, batches, steps)
    b = Run(G, models, batches, steps)
    ga, gb = G.TTFilterGroup(a.f), G.TTFilterGroup(b.f)
    for r in (a, b):
        (ga if r is a else gb).step(r.args(0))
    # a: a recorded horizon of two steps, launched twice (refilled measurements)
    horizon = 2
    zbuf = [torch.zeros((horizon,) + tuple(z.shape[1:]), dtype=torch.float32, device="cuda") for z in a.zd]
    obuf = [[torch.zeros((horizon,) + tuple(t.shape[1:]), dtype=t.dtype, device="cuda") for t in o]
            for o in a.out]
    cap_args = [(m.F, m.Q, a.comps[i], m.R, zbuf[i], *obuf[i]) for i, m in enumerate(models)]
    ga.capture(cap_args, horizon)
    assert ga.graph_kernels() > 0
    for rep in range(2):
        for i in range(len(models)):
            zbuf[i].copy_(a.zd[i][1 + rep * horizon: 1 + (rep + 1) * horizon])
        ga.launch()
        torch.cuda.synchronize()
        gt = ga.graph_times()  # per step and batch, from the timer stamps recorded in the graph
        assert gt.shape == (horizon, len(models)) and (gt > 0).all()
        for i in range(len(models)):
            for o, t in zip(obuf[i], a.out[i]):
                t[1 + rep * horizon: 1 + (rep + 1) * horizon].copy_(o)
    # b: the same four steps as group steps
    for k in range(1, steps):
        gb.step(b.args(k))
    torch.cuda.synchronize()
    for i in range(len(models)):
        for t_a, t_b in zip(a.out[i], b.out[i]):
            assert torch.equal(t_a[1:], t_b[1:]), i
        for bb in range(batches[i]):
            assert all(np.array_equal(x, y) for x, y in
                       zip(a.f[i].export_cores(bb), b.f[i].export_cores(bb)))


def test_autotune_and_cache(G, tmp_path):
    m = synth.config2(n=24)
    cache = str(tmp_path / "tune.txt")
    best, ms = G.autotune(m.lo, m.hi, m.n, m.m0, np.diag(m.P0), m.F, m.Q, batch=4, rank_cap=16,
                          eps=1e-6, steps=2, cache_path=cache)
    assert best["parts"] in (1, 2, 4) and best["tsqr_slice_blocks"] in (4, 8, 16)
    assert best["svd_threads"] in (512, 1024) and ms > 0
    again, ms2 = G.autotune(m.lo, m.hi, m.n, m.m0, np.diag(m.P0), m.F, m.Q, batch=4, rank_cap=16,
                            eps=1e-6, steps=2, cache_path=cache)
    assert again == best and abs(ms2 - ms) < 1e-3 * ms
    with open(cache) as fh:
        assert len(fh.read().strip().splitlines()) == 1
    # the chosen configuration runs and tracks the default one
    f = G.TTFilter(m.lo, m.hi, m.n, m.m0, np.diag(m.P0), batch=4, rank_cap=16, eps=1e-6, **best)
    f0 = G.TTFilter(m.lo, m.hi, m.n, m.m0, np.diag(m.P0), batch=4, rank_cap=16, eps=1e-6)
    comps = device_tables(m, f.grid_axes())
    z = np.stack([synth.simulate(m, b, steps=2)[1] for b in range(4)], axis=1)
    for k in range(2):
        for x in (f, f0):
            x.predict(m.F, m.Q)
            x.update(comps, m.R, z[k])
    for b in range(4):
        assert rel(tt.densify(f.export_cores(b)), tt.densify(f0.export_cores(b))) < 1e-4
