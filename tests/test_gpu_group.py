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


def test_group_and_graph_with_a_cross_component(G):
    """A batch whose likelihood factor couples three modes (applied by the TT
    cross, cross_rank 16) in a group with an ordinary batch: a group step, and
    a recorded two-step horizon launched, give bitwise what stepping the batch
    on its own gives."""
    import torch
    m3 = synth.Model(name="range3-small", lo=np.full(3, -4.0), hi=np.full(3, 4.0), n=np.full(3, 16),
                     m0=np.array([1.0, 0.5, 0.2]), P0=np.eye(3), F=np.eye(3) * 0.95, Q=np.eye(3) * 0.05,
                     R=np.array([[0.05]]), comps=[((0, 1, 2), synth.workloads.h_range3)], eps=1e-6, rank_cap=8)
    m2 = small_models()[1]
    B3, B2, steps = 2, 3, 3
    z3 = np.stack([synth.simulate(m3, b, steps=steps)[1] for b in range(B3)], axis=1)
    z2 = np.stack([synth.simulate(m2, b, steps=steps)[1] for b in range(B2)], axis=1)

    def contexts():
        s3, s2 = torch.cuda.Stream(), torch.cuda.Stream()
        f3 = G.TTFilter(m3.lo, m3.hi, m3.n, m3.m0, np.diag(m3.P0), batch=B3, rank_cap=8, eps=1e-6,
                        max_shift_span=10, stream=s3, cross_rank=16)
        f2 = make(G, m2, B2, s2)
        return f3, f2

    def outs(m, B):
        return [torch.zeros(B, m.d, dtype=torch.float64, device="cuda"),
                torch.zeros(B, m.d, m.d, dtype=torch.float64, device="cuda"),
                torch.zeros(B, dtype=torch.float64, device="cuda"),
                torch.zeros(B, dtype=torch.float64, device="cuda")]

    fa3, fa2 = contexts()
    fb3, fb2 = contexts()
    c3 = device_tables(m3, fa3.grid_axes())
    c2 = device_tables(m2, fa2.grid_axes())
    z3d = torch.tensor(z3, dtype=torch.float32, device="cuda")
    z2d = torch.tensor(z2, dtype=torch.float32, device="cuda")
    grp = G.TTFilterGroup([fa3, fa2])
    oa3, oa2, ob3, ob2 = outs(m3, B3), outs(m2, B2), outs(m3, B3), outs(m2, B2)
    # step 0 as a group step; steps 1, 2 as a recorded horizon of two steps
    grp.step([(m3.F, m3.Q, c3, m3.R, z3d[0], *oa3), (m2.F, m2.Q, c2, m2.R, z2d[0], *oa2)])
    zb3 = torch.zeros((2, B3, 1), dtype=torch.float32, device="cuda")
    zb2 = torch.zeros((2, B2, 1), dtype=torch.float32, device="cuda")
    ob = [[torch.zeros((2,) + tuple(t.shape), dtype=t.dtype, device="cuda") for t in o] for o in (oa3, oa2)]
    grp.capture([(m3.F, m3.Q, c3, m3.R, zb3, *ob[0]), (m2.F, m2.Q, c2, m2.R, zb2, *ob[1])], 2)
    zb3.copy_(z3d[1:3])
    zb2.copy_(z2d[1:3])
    grp.launch()
    for k in range(steps):
        for f, m, c, zd, o in ((fb3, m3, c3, z3d, ob3), (fb2, m2, c2, z2d, ob2)):
            f.predict(m.F, m.Q)
            f.update_dev(c, m.R, zd[k])
            f.estimate_dev(*o)
    torch.cuda.synchronize()
    for fa, fb, B in ((fa3, fb3, B3), (fa2, fb2, B2)):
        for b in range(B):
            assert all(np.array_equal(x, y) for x, y in zip(fa.export_cores(b), fb.export_cores(b)))
    assert torch.equal(ob[0][0][1], ob3[0]) and torch.equal(ob[0][2][1], ob3[2])
    # and the cross batch against the dense oracle (tails from the oracle TT filter with its cross)
    g = oracle_grid(m3)
    oc = m3.tables(g.axes)
    for b in range(B3):
        P = pmf.prior(g, m3.m0, m3.P0)
        X = oracle_tt_prior(m3)
        bound = 0.0
        for k in range(steps):
            P, _ = pmf.predict_rg(P, g, m3.F, m3.Q)
            P, _ = pmf.update(P, g, pmf.likelihood(g, oc, z3[k][b], m3.R))
            X, info = T.step(X, g, m3.F, m3.Q, oc, z3[k][b], m3.R, m3.eps, 8, 10)
            bound += tt_tol(m3.eps, info["tail_sum"])
        e = rel(tt.densify(fa3.export_cores(b)), P)
        assert e <= bound, (b, e, bound)
    for f in (fa3, fa2, fb3, fb2):
        f.free()
