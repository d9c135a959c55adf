#!/usr/bin/env python3
"""Throughput of the tensor-train point-mass filter step on GB300.

Workload (config 2 of the paper-shaped illustrations): d = 4, a 128^4 grid on
[-8, 8]^4, 100 independent Monte Carlo filters per GPU (seeded trajectories),
linear dynamics F = 0.95 I + 0.05 U (U seeded upper triangular), Q = 0.05 I,
range measurement z = ||x[0:2]|| + v with R = 0.01, TT rank cap 16, rounding
eps 1e-6, FP32 cores.

One bench step = one Bayesian recursion step of every filter of the batch:
predict (re-gridding shears with TT rounding, per-mode Gaussian kernel,
normalisation) -> update (likelihood on the merged first two cores, rounding,
normalisation, log normaliser) -> estimate (mean and covariance).
`value` counts filter steps per second over all GPUs (weak scaling: every
rank runs its own 100 filters, no collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "TT filter steps/s vs full-grid GPU filter at matched density error; % HBM/TC roofline"
WORKLOAD = ("config2: d=4, 128^4 grid on [-8,8]^4, F=0.95I+0.05U, Q=0.05I, range measurement "
            "R=0.01, rank cap 16, eps 1e-6")
UNIT = "filter-steps/s"
L2_FLUSH_BYTES = 256 << 20  # larger than the 126 MiB L2 of GB300
# TT configurations of the accuracy sweep: (rank cap, max shift span, rounding
# precision); rank cap x span <= 160 (wider shears run in pieces)
SWEEP = [(16, 10, "fp32", "fp32"), (32, 5, "fp32", "fp32"), (48, 3, "fp32", "fp32"),
         (16, 10, "fp64", "fp32"), (16, 10, "fp32", "tf32x3"), (16, 10, "fp32", "tf32")]
# DRAM bytes read + written by the k_tsqr launches of one config-2 filter step
# (rank cap 16): one ncu capture of every launch of a 12-filter step
# (profiles/k_tsqr_traffic_config2_part12.md: 226.7 MB over 12 filters),
# scaled by the filters a launch processes
TSQR_DRAM_BYTES_PER_FILTER_STEP = 226.64e6 / 12
# nominal dense TF32 : BF16 tensor rate of the GPU (1.1 : 2.25 PFLOP/s)
TF32_PER_BF16 = 1.1 / 2.25


def shard_mc_ids(rank: int, world: int, batch: int) -> list[int]:
    """Monte Carlo runs of one rank: rank r owns runs r*batch .. r*batch+batch-1."""
    return list(range(rank * batch, (rank + 1) * batch))


def measurement_batches(model, mc_ids, steps):
    """z[k] for k < steps, shape (steps, len(mc_ids), b)."""
    return np.stack([synth.simulate(model, mc, steps=steps)[1] for mc in mc_ids], axis=1)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx = float(p[2])
                except ValueError:
                    continue
                for nm, v in zip(names, p[5:9]):
                    if v.lower() in ("active", "1"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_step(model, mc: int):
    """Time one dense FP64 oracle filter step (predict, update, moments) of one
    Monte Carlo run on the full grid.  Returns (seconds, description)."""
    from oracle import pmf
    g = pmf.Grid(model.lo, model.hi, model.n)
    comps = model.tables(g.axes)
    x, z = synth.simulate(model, mc, steps=1)
    P = pmf.prior(g, model.m0, model.P0)
    t0 = time.perf_counter()
    P, _ = pmf.predict_rg(P, g, model.F, model.Q)
    P, _ = pmf.update(P, g, pmf.likelihood(g, comps, z[0], model.R))
    pmf.moments(P, g)
    dt = time.perf_counter() - t0
    return dt, (f"1 filter step (Monte Carlo run {mc}, step 1: predict, update, moments) of the "
                f"same workload on the dense {'x'.join(str(int(v)) for v in model.n)} grid, "
                "FP64 numpy oracle")


def log(msg):
    """Progress of the run on stderr (the JSON line goes to stdout)."""
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def ldu_ops(F):
    """The elementary re-gridding operations the library applies for x -> F x
    (F = L D U without pivoting): ("shear", m, n, a) for x_m += a x_n and
    ("scale", m, lam), in the library's order (U's shears, D, L's shears).
    Bookkeeping for the algorithmic work counts below."""
    A = np.asarray(F, dtype=np.float64)
    d = A.shape[0]
    L, U, D = np.eye(d), np.eye(d), np.zeros(d)
    for k in range(d):
        D[k] = A[k, k] - sum(L[k, j] * D[j] * U[j, k] for j in range(k))
        for i in range(k + 1, d):
            L[i, k] = (A[i, k] - sum(L[i, j] * D[j] * U[j, k] for j in range(k))) / D[k]
            U[k, i] = (A[k, i] - sum(L[k, j] * D[j] * U[j, i] for j in range(k))) / D[k]
    ops = [("shear", m, n, U[m, n]) for m in range(d) for n in range(m + 1, d) if U[m, n] != 0.0]
    ops += [("scale", m, D[m]) for m in range(d) if D[m] != 1.0]
    ops += [("shear", m, n, L[m, n]) for m in range(d - 1, -1, -1) for n in range(m) if L[m, n] != 0.0]
    return ops


def shear_span(model, m, n, a) -> int:
    """Integer shifts carrying hat weight in the shear x_m += a x_n."""
    D = (model.hi - model.lo) / model.n
    xi = model.lo[n] + (np.arange(model.n[n]) + 0.5) * D[n]
    s = a * xi / D[m]
    return int(np.floor(s).max() - np.floor(s).min()) + 2


def fullgrid_bytes_per_step(model) -> int:
    """Algorithmic HBM bytes of one dense float32 step as the full-grid filter
    runs it: with F = D U (no L shears) one fused pass per axis (its shears,
    scaling and kernel) and one pass for the likelihood with the posterior
    moments, each reading and writing the density once; otherwise a pass per
    shear, per scaling axis and per kernel axis, a normalising pass, the
    likelihood pass and a moments read."""
    ops = ldu_ops(model.F)
    cells = int(np.prod(model.n))
    lower = any(op[0] == "shear" and op[1] > op[2] for op in ops)
    if not lower:
        return cells * 4 * 2 * (model.d + 1)
    n_shear = sum(1 for op in ops if op[0] == "shear")
    n_scale = sum(1 for op in ops if op[0] == "scale")
    passes_rw = n_shear + n_scale + model.d + 1 + 1
    return cells * 4 * (2 * passes_rw + 1)


def tsqr_algorithmic_bytes(model, rank_cap) -> float:
    """Algorithmic bytes of the same R factors: every rank-expanded (r N) x
    (r S) unfolding read once in float32."""
    r = rank_cap
    tot = 0.0
    for op in ldu_ops(model.F):
        if op[0] != "shear":
            continue
        _, m, n, a = op
        S = shear_span(model, m, n, a)
        N = int(model.n[min(m, n)])
        tot += abs(m - n) * 4.0 * (r * N) * (r * S)
    return tot


def tsqr_algorithmic_flops(model, rank_cap) -> float:
    """Algorithmic flops of the R factors of one filter step's roundings (the
    rank-expanded links): per elementary shear of span S, every link it
    expands carries an (r N) x (r S) unfolding whose R factor costs
    2 (r N) (r S)^2 flops (r the rank cap, N the points per axis)."""
    r = rank_cap
    tot = 0.0
    for op in ldu_ops(model.F):
        if op[0] != "shear":
            continue
        _, m, n, a = op
        S = shear_span(model, m, n, a)
        N = int(model.n[min(m, n)])
        tot += abs(m - n) * 2.0 * (r * N) * (r * S) ** 2
    return tot


def tt_dense_rel_err(cores, P) -> float:
    """||T - P||_F / ||P||_F of a TT (cores [r_{k-1}][N_k][r_k]) and a dense
    float64 density P, from <T, T>, <T, P> and <P, P>: T is never formed."""
    cores = [np.asarray(c, dtype=np.float64) for c in cores]
    E = np.ones((1, 1))
    for C in cores:
        E = np.einsum("ab,aic,bid->cd", E, C, C)
    tt2 = float(E[0, 0])
    X = np.tensordot(P, cores[-1][:, :, 0], axes=([P.ndim - 1], [1]))
    for C in reversed(cores[:-1]):
        X = np.tensordot(X, C, axes=([X.ndim - 2, X.ndim - 1], [1, 2]))
    tp = float(np.asarray(X).reshape(-1)[0])
    pp = float(np.vdot(P, P))
    return math.sqrt(max(tt2 - 2.0 * tp + pp, 0.0) / pp)


def run_fullgrid(args, model, zs, W, K, dev, axes):
    """The plain full-grid float32 filter on the same workload (one Monte Carlo
    run, the batch's first): steps/s and achieved HBM bandwidth."""
    import torch
    import paper_2501_07942_gb300 as G
    fg = G.FullGridFilter(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), precision=32,
                          device=dev)
    comps = [(m, torch.tensor(np.asarray(t), dtype=torch.float32, device=dev))
             for m, t in model.tables(axes)]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    for k in range(W):
        fg.predict(model.F, model.Q)
        fg.update(comps, model.R, zs[k][0])
        fg.estimate()
    ms = 0.0
    if args.profile_fullgrid:
        torch.cuda.profiler.start()
    for i in range(K):
        flush.fill_(i & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fg.predict(model.F, model.Q)
        fg.update(comps, model.R, zs[W + i][0])
        fg.estimate()
        b.record(stream)
        torch.cuda.synchronize(dev)
        ms += a.elapsed_time(b)
    if args.profile_fullgrid:
        torch.cuda.profiler.stop()
    out = {"value": K / (ms * 1e-3), "unit": "filter-steps/s (one filter)", "dtype": "f32",
           "ms_per_step": ms / K}
    pk, src = peaks()
    bytes_step = fullgrid_bytes_per_step(model)
    gbs = bytes_step / (ms / K * 1e-3) / 1e9
    out["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                       "frac": gbs / pk["hbm_gbs"], "traffic": None, "peak_source": src,
                       "bytes_per_step": bytes_step}
    fg.free()
    return out


def fp64_reference_densities(model, zs, S, dev, axes):
    """The float64 full-grid GPU filter (parity-tested against the oracle to
    1e-12) on Monte Carlo run 0 for S steps: its density after every step,
    as host float64 arrays (a generator, one step at a time)."""
    import torch
    import paper_2501_07942_gb300 as G
    fg = G.FullGridFilter(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), precision=64,
                          device=dev)
    comps = [(m, torch.tensor(np.asarray(t), dtype=torch.float64, device=dev))
             for m, t in model.tables(axes)]
    try:
        for k in range(S):
            fg.predict(model.F, model.Q)
            fg.update(comps, model.R, zs[k][0])
            yield fg.density()
    finally:
        fg.free()


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    model = synth.config2()
    # warm-up steps (untimed) run the same oracle code on a 32^4 grid: the
    # numpy oracle has nothing to compile or cache, and 30 s per full-size
    # step would make the untimed part dominate the run
    small = synth.config2(n=32)
    for k in range(args.warmup):
        cpu_oracle_step(small, k % args.batch)
    times = []
    for k in range(args.steps):
        dt, desc = cpu_oracle_step(model, k % args.batch)
        times.append(dt)
    total = sum(times)
    value = len(times) / total
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "filters_per_step": 1,
                       "l2": "not applicable (host numpy oracle)",
                       "parallelism": "host cores of rank 0"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


TUNE_CACHE = os.path.join(ROOT, "paper_2501_07942_gb300", "tune_cache.txt")


def run_config4(args, dev):
    """The uneven batch (512 filters, 36 (d, N, rank cap) groups, each with its
    own random stable F, Q, R): every group a TTFilter batch on its own stream
    (launch configuration from the autotuner's persisted choices), all stepped
    together by one TTFilterGroup; a horizon of H steps recorded into one CUDA
    graph and launched until the timed steps are done, the measurements of the
    next H steps copied into the graph's buffer before each launch (inside the
    timed region).  Per-filter step latency: the GPU's global timer, written
    by one-thread kernels recorded with the graph at every step's start and at
    the end of every batch's step, read after the last timed launch (every
    filter of a batch finishes with it)."""
    log("config4 leg")
    import torch
    import paper_2501_07942_gb300 as G
    groups = synth.config4()
    total = args.c4_steps
    H = min(args.c4_horizon, total)
    reps = max(1, total // H)
    st = torch.cuda.Stream(dev)
    filters, models, streams, comps, zall, zbuf, outs, tuned = [], [], [], [], [], [], [], 0
    for m, ids in groups:
        s = torch.cuda.Stream(dev)
        smax = min(10, 160 // m.rank_cap)
        kw = tuned_config(G, m, len(ids), m.rank_cap, smax, "fp32")
        tuned += bool(kw)
        f = G.TTFilter(m.lo, m.hi, m.n, m.m0, np.diag(m.P0), batch=len(ids), rank_cap=m.rank_cap,
                       eps=m.eps, max_shift_span=smax, stream=s, device=dev, **kw)
        filters.append(f)
        models.append(m)
        streams.append(s)
        comps.append([(md, torch.tensor(np.asarray(t), dtype=torch.float32, device=dev))
                      for md, t in m.tables(f.grid_axes())])
        z = np.stack([synth.simulate(m, fid, steps=reps * H + 1)[1] for fid in ids], axis=1)
        zall.append(torch.tensor(z, dtype=torch.float32, device=dev))
        zbuf.append(torch.zeros((H,) + tuple(z.shape[1:]), dtype=torch.float32, device=dev))
        B = len(ids)
        outs.append([torch.zeros(H, B, m.d, dtype=torch.float64, device=dev),
                     torch.zeros(H, B, m.d, m.d, dtype=torch.float64, device=dev),
                     torch.zeros(H, B, dtype=torch.float64, device=dev),
                     torch.zeros(H, B, dtype=torch.float64, device=dev)])
    grp = G.TTFilterGroup(filters, stream=st, device=dev)
    step_args = lambda k: [(m.F, m.Q, comps[i], m.R, zall[i][k], outs[i][0][0], outs[i][1][0],
                            outs[i][2][0], outs[i][3][0]) for i, m in enumerate(models)]
    # one eager group step (the recorded horizon must start from a stepped
    # state), the recording, then the timed launches (the first one includes
    # the graph's upload)
    t_eager = time.time()
    grp.step(step_args(0))
    torch.cuda.synchronize(dev)
    t_eager = time.time() - t_eager
    log(f"config4: eager group step {t_eager:.1f} s")
    grp.capture([(m.F, m.Q, comps[i], m.R, zbuf[i], *outs[i]) for i, m in enumerate(models)], H)
    nk = grp.graph_kernels()
    log(f"config4: recorded {H} steps, {nk} kernels")
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(st):
        a.record(st)
        for r in range(reps):
            for i in range(len(models)):
                zbuf[i].copy_(zall[i][1 + r * H: 1 + (r + 1) * H])
            grp.launch()
        b.record(st)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b)
    gt = grp.graph_times()  # H x batches, the last timed launch
    lat = np.concatenate([np.repeat(gt[:, i], filters[i].batch) for i in range(len(filters))])
    nf = sum(f.batch for f in filters)
    mean_ok = all(bool(torch.isfinite(o[0]).all()) for o in outs)
    grp.free()
    for f in filters:
        f.free()
    return {"value": nf * reps * H / (ms * 1e-3), "unit": UNIT, "filters": nf, "groups": len(groups),
            "steps": reps * H, "graph_horizon": H, "graph_launches": reps, "kernels_per_graph": nk,
            "ms_per_step": ms / (reps * H), "estimates_finite": mean_ok,
            "eager_group_step_s": t_eager,
            "per_filter_step_ms": {"p50": float(np.percentile(lat, 50)),
                                   "p99": float(np.percentile(lat, 99)),
                                   "source": "global-timer stamps recorded in the graph, last timed launch"},
            "autotuned_groups": tuned,
            "workload": "config4: 512 filters, d in {3..6}, N in {64,128,256}, rank cap in "
                        "{8,16,32}, random stable F (rho 0.9), diagonal Q, R, range measurement"}


def run_adjoint(args, dev):
    """Config 5: the gradient of the log-likelihood (sum of log c over the run)
    of one config-2 filter over 200 steps with respect to F, diag Q and
    diag R, through the torch function over the reverse pass (checkpoints
    every 20 steps, each segment recomputed and recorded once in the backward
    pass).  Times the forward and the backward call with CUDA events on the
    filter's stream (wall-clock synchronised around each)."""
    log("gradient (config 5) leg")
    import torch
    import paper_2501_07942_gb300 as G
    model = synth.config2()
    K, every = args.adj_steps, 20
    # the first Monte Carlo run whose trajectory stays inside |x_m| < 6 for
    # all K steps (the grid is [-8, 8]^4; run 0 leaves it after about 60 steps)
    mc = next((s for s in range(100) if np.abs(synth.simulate(model, s, steps=K)[0]).max() < 6.0), 0)
    z = synth.simulate(model, mc, steps=K)[1]
    probe = G.TTFilter(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), batch=1,
                       rank_cap=model.rank_cap, eps=model.eps, device=dev)
    comps = [(m, torch.tensor(np.asarray(t), dtype=torch.float32, device=dev))
             for m, t in model.tables(probe.grid_axes())]
    probe.free()
    zd = torch.tensor(z[:, None, :], dtype=torch.float32, device=dev)  # K x 1 x b
    Ft = torch.tensor(model.F, dtype=torch.float64, requires_grad=True)
    qt = torch.tensor(np.diag(model.Q).copy(), dtype=torch.float64, requires_grad=True)
    rt = torch.tensor(np.diag(np.atleast_2d(model.R)).copy(), dtype=torch.float64, requires_grad=True)
    torch.cuda.synchronize(dev)
    t0 = time.time()
    ll = G.log_likelihood(Ft, qt, rt, lo=model.lo, hi=model.hi, n=model.n, prior_mean=model.m0,
                          prior_var=np.diag(model.P0), comps=comps, z=zd, rank_cap=model.rank_cap,
                          eps=model.eps, max_shift_span=10, checkpoint_every=every, device=dev)
    torch.cuda.synchronize(dev)
    t1 = time.time()
    ll.sum().backward()
    torch.cuda.synchronize(dev)
    t2 = time.time()
    g = np.concatenate([Ft.grad.numpy().ravel(), qt.grad.numpy(), rt.grad.numpy()])
    return {"workload": f"config5: config-2 model, 1 filter (Monte Carlo run {mc}: the first whose "
                        f"trajectory stays within 6 of the origin on every axis), {K} steps, "
                        f"checkpoints every {every} steps",
            "log_lik": float(ll.detach().numpy()[0]), "forward_s": t1 - t0, "backward_s": t2 - t1,
            "backward_ms_per_step": 1e3 * (t2 - t1) / K,
            "gradient_finite": bool(np.isfinite(g).all()), "grad_max_abs": float(np.abs(g).max()),
            "dl_dF": Ft.grad.numpy().round(6).tolist(), "dl_dq": qt.grad.numpy().round(6).tolist(),
            "dl_dr": rt.grad.numpy().round(6).tolist(),
            "checked": "against the float64 dense oracle gradient and central differences at 32^4 "
                       "(tests/test_gpu_adjoint.py)"}


def run_grid_design(args, dev):
    """Alg. 4 grid re-design against the fixed grid: config 2's model, Monte
    Carlo run 0 over 200 steps (its trajectory leaves [-8, 8]^4 after about 60
    steps and reaches |x| = 19), one filter each: fixed grid, and the grid
    re-designed after every update from the posterior moments (kappa = 5).
    Reports each filter's log-likelihood, the RMS error of its mean against
    the true state over the last 50 steps and its time per step (re-design and
    interpolation included)."""
    import torch
    import paper_2501_07942_gb300 as G
    log("grid re-design leg")
    model = synth.config2()
    K = 200
    x, z = synth.simulate(model, 0, steps=K)
    out = {}
    for name in ("fixed", "redesigned"):
        f = G.TTFilter(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), batch=1,
                       rank_cap=model.rank_cap, eps=model.eps, device=dev)
        comps = [(m, torch.tensor(np.asarray(t), dtype=torch.float32, device=dev))
                 for m, t in model.tables(f.grid_axes())]
        errs = []
        torch.cuda.synchronize(dev)
        t0 = time.time()
        for k in range(K):
            if name == "redesigned" and k > 0:
                comps = [(m, torch.tensor(np.asarray(t), dtype=torch.float32, device=dev))
                         for m, t in model.tables(f.grid_axes())]
            f.predict(model.F, model.Q)
            f.update(comps, model.R, z[k][None, :])
            mean, cov, lc, ll = f.estimate()
            errs.append(mean[0] - x[k + 1])
            if name == "redesigned":
                lo, hi = G.design_grid(model.F, model.Q, mean, cov, kappa=5.0)
                f.regrid(lo, hi)
        torch.cuda.synchronize(dev)
        dt = time.time() - t0
        e = np.array(errs[K // 2:])
        out[name] = {"log_lik": float(ll[0]), "rmse_last_50": float(np.sqrt((e ** 2).mean())),
                     "ms_per_step": 1e3 * dt / K}
        f.free()
    out["workload"] = ("config-2 model, Monte Carlo run 0, 200 steps, 1 filter; grid re-designed after "
                       "every update (Alg. 4, kappa 5) vs the fixed [-8, 8]^4 grid; wall clock per step "
                       "including the host's moments, design and measurement tables")
    return out


def run_cross(args, dev):
    """Likelihood factors on three modes by the deterministic TT cross: the
    range3 workload (config 2's grid, prior, F and Q with z = ||x[0:3]|| + v,
    R = 0.02), 128^4, 100 filters, rank cap 16, cross rank 24 with one
    refinement sweep.  Times predict + update + estimate per step (L2 flushed
    before each timed step, CUDA events on the filter's stream), the share of
    each kernel class (library profiling, on further steps), the float32
    full-grid filter on the same measurement (one filter), and the TT
    density's relative Frobenius error against the float64 full-grid filter
    on Monte Carlo run 0 after every step."""
    import torch
    import paper_2501_07942_gb300 as G
    log("cross leg (likelihood on three modes)")
    model = synth.range3()
    B, W, K = args.cross_batch, 3, args.cross_steps
    cap, smax, S = model.rank_cap, 10, 24
    zs = measurement_batches(model, list(range(B)), W + 2 * K)
    kw = tuned_config(G, model, B, cap, smax, "fp32")
    f = G.TTFilter(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), batch=B, rank_cap=cap,
                   eps=model.eps, max_shift_span=smax, device=dev, cross_rank=S, **kw)
    axes = f.grid_axes()
    comps = [(m, torch.tensor(np.asarray(t), dtype=torch.float32, device=dev))
             for m, t, *_ in model.tables(axes)]
    z_dev = torch.tensor(zs, dtype=torch.float32, device=dev)
    d = model.d
    mean = torch.zeros(B, d, dtype=torch.float64, device=dev)
    cov = torch.zeros(B, d, d, dtype=torch.float64, device=dev)
    lc = torch.zeros(B, dtype=torch.float64, device=dev)
    ll = torch.zeros(B, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(flt, k):
        flt.predict(model.F, model.Q)
        flt.update_dev(comps, model.R, z_dev[k])
        flt.estimate_dev(mean, cov, lc, ll)

    for k in range(W):
        step(f, k)
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for i in range(K):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        step(f, W + i)
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    ms = sum(a.elapsed_time(b) for a, b in ev)
    f.profile(True)
    for i in range(K):
        flush.fill_(i & 0xFF)
        step(f, W + K + i)
    torch.cuda.synchronize(dev)
    prof = f.profile_read()
    f.profile(False)
    f.free()
    del f
    torch.cuda.empty_cache()
    tot = sum(v["ms"] for v in prof.values()) or 1.0
    out = {"workload": "range3: config-2 grid, prior, F, Q; z = ||x[0:3]|| + v, R = 0.02; 128^4, "
                       f"{B} filters, rank cap {cap}, cross rank {S}, 1 refinement sweep",
           "value": B * K / (ms * 1e-3), "unit": "filter-steps/s", "ms_per_step": ms / K,
           "kernels": {k: {"ms_share": v["ms"] / tot, "launches": v["launches"]} for k, v in prof.items()
                       if v["launches"]},
           "cross_ms_per_step": prof.get("cross", {}).get("ms", 0.0) / K}
    log("cross leg: full-grid comparison")
    if args.cross_no_compare:
        return out
    out["fullgrid"] = run_fullgrid(args, model, zs, W, K, dev, axes)
    # accuracy: Monte Carlo run 0 against the float64 full-grid filter, at the
    # leg's rank cap and at rank cap 32 (span 5, cross rank 40)
    runs = [(cap, smax, S), (32, 5, 40)]
    tts = [G.TTFilter(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), batch=1, rank_cap=c,
                      eps=model.eps, max_shift_span=sp, device=dev, cross_rank=sr) for c, sp, sr in runs]
    errs = [[] for _ in runs]
    for k, P in enumerate(fp64_reference_densities(model, zs, W + K, dev, axes)):
        for f0, e in zip(tts, errs):
            f0.predict(model.F, model.Q)
            f0.update(comps, model.R, zs[k][0][None, :])
            e.append(tt_dense_rel_err(f0.export_cores(0), P))
    for f0 in tts:
        f0.free()
    out["tt_density_rel_fro_err"] = errs[0]
    out["tt_density_rel_fro_err_rank_cap_32"] = errs[1]
    return out


def tt_pairs_rel_err(cores, pairs) -> float:
    """||T - P_0 (x) P_1 (x) ...||_F / ||P_0 (x) P_1 (x) ...||_F of a TT over
    d = 2 len(pairs) modes and dense 2-D densities P_i over the modes
    (2i, 2i + 1), from inner products (the d-dimensional tensors are never
    formed)."""
    cores = [np.asarray(c, dtype=np.float64) for c in cores]
    E = np.ones((1, 1))
    for C in cores:
        E = np.einsum("ab,aic,bid->cd", E, C, C)
    tt2 = float(E[0, 0])
    v = np.ones((1,))
    pp = 1.0
    for i, P in enumerate(pairs):
        M = np.einsum("ajc,jk,ckd->ad", cores[2 * i], P, cores[2 * i + 1])
        v = v @ M
        pp *= float(np.vdot(P, P))
    tp = float(v.reshape(-1)[0])
    return math.sqrt(max(tt2 - 2.0 * tp + pp, 0.0) / pp)


def run_config3(args, dev):
    """Config 3 (d = 6 constant-velocity pairs x_{2i} += 0.1 x_{2i+1}, N = 256,
    rank cap 32, eps 1e-5, one-mode measurements x_{2i}^2 / 20) with both
    transitions: the re-gridded one (ttgbf_predict: hat shears in pieces,
    Gaussian kernel) and the textbook one (ttgbf_predict_exact: each pair's
    coupled factor on its 2-site block by the cross, rank 40), each with the
    core contractions on the CUDA cores (float32) and on the tensor cores
    (TF32; split TF32 for the re-gridded one).  Throughput of
    predict + update + estimate for a batch (L2 flushed before each timed
    step, CUDA events).  Accuracy at N = 128 (the full-grid filter's largest
    axis), Monte Carlo run 0: the TT density against the tensor product of
    the three pairs' float64 full-grid filters with the textbook direct sum
    (and with the re-gridded transition for the re-gridded TT filter's own
    operator), per step."""
    import torch
    import paper_2501_07942_gb300 as G
    log("config-3 leg (re-gridded and textbook transitions)")
    out = {"workload": "config3: d=6, N=256, F block-diagonal [[1, 0.1], [0, 1]], diagonal Q, "
                       "z_i = x_{2i}^2 / 20 + v_i, R = 0.02 I, rank cap 32, eps 1e-5; "
                       f"{args.c3_batch} filters"}
    model = synth.config3(d=6, n=256)
    B, W, K = args.c3_batch, 2, args.c3_steps
    zs = measurement_batches(model, list(range(B)), W + K)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for name, exact, con in C3_VARIANTS:
        f = G.TTFilter(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), batch=B,
                       rank_cap=model.rank_cap, eps=model.eps, max_shift_span=5, device=dev,
                       cross_rank=model.rank_cap + 8 if exact else 0, contraction=con)
        comps = [(m, torch.tensor(np.asarray(t), dtype=torch.float32, device=dev))
                 for m, t, *_ in model.tables(f.grid_axes())]
        z_dev = torch.tensor(zs, dtype=torch.float32, device=dev)

        def step(k):
            if exact:
                f.predict_exact(model.F, model.Q)
            else:
                f.predict(model.F, model.Q)
            f.update_dev(comps, model.R, z_dev[k])
            f.estimate()

        for k in range(W):
            step(k)
        torch.cuda.synchronize(dev)
        ms = 0.0
        for i in range(K):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(W + i)
            b.record(stream)
            torch.cuda.synchronize(dev)
            ms += a.elapsed_time(b)
        out[name] = {"value": B * K / (ms * 1e-3), "unit": "filter-steps/s", "ms_per_step": ms / K,
                     "max_rank": int(f.ranks().max()), "contraction": con}
        f.free()
        del f
        torch.cuda.empty_cache()
    # accuracy at N = 128 against the pairs' float64 full-grid filters
    m128 = synth.config3(d=6, n=128)
    S = args.c3_acc_steps
    z0 = synth.simulate(m128, 0, steps=S)[1]
    npair = m128.d // 2
    acc = {}
    refs = {}
    for ref_name, direct in (("textbook", True), ("regridded", False)):
        dens = [[None] * npair for _ in range(S)]
        for i in range(npair):
            sl = slice(2 * i, 2 * i + 2)
            fg = G.FullGridFilter(m128.lo[sl], m128.hi[sl], m128.n[sl], m128.m0[sl], np.diag(m128.P0)[sl],
                                  precision=64, device=dev)
            ax = [np.asarray(a) for a in fg_axes(m128.lo[sl], m128.hi[sl], m128.n[sl])]
            tab = [((0,), torch.tensor(synth.workloads.h_square20(ax[0]), dtype=torch.float64, device=dev))]
            for k in range(S):
                if direct:
                    fg.predict_direct(m128.F[sl, sl], m128.Q[sl, sl])
                else:
                    fg.predict(m128.F[sl, sl], m128.Q[sl, sl])
                fg.update(tab, m128.R[i:i + 1, i:i + 1], z0[k][i:i + 1])
                dens[k][i] = fg.density()
            fg.free()
        refs[ref_name] = dens
    for name, exact, con in C3_VARIANTS:
        f = G.TTFilter(m128.lo, m128.hi, m128.n, m128.m0, np.diag(m128.P0), batch=1, rank_cap=m128.rank_cap,
                       eps=m128.eps, max_shift_span=5, device=dev, cross_rank=m128.rank_cap + 8 if exact else 0,
                       contraction=con)
        comps = [(m, torch.tensor(np.asarray(t), dtype=torch.float32, device=dev))
                 for m, t, *_ in m128.tables(f.grid_axes())]
        e_text, e_rg = [], []
        for k in range(S):
            if exact:
                f.predict_exact(m128.F, m128.Q)
            else:
                f.predict(m128.F, m128.Q)
            f.update(comps, m128.R, z0[k][None, :])
            cores = f.export_cores(0)
            e_text.append(tt_pairs_rel_err(cores, refs["textbook"][k]))
            e_rg.append(tt_pairs_rel_err(cores, refs["regridded"][k]))
        f.free()
        acc[name] = {"vs_textbook_full_grid": e_text, "vs_regridded_full_grid": e_rg}
    out["accuracy_n128"] = acc
    out["accuracy_reference"] = ("Monte Carlo run 0 at N = 128: the tensor product of the three pairs' float64 "
                                 "full-grid GPU filters, with the textbook direct sum (ttgbf_fg_predict_direct) "
                                 "or the re-gridded transition (ttgbf_fg_predict); relative Frobenius error per "
                                 "step")
    return out


# config-3 variants: (name, textbook transition, contraction arithmetic)
C3_VARIANTS = [("regridded", False, "fp32"), ("regridded_tf32x3", False, "tf32x3"),
               ("regridded_tf32", False, "tf32"), ("textbook", True, "fp32"), ("textbook_tf32", True, "tf32")]


def fg_axes(lo, hi, n):
    """Cell-centred axes of a grid (the library's and the oracle's reading)."""
    return [lo[m] + (np.arange(n[m]) + 0.5) * (hi[m] - lo[m]) / n[m] for m in range(len(n))]


def run_leg(name, args):
    """Run one secondary leg (config4, adjoint) in a child process of its own:
    its device memory (66 GB for config 4) is returned when it exits, and a
    failure there costs that leg only.  Returns the leg's dict, or the error."""
    cmd = [sys.executable, os.path.abspath(__file__), "--leg", name, "--c4-horizon", str(args.c4_horizon),
           "--c4-steps", str(args.c4_steps), "--adj-steps", str(args.adj_steps),
           "--cross-steps", str(args.cross_steps), "--cross-batch", str(args.cross_batch),
           "--c3-batch", str(args.c3_batch), "--c3-steps", str(args.c3_steps),
           "--c3-acc-steps", str(args.c3_acc_steps)]
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    try:
        res = subprocess.run(cmd, capture_output=True, text=True, timeout=1200, env=env)
    except subprocess.TimeoutExpired:
        return {"error": "timed out after 1200 s"}
    sys.stderr.write(res.stderr)
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    if res.returncode != 0 or not lines:
        tail = res.stderr.strip().splitlines()[-1:] or [""]
        return {"error": f"exit {res.returncode}: {tail[0][:300]}"}
    return json.loads(lines[-1])


def tuned_config(G, model, batch, rank_cap, smax, precision):
    """The autotuner's persisted launch configuration for this shape ({} when
    the cache has none: the library's defaults)."""
    if not os.path.exists(TUNE_CACHE):
        return {}
    try:
        best, _ = G.autotune(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), model.F, model.Q,
                             batch=batch, rank_cap=rank_cap, eps=model.eps, max_shift_span=smax,
                             precision=precision, cache_path=TUNE_CACHE, cache_only=True)
        return best
    except LookupError:
        return {}


def make_tt(G, model, dev, batch, rank_cap, smax, precision, parts=None, contraction="fp32"):
    """A TT filter context with the autotuned launch configuration of its shape;
    parts overrides the batch split for this context only."""
    kw = tuned_config(G, model, batch, rank_cap, smax, precision)
    if parts is not None:
        kw["parts"] = parts
    return G.TTFilter(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), batch=batch,
                      rank_cap=rank_cap, eps=model.eps, max_shift_span=smax, device=dev,
                      precision=precision, contraction=contraction, **kw)


def run_ours(args, rank: int, world: int, local_rank: int, dist):
    import torch
    import paper_2501_07942_gb300 as G
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    model = synth.config2()
    B = args.batch
    W, K = args.warmup, args.steps
    cap, smax, prec, con = args.rank_cap, args.max_shift_span, args.precision, args.contraction
    mc_ids = shard_mc_ids(rank, world, B)
    zs = measurement_batches(model, mc_ids, W + 3 * K)
    f = make_tt(G, model, dev, B, cap, smax, prec, contraction=con)
    axes = f.grid_axes()
    comps = [(m, torch.tensor(np.asarray(t), dtype=torch.float32, device=dev))
             for m, t in model.tables(axes)]
    z_dev = torch.tensor(zs, dtype=torch.float32, device=dev)
    d = model.d
    mean = torch.zeros(B, d, dtype=torch.float64, device=dev)
    cov = torch.zeros(B, d, d, dtype=torch.float64, device=dev)
    lc = torch.zeros(B, dtype=torch.float64, device=dev)
    ll = torch.zeros(B, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(flt, k):
        flt.predict(model.F, model.Q)
        flt.update_dev(comps, model.R, z_dev[k])
        flt.estimate_dev(mean, cov, lc, ll)

    def timed(flt, k0, n):
        """n steps from measurement k0, L2 flushed before each, CUDA events on
        the caller's stream; returns the summed milliseconds."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(n)]
        for i in range(n):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            step(flt, k0 + i)
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        return sum(a.elapsed_time(b) for a, b in ev)

    for k in range(W):
        step(f, k)
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    l0 = G.launch_count()
    if args.profile_region:
        torch.cuda.profiler.start()
    ms = timed(f, W, K)
    if args.profile_region:
        torch.cuda.profiler.stop()
    launches = G.launch_count() - l0
    clk = clocks.stop()
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()

    # per-kernel-class shares of the timed configuration: K more steps with
    # the library's event profiling on (kept out of the timed steps above,
    # whose value it would lower by the cost of its event records)
    torch.cuda.synchronize(dev)
    f.profile(True)
    for i in range(K):
        flush.fill_(i & 0xFF)
        step(f, W + K + i)
    torch.cuda.synchronize(dev)
    prof = f.profile_read()
    f.profile(False)

    # end to end through the host-buffer C calls: z from host memory every
    # step, mean / cov / log normaliser read back to the host every step
    e2e_s = 0.0
    for i in range(K):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        f.predict(model.F, model.Q)
        f.update(comps, model.R, zs[W + 2 * K + i])
        f.estimate()
        e2e_s += time.perf_counter() - t0
    if dist is not None:
        t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    f.free()
    del f
    torch.cuda.empty_cache()
    if rank != 0:
        return

    # the dominant kernel's roofline: the same workload as ONE part on one
    # stream, so every event interval of the library's profiling brackets
    # that kernel alone (no concurrent parts sharing the SMs)
    pk, pk_src = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = nsm * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s, FP32 FMA lanes at max clock
    f1 = make_tt(G, model, dev, B, cap, smax, prec, parts=1, contraction=con)
    for k in range(W):
        step(f1, k)
    torch.cuda.synchronize(dev)
    f1.profile(True)
    for i in range(K):
        flush.fill_(i & 0xFF)
        step(f1, W + i)
    torch.cuda.synchronize(dev)
    prof1 = f1.profile_read()
    f1.free()
    del f1
    torch.cuda.empty_cache()
    tsqr = prof1["tsqr"]
    alg = tsqr_algorithmic_flops(model, cap) * B * K  # over the K profiled steps
    achieved = alg / (tsqr["ms"] * 1e-3) / 1e12 if tsqr["ms"] > 0 else 0.0
    per_step = tsqr["launches"] / K  # k_tsqr launches per step of the one-part context
    # the captured traffic applies to the workload it was taken on: config 2 at rank cap 16
    traffic = (TSQR_DRAM_BYTES_PER_FILTER_STEP * B / per_step
               if cap == 16 and con == "fp32" and prec == "fp32" and per_step > 0 else None)
    roofline = {"bound": "alu", "kernel": "k_tsqr", "achieved": achieved, "peak": fp32_peak,
                "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": traffic,
                "traffic_note": "bytes per launch: one ncu capture of a 12-filter step's k_tsqr launches "
                                "(dram__bytes_read.sum + dram__bytes_write.sum) scaled by the filters per "
                                "launch; a lower bound (L2 holds more of a 12-filter part)",
                "algorithmic_bytes_per_launch": tsqr_algorithmic_bytes(model, cap) * B / max(per_step, 1),
                "algorithmic_flops_per_filter_step": tsqr_algorithmic_flops(model, cap),
                "launches": tsqr["launches"], "ms_per_launch": tsqr["ms"] / max(tsqr["launches"], 1),
                "measured": f"{B} filters as one part on one stream, CUDA events around every "
                            "k_tsqr launch (library profiling), K steps",
                "peak_source": f"derived: {nsm} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz "
                               f"(clock from {pk_src} peaks); of derived peak"}

    # the core contractions on the tensor cores (tcgen05 kind::tf32, split
    # TF32): the same single-part profile, the grouped GEMM's flops (2 m n k
    # per tile, each of the three split products counted once: the
    # algorithmic product) over its event time, against the TF32 peak
    log("tensor-core contraction profile")
    ftc = make_tt(G, model, dev, B, cap, smax, prec, parts=1, contraction="tf32x3")
    for k in range(W):
        step(ftc, k)
    torch.cuda.synchronize(dev)
    ftc.profile(True)
    for i in range(K):
        flush.fill_(i & 0xFF)
        step(ftc, W + i)
    torch.cuda.synchronize(dev)
    gtc = ftc.profile_read()["gemm"]
    ftc.free()
    del ftc
    torch.cuda.empty_cache()
    tf32_peak = float(pk.get("bf16_tflops", 1900.0)) * TF32_PER_BF16
    ach_tc = gtc["flops"] / (gtc["ms"] * 1e-3) / 1e12 if gtc["ms"] > 0 else 0.0
    gemm_tc = {"bound": "tensor", "kernel": "k_gemm_tc (tf32x3)", "achieved": ach_tc, "peak": tf32_peak,
               "unit": "TFLOP/s", "frac": ach_tc / tf32_peak, "tensor_flops_per_flop": 3,
               "launches": gtc["launches"], "ms_per_launch": gtc["ms"] / max(gtc["launches"], 1),
               "measured": f"{B} filters as one part on one stream, CUDA events around every grouped "
                           "GEMM launch, K steps",
               "peak_source": f"{pk_src} bf16 burst x {TF32_PER_BF16:.3f} (nominal TF32 : BF16); of "
                              f"{pk_src} (scaled)"}

    # the full-grid filter on the same workload (the metric's comparison)
    log("full-grid leg")
    fullgrid = None if args.no_fullgrid else run_fullgrid(args, model, zs, W, K, dev, axes)

    # accuracy at the bench configuration and a rank-cap sweep: every TT
    # configuration runs W + K steps from the prior on the batch's
    # measurements; filter 0 (Monte Carlo run 0) is compared with the float64
    # full-grid GPU filter of that run after every step
    accuracy, sweep = None, []
    if not args.no_accuracy:
        log("accuracy leg and rank-cap sweep")
        S = W + K
        bound = 10.0 * model.eps + 1e-5
        configs = [(cap, smax, prec, con)] + [c for c in SWEEP if c != (cap, smax, prec, con)]
        runs = []
        for (rc, sp, pr, cn) in configs:
            g = make_tt(G, model, dev, B, rc, sp, pr, contraction=cn)
            runs.append({"cfg": (rc, sp, pr, cn), "f": g, "ms": 0.0, "err": []})
        for k, P in enumerate(fp64_reference_densities(model, zs, S, dev, axes)):
            for r in runs:
                g = r["f"]
                if k >= W:
                    r["ms"] += timed(g, k, 1)
                else:
                    step(g, k)
                torch.cuda.synchronize(dev)
                if k == S - 1 or r is runs[0]:
                    r["err"].append(tt_dense_rel_err(g.export_cores(0), P))
        main_errs = list(runs[0]["err"])
        for r in runs:
            rc, sp, pr, cn = r["cfg"]
            r["f"].free()
            ent = {"rank_cap": rc, "max_shift_span": sp, "precision": pr, "contraction": cn,
                   "value": B * K / (r["ms"] * 1e-3), "unit": UNIT, "ms_per_step": r["ms"] / K,
                   "tt_density_rel_fro_err": r["err"][-1], "bound": bound,
                   "matched": r["err"][-1] <= bound}
            if fullgrid is not None:
                ent["vs_fullgrid"] = ent["value"] / fullgrid["value"]
            sweep.append(ent)
        runs.clear()
        torch.cuda.empty_cache()
        accuracy = {"reference": "float64 full-grid GPU filter (ttgbf_fg, precision 64), Monte "
                                 "Carlo run 0, same measurements",
                    "steps": S, "per_step_rel_fro_err": main_errs, "bound": bound,
                    "tt_density_rel_fro_err": sweep[0]["tt_density_rel_fro_err"],
                    "matched": sweep[0]["matched"]}
    value = B * world * K / (ms * 1e-3)
    b = model.b
    tot_ms = sum(v["ms"] for v in prof.values())
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD.replace("rank cap 16", f"rank cap {cap}"),
                   "rounding_precision": prec, "contraction": con, "max_shift_span": smax,
                   "launch_config": tuned_config(G, model, B, cap, smax, prec) or "library defaults",
                   "filters_per_gpu": B, "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"replicas x{world} (independent filters, no collective)"},
        "roofline": roofline,
        "gemm_tc": gemm_tc,
        "e2e": {"value": B * world * K / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": B * b * 4, "d2h_bytes_per_step": B * (d + d * d + 2) * 8},
        "gpu_launches": launches,
        "clocks": clk,
        "kernels": {k: {"ms_share": (v["ms"] / tot_ms if tot_ms else 0.0), "launches": v["launches"]}
                    for k, v in prof.items() if v["launches"] > 0},
        "fullgrid": fullgrid,
        "config4": None if args.no_config4 or rank != 0 else run_leg("config4", args),
        "adjoint": None if args.no_adjoint or rank != 0 else run_leg("adjoint", args),
        "cross": None if args.no_cross or rank != 0 else run_leg("cross", args),
        "config3": None if args.no_config3 or rank != 0 else run_leg("config3", args),
        "grid_design": None if args.no_grid_design or rank != 0 else run_grid_design(args, dev),
        "accuracy": accuracy,
        "rank_cap_sweep": sweep,
    }
    if accuracy is not None:
        ok = [e for e in sweep if e["matched"]]
        best = min(ok, key=lambda e: e["ms_per_step"]) if ok else min(
            sweep, key=lambda e: e["tt_density_rel_fro_err"])
        line["matched_error"] = {
            "met": bool(ok),
            "config": {k: best[k] for k in ("rank_cap", "max_shift_span", "precision", "contraction")},
            "value": best["value"], "tt_density_rel_fro_err": best["tt_density_rel_fro_err"],
            "bound": best["bound"], "vs_fullgrid": best.get("vs_fullgrid")}
    if world == 1 and not args.no_cpu_baseline:
        log("cpu baseline (oracle)")
        dt, desc = cpu_oracle_step(model, mc_ids[0])
        line["cpu_baseline"] = {"value": 1.0 / dt, "unit": UNIT, "cores": os.cpu_count(),
                                "kind": "oracle", "sample": desc}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--batch", type=int, default=100)
    ap.add_argument("--rank-cap", type=int, default=16)
    ap.add_argument("--max-shift-span", type=int, default=10)
    ap.add_argument("--contraction", choices=["fp32", "tf32", "tf32x3"], default="fp32",
                    help="arithmetic of the core contractions (CUDA cores or tcgen05 tensor cores)")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32",
                    help="arithmetic of the truncating R factors and SVDs (ttgbf_opts.precision)")
    ap.add_argument("--no-config4", action="store_true", help="skip the uneven-batch leg")
    ap.add_argument("--c4-horizon", type=int, default=10,
                    help="steps recorded into one CUDA graph in the uneven-batch leg (even)")
    ap.add_argument("--c4-steps", type=int, default=10,
                    help="timed steps of the uneven-batch leg (graph launches x horizon)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the gradient (config 5) leg")
    ap.add_argument("--no-grid-design", action="store_true", help="skip the grid re-design leg")
    ap.add_argument("--no-cross", action="store_true", help="skip the three-mode likelihood (TT cross) leg")
    ap.add_argument("--no-config3", action="store_true", help="skip the config-3 (two transitions) leg")
    ap.add_argument("--c3-batch", type=int, default=32, help="filters of the config-3 leg")
    ap.add_argument("--c3-steps", type=int, default=3, help="timed steps of the config-3 leg")
    ap.add_argument("--c3-acc-steps", type=int, default=5, help="accuracy steps of the config-3 leg")
    ap.add_argument("--cross-steps", type=int, default=10, help="timed steps of the TT cross leg")
    ap.add_argument("--cross-batch", type=int, default=100, help="filters of the TT cross leg")
    ap.add_argument("--cross-no-compare", action="store_true",
                    help="TT cross leg: skip the full-grid comparison and the accuracy run")
    ap.add_argument("--leg", choices=["config4", "adjoint", "cross", "config3"], default=None,
                    help="run only this secondary leg and print its result (used by the main run)")
    ap.add_argument("--adj-steps", type=int, default=200, help="steps of the gradient leg")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the accuracy comparison and the rank-cap sweep")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fullgrid", action="store_true")
    ap.add_argument("--profile-region", action="store_true",
                    help="bracket the timed TT steps with cudaProfilerStart/Stop (for ncu "
                         "--profile-from-start off; the run's own timings are then invalid)")
    ap.add_argument("--profile-fullgrid", action="store_true",
                    help="bracket the timed full-grid steps instead")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.leg is not None:
        import torch
        torch.cuda.set_device(0)
        legs = {"config4": run_config4, "adjoint": run_adjoint, "cross": run_cross, "config3": run_config3}
        out = legs[args.leg](args, "cuda:0")
        print(json.dumps(out), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as tdist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local_rank)
        tdist.init_process_group(backend)
        dist = tdist
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_ours(args, rank, world, local_rank, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
