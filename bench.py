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


def fullgrid_bytes_per_step(model) -> int:
    """Algorithmic HBM bytes of one dense float32 step: every pass reads and
    writes the density once (shears, per-axis operators, normalise, likelihood,
    normalise) or reads it (sums, moments)."""
    from oracle import pmf
    n_shear = sum(1 for op in pmf.elementary_ops(model.F) if op[0] == "shear")
    cells = int(np.prod(model.n))
    passes_rw = n_shear + model.d + 1 + 1 + 1   # shears, axis operators, scale, likelihood, scale
    passes_r = 1 + 1                            # mass sum, moments
    return cells * 4 * (2 * passes_rw + passes_r)


def run_fullgrid(args, model, mc, zs, W, K, dev, ttf):
    """The plain full-grid float32 filter on the same workload (one Monte Carlo
    run, the batch's first): steps/s, achieved HBM bandwidth, and the density
    error of the TT filter of that run against it after the same steps."""
    import torch
    import paper_2501_07942_gb300 as G
    from oracle import tt
    fg = G.FullGridFilter(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), precision=32,
                          device=dev)
    comps = [(m, torch.tensor(np.asarray(t), dtype=torch.float32, device=dev))
             for m, t in model.tables(ttf.grid_axes())]
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
    # the TT filter of the same run after the same W + K steps
    if not args.no_tt_error:
        P = fg.density()
        T = tt.densify(ttf.export_cores(0))
        out["tt_density_rel_fro_err"] = float(np.linalg.norm(T - P) / np.linalg.norm(P))
    fg.free()
    return out


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


def run_ours(args, rank: int, world: int, local_rank: int, dist):
    import torch
    import paper_2501_07942_gb300 as G
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    model = synth.config2()
    B = args.batch
    W, K = args.warmup, args.steps
    mc_ids = shard_mc_ids(rank, world, B)
    zs = measurement_batches(model, mc_ids, W + 3 * K)
    f = G.TTFilter(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), batch=B,
                   rank_cap=model.rank_cap, eps=model.eps, device=dev)
    comps = [(m, torch.tensor(np.asarray(t), dtype=torch.float32, device=dev))
             for m, t in model.tables(f.grid_axes())]
    z_dev = torch.tensor(zs, dtype=torch.float32, device=dev)
    d = model.d
    mean = torch.zeros(B, d, dtype=torch.float64, device=dev)
    cov = torch.zeros(B, d, d, dtype=torch.float64, device=dev)
    lc = torch.zeros(B, dtype=torch.float64, device=dev)
    ll = torch.zeros(B, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(k):
        f.predict(model.F, model.Q)
        f.update_dev(comps, model.R, z_dev[k])
        f.estimate_dev(mean, cov, lc, ll)

    for k in range(W):
        step(k)
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    l0 = G.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    if args.profile_region:
        torch.cuda.profiler.start()
    for i in range(K):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        step(W + i)
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    if args.profile_region:
        torch.cuda.profiler.stop()
    launches = G.launch_count() - l0
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()

    # the full-grid filter on the same run, compared at the same step count
    fullgrid = None if args.no_fullgrid else run_fullgrid(args, model, mc_ids[0], zs, W, K, dev, f)

    # per-kernel-class times and device-counted flops: K more steps with the
    # library's event profiling on (kept out of the timed steps above, whose
    # value it would lower by the cost of its event records)
    torch.cuda.synchronize(dev)
    f.profile(True)
    for i in range(K):
        flush.fill_(i & 0xFF)
        step(W + K + i)
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
    if rank != 0:
        return
    pk, pk_src = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = nsm * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s, FP32 FMA lanes at max clock
    tot_ms = sum(v["ms"] for v in prof.values())
    top = max(prof.items(), key=lambda kv: kv[1]["ms"])
    name, rec = top
    roofline = None
    if rec["flops"] > 0 and rec["ms"] > 0:
        achieved = rec["flops"] / (rec["ms"] * 1e-3) / 1e12
        roofline = {"bound": "alu", "kernel": name, "achieved": achieved, "peak": fp32_peak,
                    "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": None,
                    "peak_source": f"derived: {nsm} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz "
                                   f"(clock from {pk_src} peaks)"}
    value = B * world * K / (ms * 1e-3)
    b = model.b
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "filters_per_gpu": B, "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"replicas x{world} (independent filters, no collective)"},
        "roofline": roofline,
        "e2e": {"value": B * world * K / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": B * b * 4, "d2h_bytes_per_step": B * (d + d * d + 2) * 8},
        "gpu_launches": launches,
        "clocks": clk,
        "kernels": {k: {"ms_share": (v["ms"] / tot_ms if tot_ms else 0.0), "launches": v["launches"],
                        "tflops": (v["flops"] / (v["ms"] * 1e-3) / 1e12 if v["ms"] > 0 else 0.0)}
                    for k, v in prof.items() if v["launches"] > 0},
        "fullgrid": fullgrid,
    }
    if world == 1 and not args.no_cpu_baseline:
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
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fullgrid", action="store_true")
    ap.add_argument("--no-tt-error", action="store_true",
                    help="skip the TT density error against the full-grid filter")
    ap.add_argument("--profile-region", action="store_true",
                    help="bracket the timed TT steps with cudaProfilerStart/Stop (for ncu "
                         "--profile-from-start off; the run's own timings are then invalid)")
    ap.add_argument("--profile-fullgrid", action="store_true",
                    help="bracket the timed full-grid steps instead")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
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
