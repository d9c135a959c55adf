"""Run the launch-configuration autotuner (ttgbf_autotune) over the workloads
this repository benchmarks and persist the choices in tune_cache.txt next to
this file (one line per batch shape and GPU), where TTFilter users and the
benchmark look them up.

    python -m paper_2501_07942_gb300.tune [--steps 2] [--only config2|config4]
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, "tune_cache.txt")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--only", choices=["config2", "config4"], default=None)
    args = ap.parse_args()
    sys.path.insert(0, os.path.dirname(HERE))
    import paper_2501_07942_gb300 as G
    import synth
    work = []
    if args.only in (None, "config2"):
        m = synth.config2()
        work.append((m, 100, 10))
    if args.only in (None, "config4"):
        for m, ids in synth.config4():
            work.append((m, len(ids), min(10, 160 // m.rank_cap)))
    for m, B, smax in work:
        t0 = time.time()
        best, ms = G.autotune(m.lo, m.hi, m.n, m.m0, np.diag(m.P0), m.F, m.Q, batch=B,
                              rank_cap=m.rank_cap, eps=m.eps, max_shift_span=smax, steps=args.steps,
                              cache_path=CACHE)
        print(f"{m.name} batch {B}: {best} {ms:.3f} ms per predict ({time.time() - t0:.1f} s)",
              flush=True)


if __name__ == "__main__":
    main()
