"""Writes tests/golden/config1_oracle.json by calling only oracle/ (and the
seeded inputs of synth/).  Run: python tests/golden/make_golden.py

The fixture is a regression guard for the dense oracle on the config-1
workload (d=2, 64x64, 20 steps, MC run 0): posterior means, covariances and
log normalisers for the textbook direct-sum transition and for the re-gridded
transition."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import pmf  # noqa: E402


def main():
    model = synth.config1()
    x, z = synth.simulate(model, 0)
    g = pmf.Grid(model.lo, model.hi, model.n)
    out = {"workload": "config1 d=2 N=64 [-10,10]^2, h=[x1, sin x2], 20 steps, mc=0",
           "z": z.tolist()}
    for tr in ("textbook", "rg"):
        r = pmf.run_filter(g, model.m0, model.P0, model.F, model.Q, model.tables(g.axes),
                           model.R, z, transition=tr)
        out[tr] = {"means": r["means"].tolist(), "covs": r["covs"].tolist(),
                   "log_c": r["log_c"].tolist()}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config1_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
