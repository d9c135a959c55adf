"""Helpers shared by the GPU parity tests: build/load the library, move
measurement tables to the device, compare densities."""
import numpy as np

import synth
from oracle import pmf, tt

EPS_TOL_FLOOR = 1e-5  # FP32 arithmetic floor of the TT parity tolerance


def lib_module():
    import paper_2501_07942_gb300 as G
    from paper_2501_07942_gb300 import build
    build.build()
    G.load()
    return G


def rel(a, b) -> float:
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def tt_tol(eps: float, tail_sum: float) -> float:
    """Parity bound of the TT path against the dense oracle for one step:
    10 * (eps + tau) + 1e-5, tau the discarded relative tails of the ORACLE's
    TT filter (oracle/ttfilter.py) on the same input, never a tail the GPU
    reports about itself.  Where the rank cap does not bind, tau is at the
    eps level."""
    return 10.0 * (eps + tail_sum) + EPS_TOL_FLOOR


def cov_tol(delta_axis, cov):
    """Covariance tolerance matching the 1e-3 grid-spacing bound on the mean:
    a first-moment error of 1e-3 D_i moves E[x_i x_j] by about
    1e-3 (D_i sigma_j + D_j sigma_i), sigma from the oracle's diagonal."""
    D = np.asarray(delta_axis, dtype=np.float64)
    sig = np.sqrt(np.maximum(np.diag(cov), 0.0))
    return 1e-3 * (D[:, None] * sig[None, :] + sig[:, None] * D[None, :])


def mean_tol(delta_axis, cov, tail_acc):
    """Posterior-mean tolerance per mode against the DENSE oracle: 1e-3 grid
    spacings, plus 2 tau sigma_m for the truncation a TT of capped rank must
    make: tau = the ORACLE TT filter's discarded relative tails summed over
    the steps so far (a relative L2 change tau of the density moves the mean
    of mode m by about tau sigma_m, sigma_m the oracle's marginal standard
    deviation).  Against the oracle's own TT filter the bound is the flat
    1e-3 grid spacings."""
    D = np.asarray(delta_axis, dtype=np.float64)
    sig = np.sqrt(np.maximum(np.diag(cov), 0.0))
    return 1e-3 * D + 2.0 * tail_acc * sig


def oracle_tt_prior(model):
    """The model's diagonal Gaussian prior as rank-1 float64 cores (the
    oracle TT filter's starting point), normalised."""
    g = pmf.Grid(model.lo, model.hi, model.n)
    var = np.diag(model.P0)
    cores = [np.exp(-0.5 * (g.axes[m] - model.m0[m]) ** 2 / var[m]).reshape(1, -1, 1)
             for m in range(g.d)]
    cores[-1] = cores[-1] / (tt.full_sum(cores) * g.delta)
    return cores


def device_tables(model: synth.Model, axes):
    import torch
    return [(m, torch.tensor(np.asarray(t), dtype=torch.float32, device="cuda"), *period)
            for m, t, *period in model.tables(axes)]


def make_filter(G, model: synth.Model, batch=1, rank_cap=None, eps=None, smax=0):
    return G.TTFilter(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), batch=batch,
                      rank_cap=model.rank_cap if rank_cap is None else rank_cap,
                      eps=model.eps if eps is None else eps, max_shift_span=smax)


def densify_filter(f, b=0):
    return tt.densify(f.export_cores(b))


def oracle_grid(model):
    return pmf.Grid(model.lo, model.hi, model.n)


def bearing_cut_model(n=(20, 18)):
    """Range and bearing (an angle of period 360) of an object near the
    negative x axis, on a fixed grid across it, so that the bearing's residual
    switches branch inside the grid (the same numbers as the oracle gradient's
    bearing pin).  Returns (model, measurements (3, 2))."""
    comps = [((0, 1), synth.workloads.h_range), ((0, 1), synth.workloads.h_bearing_deg, 360.0)]
    m = synth.Model(name="bearing-cut", lo=np.array([-15.0, -5.0]), hi=np.array([-5.0, 5.0]),
                    n=np.array(n), m0=np.array([-10.0, 0.0]), P0=2.0 * np.eye(2),
                    F=np.array([[0.96, 0.05], [-0.04, 0.97]]), Q=np.diag([0.3, 0.25]),
                    R=np.diag([0.5, 9.0]), comps=comps, eps=1e-6, rank_cap=32)
    z = np.array([[9.6, 178.0], [9.3, -177.0], [9.0, 179.5]])
    return m, z
