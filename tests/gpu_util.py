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
    10 * (eps + discarded tail) + 1e-5 (the discarded tail is zero when the
    rank cap does not bind, and then the bound is 10 eps + 1e-5)."""
    return 10.0 * (eps + tail_sum) + EPS_TOL_FLOOR


def cov_tol(delta_axis, cov):
    """Covariance tolerance matching the 1e-3 grid-spacing bound on the mean:
    a first-moment error of 1e-3 D_i moves E[x_i x_j] by about
    1e-3 (D_i sigma_j + D_j sigma_i), sigma from the oracle's diagonal."""
    D = np.asarray(delta_axis, dtype=np.float64)
    sig = np.sqrt(np.maximum(np.diag(cov), 0.0))
    return 1e-3 * (D[:, None] * sig[None, :] + sig[:, None] * D[None, :])


def mean_tol(delta_axis, cov, tail_acc):
    """Posterior-mean tolerance per mode: 1e-3 grid spacings, plus, where
    the rounding discarded more than eps (the rank cap binds), 2 tau sigma_m:
    tau = the discarded relative tails summed over the steps so far bounds
    the truncation's relative L2 change of the density, which moves the
    mean of mode m by about tau times that marginal's standard deviation
    sigma_m (from the oracle's covariance).  Without cap hits tau is at the
    eps level and the bound is the plain 1e-3 grid spacings."""
    D = np.asarray(delta_axis, dtype=np.float64)
    sig = np.sqrt(np.maximum(np.diag(cov), 0.0))
    return 1e-3 * D + 2.0 * tail_acc * sig


def device_tables(model: synth.Model, axes):
    import torch
    return [(m, torch.tensor(np.asarray(t), dtype=torch.float32, device="cuda"))
            for m, t in model.tables(axes)]


def make_filter(G, model: synth.Model, batch=1, rank_cap=None, eps=None, smax=0):
    return G.TTFilter(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), batch=batch,
                      rank_cap=model.rank_cap if rank_cap is None else rank_cap,
                      eps=model.eps if eps is None else eps, max_shift_span=smax)


def densify_filter(f, b=0):
    return tt.densify(f.export_cores(b))


def oracle_grid(model):
    return pmf.Grid(model.lo, model.hi, model.n)
