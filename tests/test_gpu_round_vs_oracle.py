"""The GPU rounding's decisions against an independent source: the float64 TT
filter of oracle/ttfilter.py run on the same input.  No bound here uses a
discarded tail that the GPU reports about itself.

1. Rounding at the benchmark shapes (128^4, rank cap 16, eps 1e-6): the input
   is the oracle TT filter's own state after two steps, a shear expands it
   (S = 9 on an adjacent link, 5 and 7 on non-adjacent ones), the GPU rounds
   its expansion and the oracle rounds its own.  Per link the ranks are equal;
   the GPU's actual error against the unrounded TT is within 5 % (+ 1e-6,
   float32) of the oracle's, which is the optimal truncation of each link
   given the others; the tails the GPU reports match the oracle's; the cores
   left of the center are orthonormal where it matters (see the test).
   A link whose rank differs must be one where the oracle's own decision is
   at the threshold (rank_is_borderline with ETA): the cores are stored in
   float32, and the orthogonalisation of float32 data perturbs the singular
   values a truncation compares with eps ||A|| / sqrt(d - 1) by about
   u sqrt(n) ||A|| (u = 6e-8, n <= 160), a quarter of that threshold at
   eps = 1e-6; a cap that binds decides alone and must agree.
2. One predict and one update from a shared input (the oracle's state, in
   float32 on both sides), with the rank cap binding (128^4, cap 16; 32^4, cap
   8) and not binding (32^4, cap 32): equal ranks, matching tails, density
   within 10 (eps + tau) + 1e-5 of the oracle's TT with tau the ORACLE's
   tails, means within 1e-3 grid spacings of the oracle TT's, log c within
   LOGC_TOL (below).
3. Flat bounds where the cap leaves the truncations at the eps level: config
   2 at 32^4 and 64^4 with rank cap 53 (span 3; shears in pieces at 64^4)
   over 6 steps from the prior.  The oracle TT filter at the same cap stays
   within the flat bound of the dense oracle at every step (checked as the
   premise: its truncations, though they add up to more than the bound, do
   not move the density that far), so every GPU step is held against the
   dense oracle at the plain 10 eps + 1e-5 (not summed over steps) and means
   within 1e-3 grid spacings."""
import math

import numpy as np
import pytest

import synth
from oracle import pmf, tt
from oracle import ttfilter as T

from gpu_util import cov_tol, device_tables, lib_module, oracle_grid, rel

pytestmark = pytest.mark.gpu

TAIL_RTOL = 0.05   # relative agreement of tails / errors with the oracle's
FP32_FLOOR = 1e-6  # absolute float32 floor of a tail or a relative error
ETA = 0.25         # relative perturbation of a truncation threshold by float32 data
# log c: the measurement tables are float32, so h is off by about u h_max and
# each likelihood exponent (z - h)^2 / 2R by |z - h| u h_max / R; over the
# points within 3 sigma_R of the measurement that is 3 sqrt(R) u h_max / R
# = 2e-5 for R = 0.01, h_max = 11.3 (config 2)
LOGC_TOL = 1e-4


@pytest.fixture(scope="module")
def G():
    return lib_module()


def rank1_prior(grid, mean, var):
    cores = [np.exp(-0.5 * (grid.axes[m] - mean[m]) ** 2 / var[m]).reshape(1, -1, 1)
             for m in range(grid.d)]
    cores[-1] = cores[-1] / (tt.full_sum(cores) * grid.delta)
    return cores


def f32(cores):
    """The shared input: float32 cores, seen by the oracle in float64."""
    return [np.asarray(c, dtype=np.float32).astype(np.float64) for c in cores]


def oracle_state(model, mc, steps, cap, smax=10):
    g = oracle_grid(model)
    comps = model.tables(g.axes)
    _, z = synth.simulate(model, mc, steps=steps + 1)
    X = rank1_prior(g, model.m0, np.diag(model.P0))
    for k in range(steps):
        X, _ = T.step(X, g, model.F, model.Q, comps, z[k], model.R, model.eps, cap, smax)
    return f32(X), z[steps]


def new_filter(G, model, cap, smax=0, batch=1, precision="fp32"):
    """precision: ttgbf_opts.precision, optionally "/" and the contraction."""
    prec, _, contraction = precision.partition("/")
    return G.TTFilter(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), batch=batch,
                      rank_cap=cap, eps=model.eps, max_shift_span=smax, precision=prec,
                      contraction=contraction or "fp32")


# ttgbf_opts.precision (R factors / SVDs of the truncating stages), and float32
# R / SVD with the core contractions on the tensor cores in split TF32
PRECISIONS = ["fp32", "fp64", "fp32/tf32x3"]


def gpu_cores(f, b=0):
    return [c.astype(np.float64) for c in f.export_cores(b)]


def link_singular_values(cores):
    """Singular values of every link's unfolding of a TT whose cores left of
    the link are left-orthonormal: those of the right part, from the Gram
    matrices contracted from the right."""
    d = len(cores)
    Gm = np.ones((1, 1))
    out = [None] * (d - 1)
    for k in range(d - 1, 0, -1):
        C = cores[k]
        Gm = np.einsum("aib,bc,dic->ad", C, Gm, C)
        w = np.linalg.eigvalsh(0.5 * (Gm + Gm.T))[::-1]
        out[k - 1] = np.sqrt(np.maximum(w, 0.0))
    return out


def final_decisions(trace):
    """The oracle's last truncation record of every link."""
    last = {}
    for rec in trace:
        last[rec["link"]] = rec
    return last


def check_ranks(gpu_ranks, orc_ranks, trace, what):
    """Equal ranks on every link, except where the oracle's own decision is at
    the threshold; returns the number of such borderline links."""
    last = final_decisions(trace)
    border = 0
    for k in range(len(orc_ranks) - 2):  # link k between cores k and k + 1
        rg, ro = gpu_ranks[k + 1], orc_ranks[k + 1]
        if rg == ro:
            continue
        assert k in last and T.rank_is_borderline(last[k], rg, ETA), (what, k, gpu_ranks, orc_ranks)
        border += 1
    return border


def check_left_orthonormal(cores, svals):
    """Cores 0..d-2 (left of the center after a full rounding) against the
    identity: returns (plain max |C^T C - I|, the same weighted by the link's
    singular values and divided by the largest squared one).  The cores are
    formed as unfolding x V S^-1 without an explicit Q, so column i of a core
    is off by about u s_1 / s_i; the tensor itself carries column i with weight
    s_i, so the weighted deviation is the one that moves the TT (about u)."""
    plain = weighted = 0.0
    for k in range(len(cores) - 1):
        C = cores[k]
        M = C.reshape(-1, C.shape[2])
        q = min(M.shape[1], len(svals[k]))  # ranks may differ on a borderline link
        M = M[:, :q]
        D = M.T @ M - np.eye(q)
        s = svals[k][:q]
        plain = max(plain, float(np.abs(D).max()))
        weighted = max(weighted, float(np.abs(s[:, None] * D * s[None, :]).max() / s[0] ** 2))
    return plain, weighted


@pytest.fixture(scope="module")
def bench_state():
    model = synth.config2(n=128)
    X, z = oracle_state(model, 0, 2, 16)
    assert max(tt.ranks(X)) == 16  # the cap binds at this state
    return model, X, z


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("m,n,a,S", [(1, 2, 0.055, 9), (0, 2, 0.03, 5), (2, 0, 0.04, 7)])
def test_round_matches_oracle_at_bench_shapes(G, bench_state, m, n, a, S, precision):
    model, X, _ = bench_state
    g = oracle_grid(model)
    s, ts = T.shear_shifts(g, m, n, a)
    assert len(ts) == S
    A = tt.shear_operator(X, m, n, s, ts)
    f = new_filter(G, model, 16, precision=precision)
    f.import_cores(0, [c.astype(np.float32) for c in X])
    f.shear(m, n, a, do_round=False)
    assert T.rel_distance(gpu_cores(f), A) < 1e-6  # the expansion itself is exact
    t0 = f.stats()[0]["tail_sum"]
    f.round()
    gpu_tail = f.stats()[0]["tail_sum"] - t0
    out = gpu_cores(f)
    trace = []
    B, tails = T.round_full(A, model.eps, 16, trace)
    err_orc = math.sqrt(sum(t * t for t in tails))
    assert abs(T.rel_distance(B, A) - err_orc) < 1e-7  # the oracle's error identity
    assert err_orc > 10 * model.eps  # the cap binds
    border = check_ranks(tt.ranks(out), tt.ranks(B), trace, "round")
    err_gpu = T.rel_distance(out, A)
    assert err_gpu <= (1 + TAIL_RTOL) * err_orc + FP32_FLOOR, (err_gpu, err_orc)
    assert abs(gpu_tail - sum(tails)) <= TAIL_RTOL * sum(tails) + FP32_FLOOR, (gpu_tail, sum(tails))
    assert T.rel_distance(out, B) <= 2 * err_orc + FP32_FLOOR
    plain, weighted = check_left_orthonormal(out, link_singular_values(B))
    print(f"{precision} shear ({m},{n}) S={S}: ranks {tt.ranks(out)} oracle {tt.ranks(B)} "
          f"({border} borderline) err gpu {err_gpu:.4e} oracle {err_orc:.4e} "
          f"tail gpu {gpu_tail:.4e} oracle {sum(tails):.4e} |C^T C - I| {plain:.2e} "
          f"weighted {weighted:.2e}")
    assert weighted < 1e-5


def _compare_step(G, model, X, z, cap, smax=0, precision="fp32"):
    """One predict, then one update, each from the oracle's state."""
    g = oracle_grid(model)
    f = new_filter(G, model, cap, smax, precision=precision)
    comps = device_tables(model, f.grid_axes())
    oc = model.tables(g.axes)
    f.import_cores(0, [c.astype(np.float32) for c in X])
    f.predict(model.F, model.Q)
    trp = []
    Yp, tp, _ = T.predict(X, g, model.F, model.Q, model.eps, cap, smax or 10, trp)
    out = gpu_cores(f)
    t_gpu = f.stats()[0]["tail_sum"]
    bp = check_ranks(tt.ranks(out), tt.ranks(Yp), trp, "predict")
    assert abs(t_gpu - sum(tp)) <= TAIL_RTOL * sum(tp) + FP32_FLOOR * len(tp), (t_gpu, sum(tp))
    assert T.rel_distance(out, Yp) <= 10 * (model.eps + sum(tp)) + 1e-5
    # update from the oracle's predicted state (the step's tail statistics
    # keep the predict's tails: the update's are the difference)
    Yp = f32(Yp)
    f.import_cores(0, [c.astype(np.float32) for c in Yp])
    t0 = f.stats()[0]["tail_sum"]
    f.update(comps, model.R, z[None, :])
    tru = []
    Yu, tu, logc = T.update(Yp, g, oc, z, model.R, model.eps, cap, tru)
    out = gpu_cores(f)
    st = f.stats()[0]
    bu = check_ranks(tt.ranks(out), tt.ranks(Yu), tru, "update")
    assert abs(st["tail_sum"] - t0 - sum(tu)) <= TAIL_RTOL * sum(tu) + FP32_FLOOR * len(tu), \
        (st["tail_sum"] - t0, sum(tu))
    assert T.rel_distance(out, Yu) <= 10 * (model.eps + sum(tu)) + 1e-5
    m, c, lc, ll = f.estimate()
    mo, co = T.moments(Yu, g)
    assert (np.abs(m[0] - mo) <= 1e-3 * g.delta_axis).all(), (m[0], mo)
    assert (np.abs(c[0] - co) <= cov_tol(g.delta_axis, co)).all()
    assert abs(lc[0] - logc) < LOGC_TOL, (lc[0], logc)
    print(f"{precision} N={model.n[0]} cap {cap}: predict tails gpu {t_gpu:.4e} oracle {sum(tp):.4e}, "
          f"update tails gpu {st['tail_sum'] - t0:.4e} oracle {sum(tu):.4e}, borderline ranks "
          f"{bp} + {bu}, |log c diff| {abs(lc[0] - logc):.2e}")
    return sum(tp), sum(tu)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("n,cap,mc,k", [(128, 16, 0, 2), (32, 8, 3, 3), (32, 32, 3, 3), (32, 32, 4, 5)])
def test_one_step_matches_oracle_tt_step(G, n, cap, mc, k, precision):
    model = synth.config2(n=n)
    smax = 5 if cap == 32 else 0  # rank cap x span <= 160 columns
    X, z = oracle_state(model, mc, k, cap, smax or 10)
    _compare_step(G, model, X, z, cap, smax, precision=precision)


@pytest.mark.parametrize("n,cap,smax,precision", [(32, 53, 3, "fp32"), (64, 53, 3, "fp32"),
                                                   (32, 53, 3, "fp64"), (32, 53, 3, "fp32/tf32x3")])
def test_flat_bounds_where_the_cap_does_not_bind(G, n, cap, smax, precision):
    model = synth.config2(n=n)
    g = oracle_grid(model)
    oc = model.tables(g.axes)
    mcs = [0, 1]
    steps = 6
    f = new_filter(G, model, cap, smax, batch=len(mcs), precision=precision)
    comps = device_tables(model, f.grid_axes())
    zs = [synth.simulate(model, mc, steps=steps)[1] for mc in mcs]
    Ps = [pmf.prior(g, model.m0, model.P0) for _ in mcs]
    X = [rank1_prior(g, model.m0, np.diag(model.P0)) for _ in mcs]
    flat = 10 * model.eps + 1e-5
    for k in range(steps):
        f.predict(model.F, model.Q)
        f.update(comps, model.R, np.stack([z[k] for z in zs]))
        m, c, lc, ll = f.estimate()
        for i in range(len(mcs)):
            Ps[i], _ = pmf.predict_rg(Ps[i], g, model.F, model.Q)
            Ps[i], logc = pmf.update(Ps[i], g, pmf.likelihood(g, oc, zs[i][k], model.R))
            X[i], info = T.step(X[i], g, model.F, model.Q, oc, zs[i][k], model.R, model.eps, cap, smax)
            # premise: the TT method itself meets the flat bound at this rank cap
            # (the oracle TT filter's density error), so the GPU path must too
            e_or = rel(tt.densify(X[i]), Ps[i])
            assert e_or < flat, (k, i, e_or)
            e = rel(tt.densify(gpu_cores(f, i)), Ps[i])
            mo, co = pmf.moments(Ps[i], g)
            print(f"N={n} step {k} filter {i}: rel err {e:.3e} (flat bound {flat:.1e}), mean err / D "
                  f"{(np.abs(m[i] - mo) / g.delta_axis).max():.2e}, ranks {f.ranks()[i].tolist()}")
            assert e <= flat, (k, i, e)
            assert (np.abs(m[i] - mo) <= 1e-3 * g.delta_axis).all(), (k, i)
            assert (np.abs(c[i] - co) <= cov_tol(g.delta_axis, co)).all(), (k, i)
            assert abs(lc[i] - logc) < LOGC_TOL, (k, i, lc[i], logc)
