"""The reverse pass of the TT filter (ttgbf_adj_*, and the torch function
paper_2501_07942_gb300.log_likelihood over it): the gradient of the
log-likelihood l = sum_k log c_k (Eq. pmf_filtrace_b) with respect to F,
diag Q and diag R, from the adjoint recursion of the filter equations with the
adjoint density as a rounded tensor train.

* Against the oracle gradient (oracle/grad.py, reverse-mode differentiation of
  the dense float64 filter) on a 32^4 grid of the config-2 model, rank cap 32
  (span 5): the TT densities of the forward pass and the rounded adjoint differ
  from their dense counterparts by truncations at the eps level, so the
  gradient agrees with the dense one to GRAD_TOL of its largest entry.
* Against central differences of the GPU filter itself (float64 rounding
  stages, h = 1e-4): the differences also see the TT filter's own deviation
  from the dense filter and the float32 noise of l divided by h (FD_TOL of the
  largest entry).
* Checkpointing (segments of 1 step, recomputed in the backward pass) gives the
  same gradient as one segment, and the torch function's gradient is the
  batch's summed per-filter gradient."""
import numpy as np
import pytest

import synth
from oracle import grad, pmf

from gpu_util import bearing_cut_model, device_tables, lib_module, oracle_grid

pytestmark = pytest.mark.gpu

GRAD_TOL = 5e-3  # relative to max |dl/dtheta| (oracle gradient)
FD_TOL = 2e-2    # relative to max |dl/dtheta| (central differences, h = 1e-4)
LL_TOL = 1e-4    # |l_gpu - l_oracle| per step


@pytest.fixture(scope="module")
def G():
    return lib_module()


def setup(n=32, batch=2, steps=3):
    model = synth.config2(n=n)
    zs = [synth.simulate(model, mc, steps=steps)[1] for mc in range(batch)]
    return model, zs


def gpu_run(G, model, zs, cap=32, smax=5, precision="fp32", every=None, F=None, Q=None, R=None,
            grads=True):
    """Per-filter l and (optionally) gradients from a fresh batch run from the
    prior; every: steps per recorded segment (default: all)."""
    import torch
    F = model.F if F is None else F
    Q = model.Q if Q is None else Q
    R = model.R if R is None else R
    K, B = len(zs[0]), len(zs)
    every = K if every is None else every
    f = G.TTFilter(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), batch=B, rank_cap=cap,
                   eps=model.eps, max_shift_span=smax, precision=precision, conv="dense", parts=1)
    comps = device_tables(model, f.grid_axes())
    z = torch.tensor(np.stack(zs, axis=1), dtype=torch.float32, device="cuda")  # K x B x b
    nseg = -(-K // every)
    a = G.Adjoint(f, every, nseg) if grads else None

    def run(s):
        for k in range(s * every, min(K, (s + 1) * every)):
            f.predict(F, Q)
            f.update_dev(comps, R, z[k])

    for s in range(nseg):
        if a:
            a.save(s)
        run(s)
    ll = f.estimate()[3]
    out = None
    if a:
        a.reset()
        for s in range(nseg - 1, -1, -1):
            a.load(s)
            a.record(True)
            run(s)
            a.record(False)
            a.backward()
        out = a.grads(len(comps))
        a.free()
    f.free()
    return ll, out


def flat(dF, dq, dr):
    return np.concatenate([np.ravel(dF), np.ravel(dq), np.ravel(dr)])


def test_gradient_matches_oracle_gradient_at_32(G):
    model, zs = setup()
    ll, (dF, dQ, dR) = gpu_run(G, model, zs)
    g = oracle_grid(model)
    oc = model.tables(g.axes)
    for b, z in enumerate(zs):
        ll_o, dF_o, dq_o, dr_o = grad.gradient(model.F, model.Q, model.R, g, model.m0, model.P0, oc, list(z))
        ref = flat(dF_o, dq_o, dr_o)
        got = flat(dF[b], dQ[b], dR[b])
        err = np.abs(got - ref).max() / np.abs(ref).max()
        print(f"filter {b}: l gpu {ll[b]:.6f} oracle {ll_o:.6f}; max |grad err| / max |grad| {err:.2e}")
        print("  dF gpu", np.round(dF[b], 4).tolist(), "oracle", np.round(dF_o, 4).tolist())
        print("  dq gpu", dQ[b], "oracle", dq_o, " dr gpu", dR[b], "oracle", dr_o)
        assert abs(ll[b] - ll_o) <= LL_TOL * len(z), (ll[b], ll_o)
        assert err <= GRAD_TOL, err


def test_gradient_matches_central_differences_fp64(G):
    model, zs = setup(batch=1)
    ll, (dF, dQ, dR) = gpu_run(G, model, zs, precision="fp64")
    h = 1e-4
    params = []
    d = model.d
    for i in range(d):
        for j in range(d):
            if model.F[i, j] != 0.0:  # a zero coupling is not applied (kink of the hat weights)
                params.append(("F", i, j))
    params += [("Q", m, m) for m in range(d)] + [("R", 0, 0)]
    got, ref = [], []
    for kind, i, j in params:
        vals = []
        for e in (h, -h):
            F, Q, R = model.F.copy(), model.Q.copy(), np.array(model.R, dtype=float).copy()
            {"F": F, "Q": Q, "R": R}[kind][i, j] += e
            vals.append(gpu_run(G, model, zs, precision="fp64", F=F, Q=Q, R=R, grads=False)[0][0])
        ref.append((vals[0] - vals[1]) / (2 * h))
        got.append({"F": dF[0][i, j], "Q": dQ[0][i], "R": dR[0][0]}[kind])
    got, ref = np.array(got), np.array(ref)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    for p, a, b in zip(params, got, ref):
        print(p, f"adjoint {a:.6f} central difference {b:.6f}")
    print(f"max |adjoint - central difference| / max |grad| = {err:.2e}")
    assert err <= FD_TOL, err


def test_checkpointed_segments_and_torch_function(G):
    import torch
    model, zs = setup(batch=2, steps=4)
    ll1, g1 = gpu_run(G, model, zs, every=4)
    ll2, g2 = gpu_run(G, model, zs, every=1)
    assert np.array_equal(ll1, ll2)
    for a, b in zip(g1, g2):
        assert np.allclose(a, b, rtol=1e-6, atol=1e-9 * np.abs(a).max())
    # the torch function over the same run: summed per-filter gradients
    Ft = torch.tensor(model.F, dtype=torch.float64, requires_grad=True)
    qt = torch.tensor(np.diag(model.Q).copy(), dtype=torch.float64, requires_grad=True)
    rt = torch.tensor(np.diag(np.atleast_2d(model.R)).copy(), dtype=torch.float64, requires_grad=True)
    probe = G.TTFilter(model.lo, model.hi, model.n, model.m0, np.diag(model.P0), batch=1, rank_cap=32,
                       eps=model.eps, max_shift_span=5)
    comps = device_tables(model, probe.grid_axes())
    probe.free()
    z = torch.tensor(np.stack(zs, axis=1), dtype=torch.float32, device="cuda")
    ll = G.log_likelihood(Ft, qt, rt, lo=model.lo, hi=model.hi, n=model.n, prior_mean=model.m0,
                          prior_var=np.diag(model.P0), comps=comps, z=z, rank_cap=32, eps=model.eps,
                          max_shift_span=5, checkpoint_every=2)
    assert np.allclose(ll.detach().numpy(), ll1, rtol=0, atol=1e-9)
    ll.sum().backward()
    assert np.allclose(Ft.grad.numpy(), g1[0].sum(0), rtol=1e-6, atol=1e-9)
    assert np.allclose(qt.grad.numpy(), g1[1].sum(0), rtol=1e-6, atol=1e-9)
    assert np.allclose(rt.grad.numpy(), g1[2].sum(0), rtol=1e-6, atol=1e-9)


def _general_model(d):
    """The models of the oracle gradient's own pins (tests/test_oracle_grad.py):
    a full F (lower couplings, so separate scalings and L shears), one-mode
    components (d = 2) and a two-mode range with a one-mode component (d = 3)."""
    if d == 2:
        g = pmf.Grid([-6.0, -5.0], [6.0, 5.0], [20, 18])
        F = np.array([[0.93, 0.12], [-0.07, 0.88]])
        Q = np.diag([0.09, 0.12])
        comps = [((0,), synth.workloads.h_identity), ((1,), synth.workloads.h_sin)]
        R = np.diag([0.2, 0.1])
        z = np.array([[0.4, 0.2], [0.1, -0.3], [-0.2, 0.1]])
    else:
        g = pmf.Grid([-4.0, -4.0, -3.0], [4.0, 4.0, 3.0], [12, 10, 9])
        F = np.array([[0.95, 0.05, -0.04], [0.03, 0.9, 0.06], [0.0, -0.05, 0.92]])
        Q = np.diag([0.1, 0.15, 0.08])
        comps = [((0, 1), synth.workloads.h_range), ((2,), synth.workloads.h_identity)]
        R = np.diag([0.3, 0.2])
        z = np.array([[1.1, 0.2], [0.9, -0.1]])
    m = synth.Model(name=f"grad-d{d}", lo=np.array(g.lo), hi=np.array(g.hi), n=np.array(g.shape),
                    m0=np.zeros(d), P0=np.eye(d), F=F, Q=Q, R=R, comps=comps, eps=1e-6, rank_cap=32)
    return m, g, z


@pytest.mark.parametrize("d", [2, 3, "bearing"])
def test_gradient_general_models_match_oracle(G, d):
    """Separate scalings (kernel and scaling not fused), L shears, one-mode
    likelihood factors (their R-derivative on one core), at d = 3 a two-mode
    range with a one-mode component, and two two-mode components (range and
    a bearing whose residual wraps across the negative x axis): against the
    oracle gradient."""
    if d == "bearing":
        model, z = bearing_cut_model()
        g = oracle_grid(model)
    else:
        model, g, z = _general_model(d)
    ll, (dF, dQ, dR) = gpu_run(G, model, [z], cap=32, smax=5)
    oc = model.tables(g.axes)
    ll_o, dF_o, dq_o, dr_o = grad.gradient(model.F, model.Q, model.R, g, model.m0, model.P0, oc, list(z))
    ref = flat(dF_o, dq_o, dr_o)
    got = flat(dF[0], dQ[0], dR[0])
    err = np.abs(got - ref).max() / np.abs(ref).max()
    print(f"d={d}: l gpu {ll[0]:.6f} oracle {ll_o:.6f}; max |grad err| / max |grad| {err:.2e}")
    print("  gpu", np.round(got, 5).tolist())
    print("  oracle", np.round(ref, 5).tolist())
    assert abs(ll[0] - ll_o) <= LL_TOL * len(z), (ll[0], ll_o)
    assert err <= GRAD_TOL, err
