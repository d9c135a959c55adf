"""Log marginal likelihood of the re-gridded point-mass filter as a
differentiable function of the model (test infrastructure only).

The filter's log-likelihood is l = sum_k log c_k (Eq. pmf_filtrace_b, the
normaliser of each update).  Written here in float64 with plain PyTorch CPU
operations, following the same definitions and order as oracle/pmf.py
(F = L D U without pivoting; U's hat shears, D's cloud-in-cell scalings, L's
shears; the separable Gaussian kernel; normalisation; the Bayes update), so
that reverse-mode differentiation gives dl/dF, dl/dQ_mm and dl/dR_cc: the
reference gradient for an adjoint of the filter step (system identification).

The operators are piecewise linear in the shear and scaling coefficients
(hat weights have kinks where a shifted index is an integer): away from the
kinks the function is smooth and the gradient is the ordinary one.  Zero
couplings of L and U and unit scalings are skipped as in oracle/pmf.py, so
the gradient with respect to them is not defined here.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import pmf

_T = torch.float64


def _hat(t: torch.Tensor) -> torch.Tensor:
    return torch.clamp(1.0 - t.abs(), min=0.0)


def ldu(F: torch.Tensor):
    """F = L diag(D) U (Doolittle, no pivoting), differentiable."""
    d = F.shape[0]
    L = [[None] * d for _ in range(d)]
    U = [[None] * d for _ in range(d)]
    D = [None] * d
    for k in range(d):
        D[k] = F[k, k] - sum((L[k][j] * D[j] * U[j][k] for j in range(k)), torch.zeros((), dtype=_T))
        for i in range(k + 1, d):
            L[i][k] = (F[i, k] - sum((L[i][j] * D[j] * U[j][k] for j in range(k)),
                                     torch.zeros((), dtype=_T))) / D[k]
            U[k][i] = (F[k, i] - sum((L[k][j] * D[j] * U[j][i] for j in range(k)),
                                     torch.zeros((), dtype=_T))) / D[k]
    return L, D, U


def _shift(P: torch.Tensor, axis: int, t: int) -> torch.Tensor:
    """out[.., j, ..] = P[.., j - t, ..] (zero where j - t is off the grid)."""
    n = P.shape[axis]
    out = torch.zeros_like(P)
    if abs(t) >= n:
        return out
    dst = [slice(None)] * P.dim()
    src = [slice(None)] * P.dim()
    dst[axis] = slice(max(0, t), n + min(0, t))
    src[axis] = slice(max(0, -t), n - max(0, t))
    out[tuple(dst)] = P[tuple(src)]
    return out


def shear(P: torch.Tensor, grid: pmf.Grid, m: int, n: int, a: torch.Tensor) -> torch.Tensor:
    """x_m <- x_m + a x_n: P'(.., j_m, .., i_n, ..) = sum_t hat(t - s_{i_n})
    P(.., j_m - t, .., i_n, ..), s_{i_n} = a xi_{n,i_n} / D_m."""
    s = a * torch.as_tensor(grid.axes[n], dtype=_T) / float(grid.delta_axis[m])
    sv = s.detach().numpy()
    out = torch.zeros_like(P)
    shape = [1] * P.dim()
    shape[n] = grid.shape[n]
    for t in range(int(math.floor(sv.min())), int(math.floor(sv.max())) + 2):
        out = out + _shift(P, m, t) * _hat(t - s).reshape(shape)
    return out


def scale(P: torch.Tensor, grid: pmf.Grid, m: int, lam: torch.Tensor) -> torch.Tensor:
    """x_m <- lam x_m by cloud-in-cell: W[j, i] = hat(j - u_i),
    u_i = (lam xi_{m,i} - lo_m) / D_m - 1/2."""
    xi = torch.as_tensor(grid.axes[m], dtype=_T)
    u = (lam * xi - float(grid.lo[m])) / float(grid.delta_axis[m]) - 0.5
    j = torch.arange(grid.shape[m], dtype=_T)
    W = _hat(j[:, None] - u[None, :])
    return torch.movedim(torch.tensordot(W, P, dims=([1], [m])), 0, m)


def convolve(P: torch.Tensor, grid: pmf.Grid, m: int, q: torch.Tensor) -> torch.Tensor:
    """P'(.., j, ..) = sum_i kappa(j - i) P(.., i, ..), kappa(t) = D N(D t; 0, q)."""
    n = grid.shape[m]
    D = float(grid.delta_axis[m])
    idx = torch.arange(n, dtype=_T)
    tt = D * (idx[:, None] - idx[None, :])
    K = D * torch.exp(-0.5 * tt * tt / q) / torch.sqrt(2 * math.pi * q)
    return torch.movedim(torch.tensordot(K, P, dims=([1], [m])), 0, m)


def likelihood(grid: pmf.Grid, comps, z, r: torch.Tensor) -> torch.Tensor:
    """L(i) = prod_c N(z_c; h_c(xi_i), R_cc), r = diag(R); the residuals as
    pmf.residual takes them."""
    L = torch.ones(grid.shape, dtype=_T)
    for c, comp in enumerate(comps):
        modes, table, period = pmf.unpack_comp(comp)
        res = torch.as_tensor(pmf.residual(float(z[c]), table, period), dtype=_T)
        lc = torch.exp(-0.5 * res ** 2 / r[c]) / torch.sqrt(2 * math.pi * r[c])
        if len(modes) == 2 and modes[0] > modes[1]:
            lc = lc.T
        shape = [1] * grid.d
        for m in modes:
            shape[m] = grid.shape[m]
        L = L * lc.reshape(shape)
    return L


def log_likelihood(F, q, r, grid: pmf.Grid, prior_mean, prior_cov, comps, zs) -> torch.Tensor:
    """l = sum_k log c_k over the steps predict -> update(z_k), k = 1..K, from
    the normalised prior (the order and operators of oracle/pmf.py).
    F: (d, d) tensor; q: (d,) diagonal of Q; r: (b,) diagonal of R."""
    P = torch.as_tensor(pmf.prior(grid, prior_mean, prior_cov), dtype=_T)
    d = grid.d
    ll = torch.zeros((), dtype=_T)
    for z in zs:
        L, D, U = ldu(F)
        for m in range(d):
            for n in range(m + 1, d):
                if U[m][n].detach().item() != 0.0:
                    P = shear(P, grid, m, n, U[m][n])
        for m in range(d):
            if D[m].detach().item() != 1.0:
                P = scale(P, grid, m, D[m])
        for m in range(d - 1, -1, -1):
            for n in range(m):
                if L[m][n].detach().item() != 0.0:
                    P = shear(P, grid, m, n, L[m][n])
        for m in range(d):
            P = convolve(P, grid, m, q[m])
        P = P / (P.sum() * grid.delta)
        W = likelihood(grid, comps, z, r) * P
        c = W.sum() * grid.delta
        P = W / c
        ll = ll + torch.log(c)
    return ll


def gradient(F, Q, R, grid: pmf.Grid, prior_mean, prior_cov, comps, zs):
    """(l, dl/dF (d x d), dl/dQ_mm (d), dl/dR_cc (b)) by reverse-mode
    differentiation of log_likelihood."""
    Ft = torch.tensor(np.asarray(F, dtype=np.float64), dtype=_T, requires_grad=True)
    qt = torch.tensor(np.diag(np.asarray(Q, dtype=np.float64)).copy(), dtype=_T, requires_grad=True)
    rt = torch.tensor(np.diag(np.atleast_2d(np.asarray(R, dtype=np.float64))).copy(), dtype=_T,
                      requires_grad=True)
    ll = log_likelihood(Ft, qt, rt, grid, prior_mean, prior_cov, comps, zs)
    ll.backward()
    return ll.detach().item(), Ft.grad.numpy(), qt.grad.numpy(), rt.grad.numpy()
