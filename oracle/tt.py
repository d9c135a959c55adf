"""Plain tensor-train helpers in float64 (test infrastructure only).

The TT format is Sec. 3, Eq. ttd_exact: A(i_1..i_d) = G_1(:, i_1, :) ...
G_d(:, i_d, :) with cores G_k of shape (r_{k-1}, N_k, r_k) and r_0 = r_d = 1.
Rounding follows the paper's "round" (Sec. 4.1, fourth bullet; Alg. 2 steps 2
and 4): orthogonalise right to left, then truncate left to right by SVD,
keeping on every link the smallest rank whose discarded singular values have
norm <= eps ||A||_F / sqrt(d - 1), then capping the rank at rmax.  The
reading of the threshold is the one that makes ||A - round(A)||_F <= eps ||A||_F
when the cap does not bind.  The TT sum and the hat shear as a TT operator
(the re-gridding shear in TT form) are pinned against the elementwise sum and
the dense push-forward of oracle/pmf.py.
"""
from __future__ import annotations

import math

import numpy as np


def densify(cores) -> np.ndarray:
    """Contract a TT into the full tensor (small cases only)."""
    out = np.asarray(cores[0], dtype=np.float64)
    shape = [out.shape[1]]
    out = out.reshape(out.shape[1], out.shape[2])
    for G in cores[1:]:
        G = np.asarray(G, dtype=np.float64)
        out = out @ G.reshape(G.shape[0], -1)
        shape.append(G.shape[1])
        out = out.reshape(-1, G.shape[2])
    return out.reshape(shape)


def ranks(cores) -> list[int]:
    return [1] + [int(G.shape[2]) for G in cores]


def inner(a, b) -> float:
    """<A, B> = sum_i A(i) B(i) by the left-to-right contraction (TT `dot`)."""
    E = np.ones((1, 1))
    for Ga, Gb in zip(a, b):
        E = np.einsum("ab,aic,bid->cd", E, Ga, Gb)
    return float(E[0, 0])


def full_sum(cores) -> float:
    """sum_i A(i) (TT `sum`)."""
    v = np.ones((1,))
    for G in cores:
        v = v @ np.asarray(G).sum(axis=1)
    return float(v[0])


def round_tt(cores, eps: float, rmax: int | None = None):
    """TT rounding.  Returns (cores, tails) where tails[k] is the discarded
    Frobenius norm on link k divided by ||A||_F."""
    G = [np.asarray(c, dtype=np.float64).copy() for c in cores]
    d = len(G)
    for k in range(d - 1, 0, -1):
        r0, n, r1 = G[k].shape
        Qm, Rm = np.linalg.qr(G[k].reshape(r0, n * r1).T)
        G[k] = Qm.T.reshape(-1, n, r1)
        G[k - 1] = np.einsum("aib,cb->aic", G[k - 1], Rm)
    norm = float(np.linalg.norm(G[0]))
    tails = []
    if norm == 0.0 or d == 1:
        return G, [0.0] * (d - 1)
    thr = eps * norm / math.sqrt(d - 1)
    for k in range(d - 1):
        r0, n, r1 = G[k].shape
        U, s, Vt = np.linalg.svd(G[k].reshape(r0 * n, r1), full_matrices=False)
        # tail[r] = norm of s[r:], for r = 0..len(s)
        tail = np.sqrt(np.concatenate([np.cumsum((s ** 2)[::-1])[::-1], [0.0]]))
        r = int(np.argmax(tail <= thr))
        r = max(1, r)
        if rmax is not None:
            r = min(r, rmax)
        tails.append(float(tail[r]) / norm)
        G[k] = U[:, :r].reshape(r0, n, r)
        G[k + 1] = np.einsum("ab,bic->aic", s[:r, None] * Vt[:r], G[k + 1])
    return G, tails


def from_dense(A: np.ndarray, eps: float = 0.0, rmax: int | None = None):
    """TT-SVD of a full tensor (used to build inputs in tests)."""
    A = np.asarray(A, dtype=np.float64)
    shape = A.shape
    d = len(shape)
    norm = float(np.linalg.norm(A))
    thr = eps * norm / math.sqrt(max(d - 1, 1))
    cores = []
    r = 1
    C = A.reshape(1, -1)
    for k in range(d - 1):
        C = C.reshape(r * shape[k], -1)
        U, s, Vt = np.linalg.svd(C, full_matrices=False)
        tail = np.sqrt(np.concatenate([np.cumsum((s ** 2)[::-1])[::-1], [0.0]]))
        rn = max(1, int(np.argmax(tail <= thr)))
        if rmax is not None:
            rn = min(rn, rmax)
        cores.append(U[:, :rn].reshape(r, shape[k], rn))
        C = s[:rn, None] * Vt[:rn]
        r = rn
    cores.append(C.reshape(r, shape[-1], 1))
    return cores


def add(a, b):
    """TT sum A + B (Sec. 3, the TT arithmetic "plus"): the first core is
    concatenated along its right rank, the last along its left rank, the
    cores between are block diagonal; the ranks add."""
    a = [np.asarray(G, dtype=np.float64) for G in a]
    b = [np.asarray(G, dtype=np.float64) for G in b]
    d = len(a)
    if d == 1:
        return [a[0] + b[0]]
    out = []
    for k, (Ga, Gb) in enumerate(zip(a, b)):
        ra0, n, ra1 = Ga.shape
        rb0, _, rb1 = Gb.shape
        if k == 0:
            out.append(np.concatenate([Ga, Gb], axis=2))
        elif k == d - 1:
            out.append(np.concatenate([Ga, Gb], axis=0))
        else:
            C = np.zeros((ra0 + rb0, n, ra1 + rb1))
            C[:ra0, :, :ra1] = Ga
            C[ra0:, :, ra1:] = Gb
            out.append(C)
    return out


def shear_operator(cores, m: int, n: int, s, ts=None):
    """The hat-interpolation shear x_m <- x_m + a x_n applied to a TT as a TT
    operator (the re-gridding shear of the transition, applied in TT form
    instead of by TT cross).  With s_i = a xi_{n,i} / D_m the weight of the
    source cell i_m for target j_m is hat(j_m - i_m - s_i) = sum over
    integers t of hat(t - s_i) [j_m - i_m = t], so the operator is
    sum_t E_t (x) H_t: E_t shifts mode m by t (zero outside the grid) and
    H_t = diag(hat(t - s_i)) weights mode n.  Each t is a rank-preserving
    term; their sum is the TT sum over t of the terms, which share the cores
    outside [min(m, n), max(m, n)].  ts: the shifts to include (default:
    every t with a nonzero weight).  Ranks inside the block grow by len(ts)."""
    s = np.asarray(s, dtype=np.float64)
    if ts is None:
        ts = range(int(math.floor(s.min())), int(math.floor(s.max())) + 2)
    ts = list(ts)
    S = len(ts)
    lo, hi = min(m, n), max(m, n)
    out = [np.asarray(G, dtype=np.float64).copy() for G in cores]
    for k in range(lo, hi + 1):
        G = np.asarray(cores[k], dtype=np.float64)
        r0, N, r1 = G.shape
        L = r0 if k == lo else r0 * S
        R = r1 if k == hi else r1 * S
        C = np.zeros((L, N, R))
        for u, t in enumerate(ts):
            if k == m:
                Gs = np.zeros_like(G)  # Gs[:, j, :] = G[:, j - t, :]
                if 0 <= t < N:
                    Gs[:, t:, :] = G[:, :N - t, :]
                elif -N < t < 0:
                    Gs[:, :N + t, :] = G[:, -t:, :]
            elif k == n:
                w = np.maximum(0.0, 1.0 - np.abs(t - s))
                Gs = G * w[None, :, None]
            else:
                Gs = G
            rows = slice(0, r0) if k == lo else slice(u * r0, (u + 1) * r0)
            cols = slice(0, r1) if k == hi else slice(u * r1, (u + 1) * r1)
            C[rows, :, cols] = Gs
        out[k] = C
    return out

