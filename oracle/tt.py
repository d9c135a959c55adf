"""Plain tensor-train helpers in float64 (test infrastructure only).

The TT format is Sec. 3, Eq. ttd_exact: A(i_1..i_d) = G_1(:, i_1, :) ...
G_d(:, i_d, :) with cores G_k of shape (r_{k-1}, N_k, r_k) and r_0 = r_d = 1.
Rounding follows the paper's "round" (Sec. 4.1, fourth bullet; Alg. 2 steps 2
and 4): orthogonalise right to left, then truncate left to right by SVD,
keeping on every link the smallest rank whose discarded singular values have
norm <= eps ||A||_F / sqrt(d - 1), then capping the rank at rmax.  The
reading of the threshold is the one that makes ||A - round(A)||_F <= eps ||A||_F
when the cap does not bind.
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
