"""Deterministic tensor-train cross interpolation (test infrastructure only:
the oracle of the GPU path's cross; only tests/, smoke() and bench.py's CPU
legs use it).

Sec. 3 ("black-box decomposition approximation", Eq. matrixDecomp): a matrix
A is approximated from r of its columns C and r of its rows R as
C Â^{-1} R, Â the r x r intersection, and the approximation is best (up to a
bounded factor) when |det Â| is largest; a tensor train is built from such
skeletons link by link, evaluating the tensor only at the entries the
skeletons touch.  The paper chooses rows and columns by a randomised greedy
search; here every choice is made by the deterministic maximum-volume
heuristic ("maxvol": Gaussian elimination with partial pivoting for a start,
then single-row exchanges while some entry of C Â^{-1} exceeds 1 + delta), so
that the same input always gives the same approximation.

What is approximated is the likelihood-weighted block of a density TT
(the update of Alg. 2, step 2, for a likelihood factor that couples the modes
lo..hi): with the cores left of lo left-orthonormal and right of hi
right-orthonormal, the block tensor

    T(a, i_lo, ..., i_hi, b) = L(i_lo, ..., i_hi) [G_lo(i_lo) ... G_hi(i_hi)](a, b)

carries the whole tensor's Frobenius geometry, so an approximation of T is an
approximation of L (.) P of the same relative accuracy.  The block's first
mode is the pair (a, i_lo) and its last the pair (i_hi, b) ("virtual" modes of
sizes r_lo N_lo and N_hi r_hi+1); the cross has k = hi - lo + 1 modes and
k - 1 links.

The sweeps (all steps in float64, numpy's Householder QR as a library step):
* start: right index sets J_l (l = k-1 .. 1) from the density block alone,
  right to left: the rows of [G_{l+1}(i) V_{l+1}(beta)] (one row per new
  multi-index (i, beta)) chosen by maxvol on an orthonormal basis of their
  span, then padded with the rows of largest norm to s_l entries;
* left-to-right half sweep: at link l the fiber matrix
  T(I_{l-1} x mode l, J_l) ((s_{l-1} n_l) x s_l) gets an orthonormal basis Q
  and maxvol rows; those rows are the new left set I_l and Q Q[rows]^{-1} is
  core l;
* right-to-left half sweep, the mirror image, renewing the right sets;
* `sweeps` pairs of these two half sweeps, then a final left-to-right sweep
  whose cores are the result; the last core is the fiber T(I_{k-1} x mode k).
Ranks: s_l = min(s, product of the virtual mode sizes left of link l,
product right of it).
"""
from __future__ import annotations

import itertools
import math

import numpy as np


# -------------------------------------------------------------- maxvol ----
def lu_rows(Q):
    """Row choice of Gaussian elimination with partial row pivoting on Q
    (M x n, M >= n): for each column in turn the not yet chosen row of
    largest magnitude (the first such row at a tie), then elimination of that
    column from the later columns.  Returns n row indices."""
    A = np.array(Q, dtype=np.float64, copy=True)
    M, n = A.shape
    free = np.ones(M, dtype=bool)
    rows = []
    for j in range(n):
        col = np.where(free, np.abs(A[:, j]), -1.0)
        p = int(np.argmax(col))
        rows.append(p)
        free[p] = False
        if A[p, j] != 0.0:
            A[:, j + 1:] -= np.outer(A[:, j] / A[p, j], A[p, j + 1:])
    return rows


def maxvol(Q, delta=0.05, max_iter=100):
    """Maximum-volume rows of Q (M x n): start from lu_rows, then while the
    largest |B_ij| of B = Q Q[rows]^{-1} exceeds 1 + delta (the first such
    entry in row-major order), put row i in place j and update B by the
    rank-one formula.  Returns (rows, B); B[rows] is the identity."""
    Q = np.asarray(Q, dtype=np.float64)
    M, n = Q.shape
    rows = lu_rows(Q)
    B = Q @ np.linalg.inv(Q[rows])
    for _ in range(max_iter):
        flat = int(np.argmax(np.abs(B)))
        i, j = divmod(flat, n)
        if abs(B[i, j]) <= 1.0 + delta:
            break
        e = np.zeros(n)
        e[j] = 1.0
        B = B - np.outer(B[:, j], B[i, :] - e) / B[i, j]
        rows[j] = i
    return rows, B


def orth(A):
    """Orthonormal basis of the columns of A (Householder QR, reduced)."""
    return np.linalg.qr(np.asarray(A, dtype=np.float64), mode="reduced")[0]


def select_rows(Y, s, delta=0.05):
    """s rows of Y (M x w): maxvol on an orthonormal basis of its columns
    (min(w, s) of them), padded by the not yet chosen rows of largest norm
    (the first at a tie).  Returns the rows and the basis's B."""
    Q = orth(Y)[:, :min(Y.shape[1], s)]
    rows, B = maxvol(Q, delta)
    if s > len(rows):
        norms = np.linalg.norm(Y, axis=1)
        norms[rows] = -1.0
        order = np.argsort(-norms, kind="stable")
        rows = list(rows) + [int(i) for i in order[:s - len(rows)]]
    return rows, B


# ----------------------------------------------------------- the block ----
class Block:
    """The likelihood-weighted density block T of the module docstring.
    cores: the k >= 2 density cores of modes lo..hi (float64, shapes
    (r_lo, N_lo, r_lo+1), ..., (r_hi, N_hi, r_hi+1)); lik: the likelihood on
    the grid indices of those modes, an array of shape (N_lo, ..., N_hi)."""

    def __init__(self, cores, lik):
        self.G = [np.asarray(c, dtype=np.float64) for c in cores]
        self.k = len(self.G)
        if self.k < 2:
            raise ValueError("a block spans at least two modes")
        self.L = np.asarray(lik, dtype=np.float64)
        self.N = [c.shape[1] for c in self.G]
        self.r_first = self.G[0].shape[0]
        self.r_last = self.G[-1].shape[2]
        # virtual mode sizes: (a, i_lo) first, (i_hi, b) last
        self.n = list(self.N)
        self.n[0] *= self.r_first
        self.n[-1] *= self.r_last

    def grid_index(self, q, v):
        """Grid index of virtual index v of block mode q (0-based)."""
        if q == 0:
            return v % self.N[0]
        if q == self.k - 1:
            return v // self.r_last
        return v

    def core_slice(self, q, v):
        """The matrix G_q at virtual index v: 1 x r for the first mode (row a
        of G_lo(i_lo)), r x 1 for the last (column b of G_hi(i_hi))."""
        if q == 0:
            a, i = divmod(v, self.N[0])
            return self.G[0][a, i, :][None, :]
        if q == self.k - 1:
            i, b = divmod(v, self.r_last)
            return self.G[q][:, i, b][:, None]
        return self.G[q][:, v, :]

    def left_vector(self, alpha):
        """Row vector G'_0(alpha_0) ... G'_{l-1}(alpha_{l-1}) (empty alpha: [1])."""
        P = np.ones((1, 1))
        for q, v in enumerate(alpha):
            P = P @ self.core_slice(q, v)
        return P[0]

    def right_vector(self, beta):
        """Column vector G'_q(beta_0) ... G'_{k-1}(beta_end) for the
        multi-index beta of the last len(beta) modes (empty beta: [1])."""
        P = np.ones((1, 1))
        q0 = self.k - len(beta)
        for t in range(self.k - 1, q0 - 1, -1):
            P = self.core_slice(t, beta[t - q0]) @ P
        return P[:, 0]

    def lik(self, vs):
        return float(self.L[tuple(self.grid_index(q, v) for q, v in enumerate(vs))])

    def value(self, vs):
        """T at the virtual multi-index vs (length k)."""
        P = np.ones((1, 1))
        for q, v in enumerate(vs):
            P = P @ self.core_slice(q, v)
        return float(P[0, 0]) * self.lik(vs)

    def fiber(self, alpha, q, beta):
        """T(alpha, v, beta) for every virtual index v of mode q."""
        u, w = self.left_vector(alpha), self.right_vector(beta)
        return np.array([float(u @ self.core_slice(q, v) @ w) * self.lik(alpha + (v,) + beta)
                         for v in range(self.n[q])])

    def dense(self):
        """T over all virtual indices (k-dimensional array)."""
        out = np.zeros(self.n)
        for vs in itertools.product(*[range(n) for n in self.n]):
            out[vs] = self.value(vs)
        return out


def link_ranks(blk, s):
    """s_l for links l = 1..k-1."""
    return [min(s, math.prod(blk.n[:l]), math.prod(blk.n[l:])) for l in range(1, blk.k)]


def start_sets(blk, s, delta=0.05):
    """Right index sets from the density block alone (module docstring,
    "start").  J[l] (l = 1..k-1) is a list of tuples of virtual indices of
    modes l..k-1 (0-based mode numbers); J[k] = [()]."""
    k = blk.k
    sz = link_ranks(blk, s)
    J = [None] * (k + 1)
    J[k] = [()]
    for l in range(k - 1, 0, -1):
        rows, Y = [], []
        for v in range(blk.n[l]):
            for beta in J[l + 1]:
                rows.append((v,) + beta)
                Y.append(blk.core_slice(l, v) @ blk.right_vector(beta))
        sel, _ = select_rows(np.array(Y), sz[l - 1], delta)
        J[l] = [rows[i] for i in sel]
    return J


def lr_step(blk, I_prev, Jq, q, delta=0.05):
    """Left-to-right step at block mode q: fiber matrix with rows (alpha, v),
    alpha in I_prev major, and columns beta in Jq.  Returns (new left set,
    core Q Q[rows]^{-1} as (|I_prev|, n_q, |Jq|))."""
    Fm = np.stack([np.concatenate([blk.fiber(alpha, q, beta) for alpha in I_prev]) for beta in Jq], axis=1)
    sel, Bm = maxvol(orth(Fm), delta)
    rows = [alpha + (v,) for alpha in I_prev for v in range(blk.n[q])]
    return [rows[i] for i in sel], Bm.reshape(len(I_prev), blk.n[q], len(sel))


def rl_step(blk, Iq, J_next, q, delta=0.05):
    """Right-to-left step at block mode q: fiber matrix with rows (v, beta),
    v major, beta in J_next, and columns alpha in Iq.  Returns (new right set,
    core (Q Q[rows]^{-1})^T as (|rows|, n_q, |J_next|))."""
    Fm = np.stack([np.stack([blk.fiber(alpha, q, beta) for beta in J_next], axis=1).reshape(-1)
                   for alpha in Iq], axis=1)
    sel, Bm = maxvol(orth(Fm), delta)
    rows = [(v,) + beta for v in range(blk.n[q]) for beta in J_next]
    return [rows[i] for i in sel], Bm.T.reshape(len(sel), blk.n[q], len(J_next))


class TransitionBlock(Block):
    """The 2-site block of cores (m, m+1) after one factor of the textbook
    transition (Eqs. pdf_predII, TPMmat) whose mode-m Gaussian is shifted by
    the coupling to mode m+1:

        T(a, j, i', b) = sum_i K(j, i, i') [G_m(i) G_{m+1}(i')](a, b),

    K of shape (N_m, N_m, N_{m+1}).  Virtual modes: (a, j) and (i', b).  The
    start sets, which look at the density alone, are those of Block."""

    def __init__(self, cores, K):
        super().__init__(cores, np.ones([c.shape[1] for c in cores]))
        if self.k != 2:
            raise ValueError("a transition block spans two modes")
        self.K = np.asarray(K, dtype=np.float64)

    def value(self, vs):
        a, j = divmod(vs[0], self.N[0])
        i1, b = divmod(vs[1], self.r_last)
        w = self.G[1][:, i1, b]                      # (r,)
        y = self.G[0][a] @ w                         # (N_m,) over i
        return float(self.K[j, :, i1] @ y)

    def fiber(self, alpha, q, beta):
        if q == 0:
            return np.array([self.value((v, beta[0])) for v in range(self.n[0])])
        return np.array([self.value((alpha[0], v)) for v in range(self.n[1])])


def block_cross(cores, lik, s, sweeps=1, delta=0.05):
    """Cross approximation of the likelihood-weighted block (module
    docstring): see cross_of_block."""
    return cross_of_block(Block(cores, lik), s, sweeps, delta)


def cross_of_block(blk, s, sweeps=1, delta=0.05):
    """Start sets, then `sweeps` pairs of (left-to-right, right-to-left) half
    sweeps, then the final left-to-right sweep whose cores are returned, in
    the density's core shapes with ranks (r_lo, s_1, ..., s_{k-1}, r_hi+1).
    Returns (cores, index sets)."""
    k = blk.k
    J = start_sets(blk, s, delta)
    I = [None] * k
    I[0] = [()]
    for _ in range(sweeps):
        for q in range(k - 1):
            I[q + 1], _core = lr_step(blk, I[q], J[q + 1], q, delta)
        for q in range(k - 1, 0, -1):
            J[q], _core = rl_step(blk, I[q], J[q + 1], q, delta)
    out = []
    for q in range(k - 1):
        I[q + 1], core = lr_step(blk, I[q], J[q + 1], q, delta)
        out.append(core)
    last = np.stack([blk.fiber(alpha, k - 1, ()) for alpha in I[k - 1]])
    out.append(last[:, :, None])
    out[0] = out[0].reshape(blk.r_first, blk.N[0], out[0].shape[2])
    out[-1] = out[-1].reshape(out[-1].shape[0], blk.N[-1], blk.r_last)
    return out, {"I": I, "J": J}
