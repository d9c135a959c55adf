"""The tensor-train point-mass filter step in float64 (test infrastructure only).

This is the TT form of the filter of Sec. 4 (Alg. 3 with linear dynamics, on a
fixed grid), written as plain TT operations so that the GPU path's rounding
decisions (ranks, discarded tails) can be checked against an independent
source rather than against what the GPU reports about itself.  Every step is
the same operator as the dense oracle (oracle/pmf.py), applied to the cores:

* predict: F = L D U (pmf.elementary_ops order).  A shear x_m += a x_n is the
  hat-weight TT operator of tt.shear_operator on the block of cores
  [lo, hi] = [min(m, n), max(m, n)], followed by TT rounding ("round", Sec. 3 /
  Alg. 2 step 4) of the links inside the block only: the TT is first put in
  mixed canonical form with its center in the block (cores left of the block
  left-orthonormal, right of it right-orthonormal), so the block's truncations
  are the ones a full rounding makes on those links.  A shear spanning more
  shifts than `smax` is applied as pieces of consecutive shifts, each rounded
  on the block, then summed as tensor trains on the block and rounded again.
  A scaling x_m <- lam x_m is the cloud-in-cell matrix on core m; then the
  Gaussian kernel (Eq. tpmconvFFT) is the Toeplitz matrix on every core's grid
  index; then normalisation (Alg. 2 step 4).
* update (Eqs. pmf_filtrace_a/b): a one-mode likelihood factor scales the
  slices of its core; a two-mode factor on modes (0, 1) multiplies the merged
  2-site core W(i_0, i_1, :) (cores 2.. right-orthonormal first), log c is the
  log of the mass of that product times the cell volume, and W is split by a
  truncated SVD that starts the left-to-right truncation sweep of the rounding
  (the remaining links are truncated in the same sweep).  Then normalisation.
  A factor on any other set of modes (three or more, or two other than
  (0, 1)) multiplies the block of cores it spans afterwards, one such factor
  at a time: exactly, or by the deterministic cross of oracle/cross.py, then
  the block's links are rounded and the TT normalised; its log c adds.
* Truncation rule on each link (the reading of the rounding tolerance): keep
  the smallest rank whose discarded singular values have norm <= eps ||A||_F /
  sqrt(d - 1), ||A||_F taken when the sweep starts, then cap the rank at rmax.
  The discarded tail of a link is reported relative to ||A||_F.

Library primitives (numpy QR, SVD, einsum) serve as steps; nothing is fused.
"""
from __future__ import annotations

import math

import numpy as np

from . import pmf, tt


def _cores(cores):
    return [np.array(c, dtype=np.float64, copy=True) for c in cores]


# ------------------------------------------------------ orthogonalisation ----
def right_orth(G, k):
    """Core k right-orthonormal (its unfolding r_{k-1} x (N_k r_k) gets
    orthonormal rows); the triangular factor moves into core k-1."""
    r0, n, r1 = G[k].shape
    Qm, Rm = np.linalg.qr(G[k].reshape(r0, n * r1).T)
    G[k] = Qm.T.reshape(-1, n, r1)
    G[k - 1] = np.einsum("aib,cb->aic", G[k - 1], Rm)


def left_orth(G, k):
    """Core k left-orthonormal (its unfolding (r_{k-1} N_k) x r_k gets
    orthonormal columns); the triangular factor moves into core k+1."""
    r0, n, r1 = G[k].shape
    Qm, Rm = np.linalg.qr(G[k].reshape(r0 * n, r1))
    G[k] = Qm.reshape(r0, n, -1)
    G[k + 1] = np.einsum("ab,bic->aic", Rm, G[k + 1])


def canonical(G, lo, hi):
    """Mixed canonical form with the center inside [lo, hi]: cores < lo
    left-orthonormal, cores > hi right-orthonormal (exact, no truncation)."""
    for k in range(lo):
        left_orth(G, k)
    for k in range(len(G) - 1, hi, -1):
        right_orth(G, k)


# ------------------------------------------------------------- truncation ----
def _rank_and_tail(s, thr, rmax):
    """Smallest rank r >= 1 with ||s[r:]|| <= thr, capped at rmax; and
    ||s[r:]||."""
    tail = np.sqrt(np.concatenate([np.cumsum((s ** 2)[::-1])[::-1], [0.0]]))
    r = max(1, int(np.argmax(tail <= thr)))
    if rmax is not None:
        r = min(r, rmax)
    return r, float(tail[r])


def left_sweep(G, k0, k1, thr, rmax, normA, trace=None):
    """Truncated SVD of the links k0..k1-1 (between cores k and k+1), left to
    right, for a TT whose cores left of k0 are left-orthonormal and right of
    k0 right-orthonormal.  Returns the relative tails.  trace (a list, when
    given) receives one record per link: link index, singular values,
    threshold, norm and the rank kept."""
    tails = []
    for k in range(k0, k1):
        r0, n, r1 = G[k].shape
        U, s, Vt = np.linalg.svd(G[k].reshape(r0 * n, r1), full_matrices=False)
        r, tail = _rank_and_tail(s, thr, rmax)
        if trace is not None:
            trace.append({"link": k, "s": s.copy(), "thr": thr, "normA": normA, "rank": r,
                          "rmax": rmax})
        tails.append(tail / normA if normA > 0 else 0.0)
        G[k] = U[:, :r].reshape(r0, n, r)
        G[k + 1] = np.einsum("ab,bic->aic", s[:r, None] * Vt[:r], G[k + 1])
    return tails


def round_block(G, lo, hi, eps, rmax, trace=None):
    """Rounding of the links inside [lo, hi] of a TT whose cores outside the
    block are orthonormal (left of lo left-, right of hi right-orthonormal):
    right-to-left orthogonalisation of cores hi..lo+1, then left-to-right
    truncation of links lo..hi-1.  ||A|| is the norm of core lo once the
    orthogonalisation is done.  Returns the relative tails."""
    d = len(G)
    for k in range(hi, lo, -1):
        right_orth(G, k)
    normA = float(np.linalg.norm(G[lo]))
    if d < 2 or normA == 0.0:
        return [0.0] * (hi - lo)
    thr = eps * normA / math.sqrt(d - 1)
    return left_sweep(G, lo, hi, thr, rmax, normA, trace)


def round_full(cores, eps, rmax, trace=None):
    """Full TT rounding (every link): round_block over [0, d-1]."""
    G = _cores(cores)
    tails = round_block(G, 0, len(G) - 1, eps, rmax, trace) if len(G) > 1 else []
    return G, tails


# --------------------------------------------------------------- predict ----
def apply_mode(G, k, M):
    """Core k <- M applied to its grid index: G'(:, j, :) = sum_i M[j, i] G(:, i, :)."""
    G[k] = np.einsum("ji,aib->ajb", M, G[k])


def add_block(pieces, lo, hi):
    """TT sum of tensor trains that share every core outside [lo, hi] (the
    TT "plus" restricted to a block): core lo concatenated along its right
    rank, core hi along its left rank, the cores between block diagonal."""
    out = [c.copy() for c in pieces[0]]
    for k in range(lo, hi + 1):
        parts = [p[k] for p in pieces]
        if k == lo and k == hi:
            raise ValueError("a block spans at least two cores")
        if k == lo:
            out[k] = np.concatenate(parts, axis=2)
        elif k == hi:
            out[k] = np.concatenate(parts, axis=0)
        else:
            n = parts[0].shape[1]
            C = np.zeros((sum(p.shape[0] for p in parts), n, sum(p.shape[2] for p in parts)))
            a = b = 0
            for p in parts:
                C[a:a + p.shape[0], :, b:b + p.shape[2]] = p
                a += p.shape[0]
                b += p.shape[2]
            out[k] = C
    return out


def shear_shifts(grid: pmf.Grid, m: int, n: int, a: float):
    """Fractional shifts s_i = a xi_{n,i} / D_m of the hat-weight shear and the
    integer shifts t with a nonzero weight."""
    s = a * grid.axes[n] / grid.delta_axis[m]
    ts = list(range(int(math.floor(s.min())), int(math.floor(s.max())) + 2))
    return s, ts


def shear_round(G, grid, m, n, a, eps, rmax, smax=10, trace=None):
    """Shear x_m += a x_n as a TT operator followed by rounding of its block
    (pieces of at most smax shifts when it spans more).  Returns (cores,
    tails)."""
    lo, hi = min(m, n), max(m, n)
    canonical(G, lo, hi)
    s, ts = shear_shifts(grid, m, n, a)
    S = len(ts)
    if S <= smax:
        G = tt.shear_operator(G, m, n, s, ts)
        return G, round_block(G, lo, hi, eps, rmax, trace)
    npieces = -(-S // smax)
    tails, pieces = [], []
    for p in range(npieces):
        u0, u1 = S * p // npieces, S * (p + 1) // npieces
        P = tt.shear_operator(G, m, n, s, ts[u0:u1])
        tails += round_block(P, lo, hi, eps, rmax, trace)
        pieces.append(P)
    G = add_block(pieces, lo, hi)
    tails += round_block(G, lo, hi, eps, rmax, trace)
    return G, tails


def mass(G, grid) -> float:
    """Sum of the TT times the cell volume (TT `sum`)."""
    return tt.full_sum(G) * grid.delta


def normalise(G, grid):
    """Scale the last core so that the TT integrates to one; returns the mass
    before scaling."""
    c = mass(G, grid)
    G[-1] = G[-1] / c
    return c


def predict(cores, grid: pmf.Grid, F, Q, eps, rmax, smax=10, trace=None):
    """TT predictive step with the re-gridded transition.  Returns (cores,
    tails of every rounding in order, mass before normalisation)."""
    Q = np.asarray(Q, dtype=np.float64)
    G = _cores(cores)
    tails = []
    for op in pmf.elementary_ops(F):
        if op[0] == "shear":
            G, t = shear_round(G, grid, op[1], op[2], op[3], eps, rmax, smax, trace)
            tails += t
        else:
            apply_mode(G, op[1], pmf.cic_matrix(grid, op[1], op[2]))
    for m in range(grid.d):
        n_m = grid.shape[m]
        apply_mode(G, m, pmf.toeplitz_kernel(pmf.gauss_kernel(grid.delta_axis[m], float(Q[m, m]), n_m),
                                             n_m))
    c = normalise(G, grid)
    return G, tails, c


# ------------------------------------------------- textbook transition ----
def transition_factor(grid: pmf.Grid, F, Q, m):
    """The mode-m factor of the textbook transition (Eq. TPMmat,
    T[j, i] = N(xi_j; F xi_i, Q) delta) for an upper bidiagonal F and a
    diagonal Q, whose Gaussian factorises over the modes:
    K_m(j, i, i') = D_m N(xi_{m,j} - F_mm xi_{m,i} - F_{m,m+1} xi_{m+1,i'}; 0, Q_mm),
    shape (N_m, N_m, N_{m+1}); (N_m, N_m) for the last mode and for a mode
    without coupling."""
    F = np.asarray(F, dtype=np.float64)
    q = float(np.asarray(Q, dtype=np.float64)[m, m])
    xm = grid.axes[m]
    coupled = m + 1 < grid.d and F[m, m + 1] != 0.0
    x = xm[:, None] - F[m, m] * xm[None, :]
    if coupled:
        x = x[:, :, None] - F[m, m + 1] * grid.axes[m + 1][None, None, :]
    return grid.delta_axis[m] * np.exp(-0.5 * x * x / q) / math.sqrt(2 * math.pi * q)


def check_bidiagonal(F, Q):
    F = np.asarray(F, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    d = F.shape[0]
    for m in range(d):
        for n in range(d):
            if F[m, n] != 0.0 and not (n == m or n == m + 1):
                raise ValueError("the exact transition needs an upper bidiagonal F")
    if np.any(Q != np.diag(np.diag(Q))):
        raise ValueError("the exact transition needs a diagonal Q")


def predict_exact(cores, grid: pmf.Grid, F, Q, eps, rmax, cross=None, trace=None):
    """TT predictive step with the textbook transition (Eqs. pdf_predII,
    TPMmat) for an upper bidiagonal F and a diagonal Q, without the
    re-gridding's interpolation: the modes' factors K_m applied in the order
    m = 0, 1, ..., each summing out i_m while i_{m+1} is still the old index.
    The TT starts in canonical form with its center at core 0; a coupled
    factor acts on the 2-site block (m, m+1) (formed exactly, or by the cross
    of oracle/cross.py when cross = {"s": rank, "sweeps": n}) and the block's
    link is rounded (round_block, center then at m + 1); an uncoupled factor
    is a matrix on core m followed by the truncating left step of the
    rounding; the last mode's factor is a matrix on the last core.  Then
    normalisation.  Returns (cores, tails, mass before normalisation)."""
    from . import cross as X
    check_bidiagonal(F, Q)
    F = np.asarray(F, dtype=np.float64)
    G = _cores(cores)
    d = len(G)
    canonical(G, 0, 0)
    tails = []
    for m in range(d - 1):
        K = transition_factor(grid, F, Q, m)
        if K.ndim == 3:
            if cross is None:
                W = np.einsum("aic,cjb->aijb", G[m], G[m + 1])
                W = np.einsum("kij,aijb->akjb", K, W)
                r0, n0, n1, r1 = W.shape
                Qm, Rm = np.linalg.qr(W.reshape(r0 * n0, n1 * r1))
                G[m] = Qm.reshape(r0, n0, -1)
                G[m + 1] = Rm.reshape(-1, n1, r1)
            else:
                blk = X.TransitionBlock([G[m], G[m + 1]], K)
                (G[m], G[m + 1]), _ = X.cross_of_block(blk, cross["s"], cross.get("sweeps", 1),
                                                       cross.get("delta", 0.05))
            tails += round_block(G, m, m + 1, eps, rmax, trace)
        else:
            apply_mode(G, m, K)
            normA = float(np.linalg.norm(G[m]))
            thr = eps * normA / math.sqrt(d - 1) if d > 1 else 0.0
            tails += left_sweep(G, m, m + 1, thr, rmax, normA, trace)
    apply_mode(G, d - 1, transition_factor(grid, F, Q, d - 1))
    c = normalise(G, grid)
    return G, tails, c


# ---------------------------------------------------------------- update ----
def _lik_factor(table, z, r, period):
    return np.exp(-0.5 * pmf.residual(z, table, period) ** 2 / r) / math.sqrt(2 * math.pi * r)


def is_block_comp(modes) -> bool:
    """Whether a component is applied as a block (by the cross or, for the
    exact reference, a dense block product): every component other than a
    one-mode one and a two-mode one on modes (0, 1)."""
    return len(modes) > 2 or (len(modes) == 2 and tuple(modes) != (0, 1))


def block_of(modes):
    """The block of cores lo..hi a component couples."""
    return min(modes), max(modes)


def block_likelihood(grid: pmf.Grid, modes, factor):
    """A component's likelihood factor (its table's shape, modes in the
    component's order) as an array over every grid index of its block."""
    lo, hi = block_of(modes)
    order = np.argsort(modes)
    f = np.transpose(factor, order)
    shape = [1] * (hi - lo + 1)
    for m in modes:
        shape[m - lo] = grid.shape[m]
    return np.broadcast_to(f.reshape(shape), tuple(grid.shape[lo:hi + 1]))


def _exact_block_product(G, lo, hi, lik):
    """Cores lo..hi <- the exact TT (ranks r_lo, full, ..., r_hi+1) of the
    block (G_lo ... G_hi) times the likelihood, by successive QR splits of
    the dense product."""
    W = G[lo]
    for k in range(lo + 1, hi + 1):
        W = np.tensordot(W, G[k], axes=([W.ndim - 1], [0]))
    W = W * lik[None, ..., None]
    r0 = W.shape[0]
    rest = W.reshape(r0, -1)
    for k in range(lo, hi):
        n = G[k].shape[1]
        Qm, Rm = np.linalg.qr(rest.reshape(r0 * n, -1))
        G[k] = Qm.reshape(r0, n, -1)
        r0 = G[k].shape[2]
        rest = Rm
    G[hi] = rest.reshape(r0, G[hi].shape[1], -1)


def update_block(G, grid, comp, z, r, eps, rmax, cross=None, trace=None):
    """Multiply a normalised TT by the likelihood factor of a block
    component (modes lo..hi) and round the block's links: the TT is put in
    canonical form with its center in the block, the block times the factor
    is formed exactly (cross None) or by the deterministic cross of
    oracle/cross.py (cross = {"s": rank, "sweeps": n}), log c is the log of
    the product's mass, and the block is rounded (round_block) and the TT
    normalised.  Returns (cores, tails, log c)."""
    from . import cross as X
    modes, table, period = pmf.unpack_comp(comp)
    lo, hi = block_of(modes)
    canonical(G, lo, hi)
    lik = block_likelihood(grid, modes, _lik_factor(table, z, r, period))
    if cross is None:
        _exact_block_product(G, lo, hi, lik)
    else:
        G[lo:hi + 1], _ = X.block_cross(G[lo:hi + 1], lik, cross["s"], cross.get("sweeps", 1),
                                        cross.get("delta", 0.05))
    logc = math.log(mass(G, grid))
    tails = round_block(G, lo, hi, eps, rmax, trace)
    normalise(G, grid)
    return G, tails, logc


def update(cores, grid: pmf.Grid, comps, z, R, eps, rmax, trace=None, cross=None):
    """TT Bayes update.  comps = [(modes, table[, period])] as for pmf.likelihood; the
    two-mode components on modes (0, 1) multiply the merged 2-site core (the
    likelihood is the product of the components, Eq. pmf_filtrace_a); one-
    and (0, 1)-components are applied first, with log c, rounding and
    normalisation; then every block component in turn (update_block), its
    log c added.  Returns (cores, tails, log c)."""
    R = np.atleast_2d(np.asarray(R, dtype=np.float64))
    z = np.atleast_1d(np.asarray(z, dtype=np.float64))
    G = _cores(cores)
    d = len(G)
    twos, blocks = [], []
    for c, comp in enumerate(comps):
        modes, table, period = pmf.unpack_comp(comp)
        r = float(R[c, c])
        if len(modes) == 1:
            m = modes[0]
            G[m] = G[m] * _lik_factor(table, z[c], r, period)[None, :, None]
        elif is_block_comp(modes):
            blocks.append((c, comp, r))
        else:
            twos.append((c, table, r, period))
    tails = []
    if not twos:
        logc = math.log(mass(G, grid))
    else:
        for k in range(d - 1, 1, -1):
            right_orth(G, k)
        W = np.einsum("ia,ajb->ijb", G[0][0], G[1])
        for c, table, r, period in twos:
            W = W * _lik_factor(table, z[c], r, period)[:, :, None]
        logc = math.log(tt.full_sum([W.reshape(1, -1, W.shape[2])] + G[2:]) * grid.delta)
        N0, N1, r2 = W.shape
        normA = float(np.linalg.norm(W))
        thr = eps * normA / math.sqrt(d - 1) if d > 1 else 0.0
        U, s, Vt = np.linalg.svd(W.reshape(N0, N1 * r2), full_matrices=False)
        rk, tail = _rank_and_tail(s, thr, rmax)
        if trace is not None:
            trace.append({"link": 0, "s": s.copy(), "thr": thr, "normA": normA, "rank": rk,
                          "rmax": rmax})
        tails.append(tail / normA)
        G[0] = U[:, :rk].reshape(1, N0, rk)
        G[1] = (s[:rk, None] * Vt[:rk]).reshape(rk, N1, r2)
        tails += left_sweep(G, 1, d - 1, thr, rmax, normA, trace)
    normalise(G, grid)
    for c, comp, r in blocks:
        G, tb, lcb = update_block(G, grid, comp, z[c], r, eps, rmax, cross, trace)
        tails += tb
        logc += lcb
    return G, tails, logc


def step(cores, grid, F, Q, comps, z, R, eps, rmax, smax=10, cross=None):
    """predict -> update.  Returns (cores, dict of tails / log c / mass)."""
    G, tp, mp = predict(cores, grid, F, Q, eps, rmax, smax)
    G, tu, logc = update(G, grid, comps, z, R, eps, rmax, cross=cross)
    return G, {"tails_predict": tp, "tails_update": tu, "tail_sum": float(sum(tp) + sum(tu)),
               "log_c": logc, "mass_pred": mp}


# --------------------------------------------------------------- moments ----
def rank_is_borderline(rec, rank, eta):
    """Whether a rank other than the oracle's on a link is a decision at the
    threshold: data whose singular values are perturbed by up to eta thr could
    take it.  Keeping more (rank > r): the tail of rank - 1 is within eta thr
    below the threshold; keeping fewer: the tail of `rank` is within eta thr
    above it.  A rank above the cap never is."""
    s, thr, r = rec["s"], rec["thr"], rec["rank"]
    if rank == r:
        return True
    tail = np.sqrt(np.concatenate([np.cumsum((s ** 2)[::-1])[::-1], [0.0]]))
    if rank < 1 or rank >= len(tail) or (rec["rmax"] is not None and rank > rec["rmax"]):
        return False
    if rank > r:
        return bool(tail[rank - 1] >= (1.0 - eta) * thr)
    return bool(tail[rank] <= (1.0 + eta) * thr)


def moments(cores, grid: pmf.Grid):
    """Point-mass mean and covariance of a TT density (unit mass assumed, as
    pmf.moments) by TT contractions: A_k^(p) = sum_i xi_{k,i}^p G_k(:, i, :),
    mean_m = A^(0) ... A_m^(1) ... A^(0), E[x_m x_n] from A_m^(1), A_n^(1)
    (A_m^(2) on the diagonal)."""
    d = grid.d
    G = [np.asarray(c, dtype=np.float64) for c in cores]
    A = [[np.einsum("aib,i->ab", G[k], grid.axes[k] ** p) for p in range(3)] for k in range(d)]

    def chain(pw):
        v = np.ones((1,))
        for k in range(d):
            v = v @ A[k][pw[k]]
        return float(v[0])

    tot = chain([0] * d)
    mean = np.array([chain([1 if k == m else 0 for k in range(d)]) for m in range(d)]) / tot
    E2 = np.zeros((d, d))
    for m in range(d):
        for n in range(m, d):
            pw = [0] * d
            if m == n:
                pw[m] = 2
            else:
                pw[m] = pw[n] = 1
            E2[m, n] = E2[n, m] = chain(pw) / tot
    return mean, E2 - np.outer(mean, mean)


def rel_distance(a, b) -> float:
    """||A - B||_F / ||B||_F of two TTs by inner products (no densification)."""
    aa, bb, ab = tt.inner(a, a), tt.inner(b, b), tt.inner(a, b)
    return math.sqrt(max(aa - 2 * ab + bb, 0.0) / bb)
