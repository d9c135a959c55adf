"""Dense FP64 point-mass filter (the oracle).  Test infrastructure only.

Everything here is written from arXiv 2501.07942 Sec. 2 ("Grid-Based
Estimation") and the step structure of Alg. 2/3, in float64, on the full grid.
It is deliberately plain: no blocking, fusion or reordering beyond what each
definition states.

Conventions (readings of the paper, applied identically on the CUDA path):

* Grid (Sec. 2, Eq. pdf_pm): equidistant, cell-centred.  Mode m has N_m cells
  of width D_m = (hi_m - lo_m)/N_m on [lo_m, hi_m]; point i sits at
  xi_{m,i} = lo_m + (i + 1/2) D_m; the cell volume is delta = prod_m D_m.
  Weights P are density values; they integrate to one: sum(P) * delta = 1.
* Predictive step, re-gridded transition T_RG (the grid stays fixed and
  axis-aligned; the paper re-grids by TT interpolation, Alg. 3 step 5 and
  Alg. 4 step 5, which it leaves unspecified):
  F = L D U (no pivoting).  The push-forward x -> F x is applied as U's
  elementary shears (rows ascending, couplings ascending), then D's per-axis
  scalings, then L's shears (rows descending, couplings ascending).  A shear
  x_m += a x_n moves the mass of cell i_m to the fractional index
  i_m + a xi_{n,i_n}/D_m with hat (linear-interpolation) weights; a scaling
  x_m <- lam x_m moves each cell centre to lam xi_{m,i} with the same hat
  weights (cloud-in-cell).  Then the separable Gaussian transition kernel
  (diagonal Q) is applied as the linear convolution of Eq. tpmconvFFT with
  kappa_m(t) = D_m N(D_m t; 0, q_m), t = -(N_m-1)..(N_m-1), truncated to the
  grid (zero outside: mass that leaves the grid is lost), then the density is
  renormalised (Alg. 2 step 4 "Normalize").
* Predictive step, textbook transition T (Eqs. pdf_predII, TPMmat):
  P'(j) = sum_i N(xi_j; F xi_i, Q) P(i) delta, then renormalised.
* Update (Eqs. pmf_filtrace_a/b): L(i) = prod_c N(z_c; h_c(xi_i), R_cc);
  c = sum_i L(i) P(i) delta; P <- L P / c; log c is accumulated.
* Estimate: point-mass moments, mean = sum xi P delta,
  cov = sum (xi - mean)(xi - mean)^T P delta.
"""
from __future__ import annotations

import math

import numpy as np


# ---------------------------------------------------------------- grid ----
class Grid:
    """Equidistant cell-centred grid (Sec. 2, Eq. pdf_pm; Sec. 4 first bullet:
    stored axis per axis, N_1 + ... + N_d numbers)."""

    def __init__(self, lo, hi, n):
        self.lo = np.asarray(lo, dtype=np.float64).copy()
        self.hi = np.asarray(hi, dtype=np.float64).copy()
        self.n = np.asarray(n, dtype=np.int64).copy()
        if not (self.lo.shape == self.hi.shape == self.n.shape and self.lo.ndim == 1):
            raise ValueError("lo, hi, n must be 1-D arrays of equal length")
        if np.any(self.n < 1) or np.any(self.hi <= self.lo):
            raise ValueError("need n >= 1 and hi > lo on every axis")
        self.d = int(self.lo.size)
        self.delta_axis = (self.hi - self.lo) / self.n
        self.axes = [self.lo[m] + (np.arange(self.n[m]) + 0.5) * self.delta_axis[m]
                     for m in range(self.d)]
        self.delta = float(np.prod(self.delta_axis))
        self.shape = tuple(int(v) for v in self.n)

    def points(self) -> np.ndarray:
        """All grid points, shape (N_1*...*N_d, d), C order (last mode fastest)."""
        mesh = np.meshgrid(*self.axes, indexing="ij")
        return np.stack([g.ravel() for g in mesh], axis=1)


def normalise(P: np.ndarray, grid: Grid):
    """Scale weights so that sum(P) * delta = 1 (Sec. 2: the PMD integrates
    to one).  Returns (P / mass, mass)."""
    mass = float(P.sum()) * grid.delta
    if not mass > 0.0:
        raise FloatingPointError("density has no positive mass")
    return P / mass, mass


def gaussian_on_grid(grid: Grid, mean, cov) -> np.ndarray:
    """Point evaluation of N(x; mean, cov) at every grid point."""
    mean = np.asarray(mean, dtype=np.float64)
    cov = np.asarray(cov, dtype=np.float64)
    if np.all(cov == np.diag(np.diag(cov))):
        # diagonal covariance: the density is the product of its 1-D marginals
        out = np.ones(())
        for m in range(grid.d):
            v = cov[m, m]
            f = np.exp(-0.5 * (grid.axes[m] - mean[m]) ** 2 / v) / math.sqrt(2 * math.pi * v)
            out = np.multiply.outer(out, f)
        return out
    X = grid.points() - mean
    icov = np.linalg.inv(cov)
    quad = np.einsum("pi,ij,pj->p", X, icov, X)
    logn = -0.5 * quad - 0.5 * grid.d * math.log(2 * math.pi) - 0.5 * np.linalg.slogdet(cov)[1]
    return np.exp(logn).reshape(grid.shape)


def prior(grid: Grid, mean, cov) -> np.ndarray:
    """Initial PMD (Alg. 2 step 1): the prior pdf evaluated at the grid points,
    then normalised."""
    return normalise(gaussian_on_grid(grid, mean, cov), grid)[0]


# ----------------------------------------------- re-gridded prediction ----
def ldu(F) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """F = L diag(D) U with L unit lower and U unit upper triangular, computed
    by Doolittle elimination without pivoting.  Raises on a zero pivot."""
    A = np.asarray(F, dtype=np.float64)
    d = A.shape[0]
    L = np.eye(d)
    U = np.eye(d)
    D = np.zeros(d)
    scale = max(1.0, float(np.abs(A).max()))
    for k in range(d):
        D[k] = A[k, k] - sum(L[k, j] * D[j] * U[j, k] for j in range(k))
        if abs(D[k]) <= 1e-12 * scale:
            raise np.linalg.LinAlgError(f"zero pivot at {k}: F has no LDU factorisation")
        for i in range(k + 1, d):
            L[i, k] = (A[i, k] - sum(L[i, j] * D[j] * U[j, k] for j in range(k))) / D[k]
            U[k, i] = (A[k, i] - sum(L[k, j] * D[j] * U[j, i] for j in range(k))) / D[k]
    return L, D, U


def elementary_ops(F):
    """The canonical sequence of elementary re-gridding operations for x -> F x.

    Returns a list of ("shear", m, n, a) meaning x_m += a x_n, and
    ("scale", m, lam) meaning x_m <- lam x_m, in the order they are applied:
    U's shears (rows m ascending; couplings n > m ascending), D's scalings
    (m ascending), L's shears (rows m descending; couplings n < m ascending).
    Zero couplings and unit scalings are skipped (they are identities)."""
    L, D, U = ldu(F)
    d = len(D)
    ops = []
    for m in range(d):
        for n in range(m + 1, d):
            if U[m, n] != 0.0:
                ops.append(("shear", m, n, float(U[m, n])))
    for m in range(d):
        if D[m] != 1.0:
            ops.append(("scale", m, float(D[m])))
    for m in range(d - 1, -1, -1):
        for n in range(m):
            if L[m, n] != 0.0:
                ops.append(("shear", m, n, float(L[m, n])))
    return ops


def hat(t):
    """Linear-interpolation (hat) weight, max(0, 1 - |t|)."""
    return np.maximum(0.0, 1.0 - np.abs(t))


def _shifted_add(out, src, axis, t, w):
    """out[..., j, ...] += w * src[..., j - t, ...] along `axis` for the j whose
    source index j - t lies on the grid (zero outside the grid)."""
    n = src.shape[axis]
    if abs(t) >= n or w == 0.0:
        return
    dst = [slice(None)] * src.ndim
    srs = [slice(None)] * src.ndim
    dst[axis] = slice(max(0, t), n + min(0, t))
    srs[axis] = slice(max(0, -t), n - max(0, t))
    out[tuple(dst)] += w * src[tuple(srs)]


def shear(P: np.ndarray, grid: Grid, m: int, n: int, a: float) -> np.ndarray:
    """Push-forward of the PMD under x_m <- x_m + a x_n (m != n):
    P'(.., j_m, .., i_n, ..) = sum_{i_m} hat(j_m - i_m - a xi_{n,i_n}/D_m) P(.., i_m, .., i_n, ..).
    For each i_n only the two integer offsets t = j_m - i_m next to the
    fractional shift s carry weight."""
    if m == n:
        raise ValueError("a shear couples two different modes")
    # Work on a copy with mode n first so that each i_n slice is contiguous.
    src_all = np.ascontiguousarray(np.moveaxis(P, n, 0))
    out = np.zeros_like(src_all)
    ax = m if m < n else m - 1   # axis m inside a slice with axis n removed
    for i_n in range(grid.shape[n]):
        s = a * grid.axes[n][i_n] / grid.delta_axis[m]
        k = math.floor(s)
        for t in (k, k + 1):
            _shifted_add(out[i_n], src_all[i_n], ax, t, float(hat(t - s)))
    return np.ascontiguousarray(np.moveaxis(out, 0, n))


def cic_matrix(grid: Grid, m: int, lam: float) -> np.ndarray:
    """N_m x N_m cloud-in-cell matrix W[j, i] = hat(j - u_i) with
    u_i = (lam xi_{m,i} - lo_m)/D_m - 1/2, the fractional index of the moved
    cell centre."""
    xi = grid.axes[m]
    u = (lam * xi - grid.lo[m]) / grid.delta_axis[m] - 0.5
    j = np.arange(grid.shape[m], dtype=np.float64)
    return hat(j[:, None] - u[None, :])


def apply_along(P: np.ndarray, M: np.ndarray, axis: int) -> np.ndarray:
    """P'(.., j, ..) = sum_i M[j, i] P(.., i, ..) along one axis."""
    return np.moveaxis(np.tensordot(M, P, axes=([1], [axis])), 0, axis)


def scale_axis(P: np.ndarray, grid: Grid, m: int, lam: float) -> np.ndarray:
    """Push-forward under x_m <- lam x_m by cloud-in-cell."""
    return apply_along(P, cic_matrix(grid, m, lam), m)


def gauss_kernel(delta_m: float, q_m: float, n_m: int) -> np.ndarray:
    """kappa(t) = D N(D t; 0, q) for t = -(n-1)..(n-1): the middle row of the
    TPM of Eq. TPMmat for a 1-D random walk with variance q (Eq. tpmconvFFT's
    T^mid)."""
    t = np.arange(-(n_m - 1), n_m, dtype=np.float64)
    return delta_m * np.exp(-0.5 * (delta_m * t) ** 2 / q_m) / math.sqrt(2 * math.pi * q_m)


def toeplitz_kernel(kappa: np.ndarray, n_m: int) -> np.ndarray:
    """K[j, i] = kappa(j - i): linear convolution truncated to the grid."""
    idx = np.arange(n_m)
    return kappa[(idx[:, None] - idx[None, :]) + (n_m - 1)]


def convolve_axis(P: np.ndarray, grid: Grid, m: int, q_m: float) -> np.ndarray:
    """P'(.., j_m, ..) = sum_{i_m} kappa_m(j_m - i_m) P(.., i_m, ..)."""
    n_m = grid.shape[m]
    K = toeplitz_kernel(gauss_kernel(grid.delta_axis[m], q_m, n_m), n_m)
    return apply_along(P, K, m)


def regrid(P: np.ndarray, grid: Grid, F) -> np.ndarray:
    """Apply R_F = L D U (the re-gridding part of T_RG) as elementary ops."""
    for op in elementary_ops(F):
        if op[0] == "shear":
            P = shear(P, grid, op[1], op[2], op[3])
        else:
            P = scale_axis(P, grid, op[1], op[2])
    return P


def predict_rg(P: np.ndarray, grid: Grid, F, Q):
    """Predictive PMD with the re-gridded transition T_RG = K_Q o R_F, then
    normalisation.  Q must be diagonal.  Returns (P', mass before
    normalisation)."""
    Q = np.asarray(Q, dtype=np.float64)
    if np.any(Q != np.diag(np.diag(Q))):
        raise ValueError("the separable transition needs a diagonal Q")
    P = regrid(P, grid, F)
    for m in range(grid.d):
        P = convolve_axis(P, grid, m, float(Q[m, m]))
    return normalise(P, grid)


def predict_textbook(P: np.ndarray, grid: Grid, F, Q):
    """Predictive PMD by the direct sum of Eq. pdf_predII with the dense TPM of
    Eq. TPMmat, T[j, i] = N(xi_j; F xi_i, Q) delta, then normalisation.
    O(N^2) memory: small grids only.  Returns (P', mass before normalisation)."""
    F = np.asarray(F, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    X = grid.points()
    FX = X @ F.T
    iQ = np.linalg.inv(Q)
    lognorm = -0.5 * grid.d * math.log(2 * math.pi) - 0.5 * np.linalg.slogdet(Q)[1]
    diff = X[:, None, :] - FX[None, :, :]
    T = np.exp(-0.5 * np.einsum("jik,kl,jil->ji", diff, iQ, diff) + lognorm) * grid.delta
    Pn = (T @ P.ravel()).reshape(grid.shape)
    return normalise(Pn, grid)


# ------------------------------------------------------------- update ----
def unpack_comp(comp):
    """(modes, table) or (modes, table, period) -> (modes, table, period),
    period 0 for an ordinary component."""
    modes, table = comp[0], comp[1]
    return modes, table, float(comp[2]) if len(comp) > 2 else 0.0


def residual(z, h, period=0.0) -> np.ndarray:
    """z - h.  For an angle-like component (period > 0: the four-quadrant
    bearing of Sec. 5 in degrees has period 360) the residual is the
    representative of z - h modulo the period nearest to zero, i.e. the
    angle is compared on its nearer branch."""
    r = np.asarray(z, dtype=np.float64) - np.asarray(h, dtype=np.float64)
    if period > 0.0:
        r = r - period * np.round(r / period)
    return r


def likelihood(grid: Grid, comps, z, R) -> np.ndarray:
    """Likelihood tensor L (Sec. 4, fourth bullet) of a measurement whose
    components each depend on one or two modes:
    L(i) = prod_c N(z_c; h_c(xi_i), R_cc).  comps[c] = (modes, table) or
    (modes, table, period) with table[i_m] or table[i_m, i_n] = h_c at the
    grid points (period: see residual).  R diagonal."""
    R = np.atleast_2d(np.asarray(R, dtype=np.float64))
    z = np.atleast_1d(np.asarray(z, dtype=np.float64))
    if np.any(R != np.diag(np.diag(R))):
        raise ValueError("R must be diagonal")
    L = np.ones(grid.shape)
    for c, comp in enumerate(comps):
        modes, table, period = unpack_comp(comp)
        r = float(R[c, c])
        lc = np.exp(-0.5 * residual(z[c], table, period) ** 2 / r) / math.sqrt(2 * math.pi * r)
        shape = [1] * grid.d
        for k, m in enumerate(modes):
            shape[m] = grid.shape[m]
        if len(modes) == 2 and modes[0] > modes[1]:
            lc = lc.T
        L = L * lc.reshape(shape)
    return L


def update(P: np.ndarray, grid: Grid, L: np.ndarray):
    """Bayes update, Eqs. pmf_filtrace_a/b: c = sum L P delta, P <- L P / c.
    Returns (P', log c)."""
    c = float((L * P).sum()) * grid.delta
    if not c > 0.0:
        raise FloatingPointError("measurement has zero likelihood on the grid")
    return L * P / c, math.log(c)


# ----------------------------------------------------------- estimate ----
def moments(P: np.ndarray, grid: Grid):
    """Point-mass mean and covariance: mean = sum xi P delta,
    cov = sum (xi - mean)(xi - mean)^T P delta."""
    d = grid.d
    mean = np.zeros(d)
    marg = []
    for m in range(d):
        other = tuple(k for k in range(d) if k != m)
        pm = P.sum(axis=other) * grid.delta
        marg.append(pm)
        mean[m] = float(pm @ grid.axes[m])
    cov = np.zeros((d, d))
    for m in range(d):
        for n in range(m, d):
            if m == n:
                cov[m, m] = float(marg[m] @ (grid.axes[m] - mean[m]) ** 2)
            else:
                other = tuple(k for k in range(d) if k not in (m, n))
                pmn = P.sum(axis=other) * grid.delta
                cov[m, n] = cov[n, m] = float(
                    (grid.axes[m] - mean[m]) @ pmn @ (grid.axes[n] - mean[n]))
    return mean, cov


# ------------------------------------------------------------- filter ----
def run_filter(grid: Grid, prior_mean, prior_cov, F, Q, comps, R, zs,
               transition: str = "rg", P0=None, callback=None):
    """Run the point-mass filter for len(zs) steps: per step, predict, update
    with z_k, estimate (step unit and order: predict -> update -> estimate;
    the prior is the density at k = 0 and there is no z_0).

    Returns dict(means (K, d), covs (K, d, d), log_c (K,), log_lik, P)."""
    P = prior(grid, prior_mean, prior_cov) if P0 is None else P0
    means, covs, logc = [], [], []
    pred = predict_rg if transition == "rg" else predict_textbook
    for k, z in enumerate(zs):
        P, _ = pred(P, grid, F, Q)
        P, lc = update(P, grid, likelihood(grid, comps, z, R))
        m, c = moments(P, grid)
        means.append(m)
        covs.append(c)
        logc.append(lc)
        if callback is not None:
            callback(k, P)
    return {"means": np.array(means), "covs": np.array(covs), "log_c": np.array(logc),
            "log_lik": float(np.sum(logc)), "P": P}
