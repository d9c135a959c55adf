"""System models and seeded trajectories for the benchmark workloads.

Every random draw uses numpy's PCG64 through ``np.random.default_rng`` with a
structured seed ``[config, stream, index]`` so that the oracle side and the
CUDA side read identical inputs.

Workloads (shapes of the paper's illustrations, Sec. 5, scaled in d):

* config 1: d=2, 64x64 on [-10,10]^2, prior N(0, 4 I), F=[[0.9,0.1],[0,0.9]],
  Q=0.1 I, z=[x_1, sin x_2] + v, R=0.05 I, 20 steps; linear variant z = x + v.
* config 2: d=4, 128^4 on [-8,8]^4, prior N(0, I) (not stated; reading),
  F = 0.95 I + 0.05 U with U upper triangular (diagonal included), entries
  U(-1,1), Q=0.05 I, z = ||x[0:2]|| + v, R=0.01, 50 steps, 100 Monte Carlo runs.
* config 3: d in {6, 8}, 256 points per axis; positions (even modes) on
  [-40,40], velocities (odd modes) on [-10,10]; prior N(0, diag(4, 1, ...));
  F = blockdiag([[1, 0.1], [0, 1]]); Q_mm ~ U(0.01, 0.1); z_i = x_{2i}^2/20 + v_i,
  R = 0.02 I; 100 steps.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def _rng(*key) -> np.random.Generator:
    return np.random.default_rng(list(key))


# Measurement component functions h_c(coordinates of its modes).
def h_identity(x):
    return np.asarray(x, dtype=np.float64)


def h_sin(x):
    return np.sin(np.asarray(x, dtype=np.float64))


def h_range(x, y):
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    return np.sqrt(x * x + y * y)


def h_bearing_deg(x, y):
    """Four-quadrant angle of (x, y) from the origin, in degrees."""
    return np.degrees(np.arctan2(np.asarray(y, dtype=np.float64), np.asarray(x, dtype=np.float64)))


def h_square20(x):
    x = np.asarray(x, dtype=np.float64)
    return x * x / 20.0


@dataclass
class Model:
    """A linear-dynamics, additive-Gaussian-noise model (Eqs. asx/asz with
    f(x) = F x) with a measurement made of components on one or two modes."""
    name: str
    lo: np.ndarray
    hi: np.ndarray
    n: np.ndarray
    m0: np.ndarray
    P0: np.ndarray
    F: np.ndarray
    Q: np.ndarray
    R: np.ndarray
    comps: list = field(default_factory=list)   # [(modes tuple, function[, period])]
    steps: int = 10
    eps: float = 1e-6
    rank_cap: int = 16
    config_id: int = 0

    @property
    def d(self) -> int:
        return int(len(self.lo))

    @property
    def b(self) -> int:
        return len(self.comps)

    def h(self, x: np.ndarray) -> np.ndarray:
        """Full measurement function h(x) for one state vector."""
        return np.array([float(fn(*[x[m] for m in modes])) for modes, fn, *_ in self.comps])

    def tables(self, axes):
        """Measurement components evaluated on grid axes supplied by the
        caller: [(modes, table)] with table of shape (N_m,), (N_m, N_n), ...
        (one axis per mode of the component, in its order);
        a component declared with a period (an angle) keeps it as a third
        entry, (modes, table, period)."""
        out = []
        for modes, fn, *period in self.comps:
            k = len(modes)
            args = [np.asarray(axes[m], dtype=np.float64).reshape([-1 if t == j else 1 for t in range(k)])
                    for j, m in enumerate(modes)]
            out.append((modes, fn(*args), *period))
        return out


def simulate(model: Model, mc: int, steps: int | None = None):
    """Seeded truth and measurements: x_0 ~ N(m0, P0); for k = 1..K:
    x_k = F x_{k-1} + w_{k-1}, z_k = h(x_k) + v_k.  Returns (x (K+1, d), z (K, b))."""
    K = model.steps if steps is None else steps
    rng = _rng(model.config_id, 2, mc)
    d = model.d
    x = np.zeros((K + 1, d))
    x[0] = rng.multivariate_normal(model.m0, model.P0)
    z = np.zeros((K, model.b))
    Lq = np.linalg.cholesky(model.Q)
    Lr = np.linalg.cholesky(model.R)
    for k in range(1, K + 1):
        x[k] = model.F @ x[k - 1] + Lq @ rng.standard_normal(d)
        z[k - 1] = model.h(x[k]) + Lr @ rng.standard_normal(model.b)
    return x, z


def config1(linear: bool = False) -> Model:
    comps = [((0,), h_identity), ((1,), h_identity if linear else h_sin)]
    return Model(name="config1-linear" if linear else "config1",
                 lo=np.full(2, -10.0), hi=np.full(2, 10.0), n=np.full(2, 64),
                 m0=np.zeros(2), P0=4.0 * np.eye(2),
                 F=np.array([[0.9, 0.1], [0.0, 0.9]]), Q=0.1 * np.eye(2),
                 R=0.05 * np.eye(2), comps=comps, steps=20, eps=1e-6, rank_cap=16,
                 config_id=1)


def config1_linear() -> Model:
    return config1(linear=True)


def config2_F() -> np.ndarray:
    rng = _rng(2, 1, 0)
    U = np.triu(rng.uniform(-1.0, 1.0, size=(4, 4)))
    return 0.95 * np.eye(4) + 0.05 * U


def config2(n: int = 128) -> Model:
    return Model(name="config2", lo=np.full(4, -8.0), hi=np.full(4, 8.0), n=np.full(4, n),
                 m0=np.zeros(4), P0=np.eye(4), F=config2_F(), Q=0.05 * np.eye(4),
                 R=np.array([[0.01]]), comps=[((0, 1), h_range)], steps=50,
                 eps=1e-6, rank_cap=16, config_id=2)


def h_range3(x, y, z):
    return np.sqrt(x * x + y * y + z * z)


def range3(n: int = 128) -> Model:
    """Config 2's model (grid, prior, F, Q) with a likelihood that couples
    three modes: the range over the first three coordinates,
    z = ||x[0:3]|| + v, R = 0.02, 50 steps (the workload of the TT cross for
    factors on three or more modes)."""
    base = config2(n)
    return Model(name="range3", lo=base.lo, hi=base.hi, n=base.n, m0=base.m0, P0=base.P0, F=base.F,
                 Q=base.Q, R=np.array([[0.02]]), comps=[((0, 1, 2), h_range3)], steps=50, eps=1e-6,
                 rank_cap=16, config_id=7)


def radar(n: int = 128) -> Model:
    """The 2-D radar model of the paper's numerical study (Sec. 5): position
    x_{k+1} = [[1.1, 0.1], [-0.2, 1.1]] x_k + w, Q = I, range and bearing (in
    degrees, an angle of period 360) from the origin with R = diag(1, 0.1),
    10 steps.  Initial condition and grid are not stated there: prior
    N([20, 20], 4 I) (the bearing then turns clockwise from about 45 to
    between -35 and -60 degrees over the 10 steps, far from the +-180 cut),
    first grid the prior mean +- 10."""
    m0 = np.array([20.0, 20.0])
    return Model(name="radar", lo=m0 - 10.0, hi=m0 + 10.0, n=np.full(2, n), m0=m0, P0=4.0 * np.eye(2),
                 F=np.array([[1.1, 0.1], [-0.2, 1.1]]), Q=np.eye(2), R=np.diag([1.0, 0.1]),
                 comps=[((0, 1), h_range), ((0, 1), h_bearing_deg, 360.0)], steps=10, eps=1e-6, rank_cap=16,
                 config_id=6)


def config3(d: int = 6, n: int = 256) -> Model:
    if d % 2:
        raise ValueError("config 3 has an even state dimension")
    rng = _rng(3, 1, d)
    lo = np.array([-40.0 if m % 2 == 0 else -10.0 for m in range(d)])
    hi = -lo
    F = np.eye(d)
    for i in range(d // 2):
        F[2 * i, 2 * i + 1] = 0.1
    Q = np.diag(rng.uniform(0.01, 0.1, size=d))
    P0 = np.diag([4.0 if m % 2 == 0 else 1.0 for m in range(d)])
    comps = [((2 * i,), h_square20) for i in range(d // 2)]
    return Model(name=f"config3-d{d}", lo=lo, hi=hi, n=np.full(d, n), m0=np.zeros(d), P0=P0,
                 F=F, Q=Q, R=0.02 * np.eye(d // 2), comps=comps, steps=100, eps=1e-5,
                 rank_cap=32, config_id=3)


def random_index_bumps_tt(n, terms: int, seed: int, dtype=np.float64):
    """A seeded positive TT of rank `terms`: the sum of `terms` separable bumps
    exp(-(i - c)^2 / (2 w^2)) in index space with random centre, width and
    weight per term and mode (block-diagonal cores).  Input data only."""
    rng = _rng(9, 1, seed)
    d = len(n)
    cores = []
    for k in range(d):
        nk = int(n[k])
        r0 = 1 if k == 0 else terms
        r1 = 1 if k == d - 1 else terms
        G = np.zeros((r0, nk, r1), dtype=np.float64)
        i = np.arange(nk, dtype=np.float64)
        for t in range(terms):
            c = rng.uniform(0.3 * nk, 0.7 * nk)
            w = rng.uniform(0.06 * nk, 0.15 * nk)
            a = rng.uniform(0.5, 1.5)
            v = a * np.exp(-0.5 * ((i - c) / w) ** 2)
            a0 = 0 if k == 0 else t
            a1 = 0 if k == d - 1 else t
            G[a0, :, a1] += v
        cores.append(G.astype(dtype))
    return cores


def config4(n_filters: int = 512, seed: int = 0):
    """Uneven batch of independent filters: each filter draws its state
    dimension d in {3..6}, points per axis N in {64, 128, 256} and rank cap in
    {8, 16, 32}; filters with the same (d, N, cap) form one group with one
    model, on [-8, 8]^d with prior N(0, 4 I), config 2's range measurement on
    modes (0, 1) (for N = 256: z = x_0 + v, since the two-mode update splits a
    2-site core whose first mode holds at most 160 points), Q_mm ~ U(0.01, 0.1),
    R ~ U(0.005, 0.02), and a random stable
    F of spectral radius 0.9 drawn in factored form F = c L D U: L, U unit
    triangular with off-diagonal entries U(-a, a), D_mm ~ U(0.7, 1),
    c = 0.9 / rho(L D U) (c rescales D only, so F's LDU factors are c D with
    the same L and U).  The bound a = (2 S - 3) D_x / (2 x_max), D_x the grid
    spacing, x_max = 8, S = min(10, 160 / cap), keeps every coupling's shift
    a x / D_x within 2 S - 3 cells, so no elementary shear of the re-gridding
    spans more than 2 S integer shifts (two expansions of S at most).
    Returns [(Model, filter ids)], one entry per group, sorted by shape."""
    rng = _rng(4, 0, seed)
    ds = rng.integers(3, 7, size=n_filters)
    Ns = rng.choice([64, 128, 256], size=n_filters)
    caps = rng.choice([8, 16, 32], size=n_filters)
    groups = {}
    for f in range(n_filters):
        groups.setdefault((int(ds[f]), int(Ns[f]), int(caps[f])), []).append(f)
    out = []
    for (d, N, cap), ids in sorted(groups.items()):
        g = _rng(4, 1, d * 10000 + N * 10 + cap // 8)
        S = min(10, 160 // cap)
        a = (2 * S - 3) * (16.0 / N) / (2 * 8.0)
        L = np.eye(d) + np.tril(g.uniform(-a, a, size=(d, d)), -1)
        U = np.eye(d) + np.triu(g.uniform(-a, a, size=(d, d)), 1)
        D = np.diag(g.uniform(0.7, 1.0, size=d))
        F0 = L @ D @ U
        F = 0.9 * F0 / max(abs(np.linalg.eigvals(F0)))
        model = Model(name=f"config4-d{d}-N{N}-r{cap}", lo=np.full(d, -8.0), hi=np.full(d, 8.0),
                      n=np.full(d, N), m0=np.zeros(d), P0=4.0 * np.eye(d), F=F,
                      Q=np.diag(g.uniform(0.01, 0.1, size=d)), R=np.array([[g.uniform(0.005, 0.02)]]),
                      comps=[((0, 1), h_range)] if N <= 160 else [((0,), h_identity)], steps=50,
                      eps=1e-6, rank_cap=cap, config_id=4)
        out.append((model, ids))
    return out
