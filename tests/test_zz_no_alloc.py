"""The allocation-free entry point ttgbf_moments_noalloc, called through the C
ABI.  It exists for callers that cannot call cudaMalloc (allocation is
forbidden while a framework records a CUDA graph, or the caller runs with a
fixed memory budget inside another framework's pool); its scratch is a
static device array inside the library.

Its mass, mean and covariance must equal the oracle's point-mass moments of
the same densified TT cores, and the moments ttgbf_estimate gives for them,
within the moment tolerance of the other GPU tests, on two calls in a row
(every call shares the static array).  A second case fills the array almost
to its limit with rank-64 cores (the largest rank it takes).  This file is
collected last on purpose."""
import ctypes

import numpy as np
import pytest

import synth
from oracle import pmf, tt

from gpu_util import device_tables, lib_module, make_filter

pytestmark = pytest.mark.gpu

MOMENT_ATOL = 1e-6  # the moment tolerance of the other GPU tests
SCRATCH_DOUBLES = (16 << 20) // 8  # TTGBF_NOALLOC_SCRATCH_BYTES / sizeof(double)
MAX_RANK = 64  # TTGBF_NOALLOC_MAX_RANK


def _bind(lib, G):
    fn = lib.ttgbf_moments_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int32, ctypes.POINTER(G.Grid), ctypes.POINTER(ctypes.c_void_p),
                   ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p, ctypes.c_int32,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return fn


def _oracle_moments(cores, grid):
    """Mass, mean and covariance of the densified TT by the oracle's
    definitions (the density divided by its mass first)."""
    P = tt.densify([np.asarray(c, dtype=np.float64) for c in cores])
    mass = float(P.sum()) * grid.delta
    mean, cov = pmf.moments(P / mass, grid)
    return mass, mean, cov


class _Caller:
    """The caller's own device copy of B filters' cores (core k of filter b at
    base_k + b * stride_k) and output buffers."""

    def __init__(self, G, model_lo, model_hi, n, cores_per_filter):
        import torch
        self.G = G
        self.B = len(cores_per_filter)
        self.d = d = len(n)
        ranks = np.array([[1] + [int(c.shape[2]) for c in cs] for cs in cores_per_filter],
                         dtype=np.int32)
        self.rmax = int(ranks.max())
        self.strides = [max(int(cs[k].size) for cs in cores_per_filter) for k in range(d)]
        self.bufs = [torch.zeros(self.B, self.strides[k], dtype=torch.float32, device="cuda")
                     for k in range(d)]
        for b, cs in enumerate(cores_per_filter):
            for k, core in enumerate(cs):
                self.bufs[k][b, :core.size] = torch.from_numpy(
                    np.ascontiguousarray(core, dtype=np.float32).ravel()).cuda()
        self.ranks_dev = torch.tensor(ranks, dtype=torch.int32, device="cuda")
        self.mass = torch.empty(self.B, dtype=torch.float64, device="cuda")
        self.mean = torch.empty(self.B, d, dtype=torch.float64, device="cuda")
        self.cov = torch.empty(self.B, d, d, dtype=torch.float64, device="cuda")
        self.g, self._keep = G._grid(model_lo, model_hi, n)
        self.cores_arr = (ctypes.c_void_p * d)(*[t.data_ptr() for t in self.bufs])
        self.stride_arr = (ctypes.c_int64 * d)(*self.strides)
        self.stream = torch.cuda.current_stream().cuda_stream

    def call(self, fn, batch=None, rank_max=None):
        for t in (self.mass, self.mean, self.cov):
            t.fill_(float("nan"))
        return fn(self.B if batch is None else batch, ctypes.byref(self.g), self.cores_arr,
                  self.stride_arr, self.ranks_dev.data_ptr(),
                  self.rmax if rank_max is None else rank_max, self.mass.data_ptr(),
                  self.mean.data_ptr(), self.cov.data_ptr(), self.stream)

    def results(self):
        import torch
        torch.cuda.synchronize()
        return self.mass.cpu().numpy(), self.mean.cpu().numpy(), self.cov.cpu().numpy()


def test_noalloc_moments_match_oracle_and_estimate():
    G = lib_module()
    fn = _bind(G.load(), G)
    model = synth.config2(n=24)
    B = 3
    f = make_filter(G, model, batch=B)
    comps = device_tables(model, f.grid_axes())
    zs = np.stack([synth.simulate(model, mc, steps=2)[1] for mc in (11, 12, 13)], axis=1)
    for k in range(2):
        f.predict(model.F, model.Q)
        f.update(comps, model.R, zs[k])
    mean_est, cov_est, _, _ = f.estimate()
    cores = [f.export_cores(b) for b in range(B)]
    grid = pmf.Grid(model.lo, model.hi, model.n)
    ref = [_oracle_moments(cs, grid) for cs in cores]
    caller = _Caller(G, model.lo, model.hi, model.n, cores)
    for _ in range(2):  # two calls in a row share the static scratch array
        rc = caller.call(fn)
        assert rc == 0, G.strerror(rc)
        mass, mean, cov = caller.results()
        for b in range(B):
            np.testing.assert_allclose(mass[b], ref[b][0], rtol=0, atol=MOMENT_ATOL)
            np.testing.assert_allclose(mean[b], ref[b][1], rtol=0, atol=MOMENT_ATOL)
            np.testing.assert_allclose(cov[b], ref[b][2], rtol=0, atol=MOMENT_ATOL)
        np.testing.assert_allclose(mean, mean_est, rtol=0, atol=MOMENT_ATOL)
        np.testing.assert_allclose(cov, cov_est, rtol=0, atol=MOMENT_ATOL)
    # sizes beyond the static array are rejected before any launch
    assert caller.call(fn, rank_max=MAX_RANK + 1) == -5
    assert caller.call(fn, batch=100000, rank_max=MAX_RANK) == -5


def test_noalloc_rank64_batch_near_scratch_limit():
    """Ranks at TTGBF_NOALLOC_MAX_RANK and a batch whose float64 scratch
    (batch x d x 3 x 64^2 doubles) just fits the static array: 42 filters of
    d = 4 use 98.4 % of it; 43 do not fit and are rejected."""
    G = lib_module()
    fn = _bind(G.load(), G)
    d, N, r = 4, 8, MAX_RANK
    B = SCRATCH_DOUBLES // (d * 3 * r * r)
    assert B == 42
    lo, hi = np.full(d, -2.0), np.full(d, 2.0)
    rng = np.random.default_rng([77, 1, 0])
    rk = [1, r, r, r, 1]
    cores = [[rng.uniform(0.05, 1.0, size=(rk[k], N, rk[k + 1])).astype(np.float32)
              for k in range(d)] for _ in range(B)]
    grid = pmf.Grid(lo, hi, np.full(d, N))
    ref = [_oracle_moments(cs, grid) for cs in cores]
    caller = _Caller(G, lo, hi, np.full(d, N), cores)
    assert caller.rmax == r
    for _ in range(2):
        rc = caller.call(fn)
        assert rc == 0, G.strerror(rc)
        mass, mean, cov = caller.results()
        for b in range(B):
            np.testing.assert_allclose(mass[b] / ref[b][0], 1.0, rtol=0, atol=1e-12)
            np.testing.assert_allclose(mean[b], ref[b][1], rtol=0, atol=MOMENT_ATOL)
            np.testing.assert_allclose(cov[b], ref[b][2], rtol=0, atol=MOMENT_ATOL)
    assert caller.call(fn, batch=B + 1) == -5
