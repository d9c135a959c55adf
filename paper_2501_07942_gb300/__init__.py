"""ttgbf: tensor-train grid-based (point-mass) filtering on GB300.

Python binding of the C ABI in ``include/ttgbf.h`` (library ``libttgbf.so``
built in-tree by ``paper_2501_07942_gb300.build``).  The binding only
marshals arguments: every step of the filter runs in the library's CUDA
kernels.  PyTorch supplies device memory (the workspace and the measurement
tables) and the CUDA stream.

Method names follow the C entry points (``ttgbf_<name>``): ``predict``,
``update``, ``update_dev``, ``estimate``, ``estimate_dev``, ``free``,
``ranks``, ``stats``, ``grid_axes``, ``export_cores``, ``import_cores``,
``shear``, ``scale``, ``convolve``, ``round``, ``normalise``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libttgbf.so")

TTGBF_OK = 0
ERRORS = {
    -1: "TTGBF_EINVAL", -2: "TTGBF_ENONFINITE", -3: "TTGBF_ENOMEM", -4: "TTGBF_ECUDA",
    -5: "TTGBF_ECAPACITY", -6: "TTGBF_ESINGULAR", -7: "TTGBF_EPOISONED",
}

# Every symbol the header declares (checked by the CPU test suite).
EXPORTED = [
    "ttgbf_workspace_bytes", "ttgbf_init", "ttgbf_predict", "ttgbf_predict_exact", "ttgbf_update",
    "ttgbf_update_dev",
    "ttgbf_estimate", "ttgbf_estimate_dev", "ttgbf_free", "ttgbf_strerror", "ttgbf_ranks",
    "ttgbf_stats", "ttgbf_grid_axes", "ttgbf_export_cores", "ttgbf_densify", "ttgbf_import_cores",
    "ttgbf_shear",
    "ttgbf_scale", "ttgbf_convolve", "ttgbf_round", "ttgbf_normalise", "ttgbf_profile",
    "ttgbf_profile_read", "ttgbf_launch_count", "ttgbf_moments_noalloc", "ttgbf_fg_workspace_bytes",
    "ttgbf_fg_init", "ttgbf_fg_predict", "ttgbf_fg_predict_direct", "ttgbf_fg_update",
    "ttgbf_fg_estimate", "ttgbf_fg_density", "ttgbf_fg_free", "ttgbf_group_create",
    "ttgbf_group_step", "ttgbf_group_capture", "ttgbf_group_launch", "ttgbf_group_graph_kernels",
    "ttgbf_group_times", "ttgbf_group_graph_times", "ttgbf_group_free", "ttgbf_autotune",
    "ttgbf_adj_create", "ttgbf_adj_free", "ttgbf_adj_reset", "ttgbf_adj_save", "ttgbf_adj_load",
    "ttgbf_adj_record", "ttgbf_adj_backward", "ttgbf_adj_grads", "ttgbf_ldu_adjoint",
    "ttgbf_design_grid", "ttgbf_regrid",
]


class TTGBFError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({strerror(code)})")


class Grid(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("n", ctypes.POINTER(ctypes.c_int32)),
                ("lo", ctypes.POINTER(ctypes.c_double)), ("hi", ctypes.POINTER(ctypes.c_double))]


class Prior(ctypes.Structure):
    _fields_ = [("mean", ctypes.POINTER(ctypes.c_double)), ("var", ctypes.POINTER(ctypes.c_double))]


class Opts(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int32), ("rank_cap", ctypes.c_int32), ("eps", ctypes.c_double),
                ("max_shift_span", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t),
                ("precision", ctypes.c_int32), ("conv", ctypes.c_int32), ("parts", ctypes.c_int32),
                ("tsqr_slice_blocks", ctypes.c_int32), ("svd_threads", ctypes.c_int32),
                ("cross_rank", ctypes.c_int32), ("cross_sweeps", ctypes.c_int32),
                ("contraction", ctypes.c_int32)]


PRECISION = {"fp32": 0, "fp64": 1}  # TTGBF_PRECISION_FP32 / TTGBF_PRECISION_FP64
CONV = {"auto": 0, "dense": 1, "fft": 2}  # TTGBF_CONV_AUTO / _DENSE / _FFT
CONTRACT = {"fp32": 0, "tf32": 1, "tf32x3": 2}  # TTGBF_CONTRACT_FP32 / _TF32 / _TF32X3


class MeasComp(ctypes.Structure):
    _fields_ = [("nmodes", ctypes.c_int32), ("modes", ctypes.c_int32 * 2),
                ("htab", ctypes.c_void_p), ("period", ctypes.c_double)]


class Meas(ctypes.Structure):
    _fields_ = [("b", ctypes.c_int32), ("comp", ctypes.POINTER(MeasComp))]


class GroupStepArgs(ctypes.Structure):
    _fields_ = [("F", ctypes.POINTER(ctypes.c_double)), ("Q", ctypes.POINTER(ctypes.c_double)),
                ("h", ctypes.POINTER(Meas)), ("R", ctypes.POINTER(ctypes.c_double)),
                ("z_dev", ctypes.c_void_p), ("mean", ctypes.c_void_p), ("cov", ctypes.c_void_p),
                ("log_c", ctypes.c_void_p), ("log_lik", ctypes.c_void_p)]


class StepStats(ctypes.Structure):
    _fields_ = [("tail_sum", ctypes.c_double), ("tail_max", ctypes.c_double),
                ("mass_pred", ctypes.c_double), ("log_c", ctypes.c_double),
                ("log_lik", ctypes.c_double), ("max_rank", ctypes.c_int32),
                ("cap_hits", ctypes.c_int32)]


class KernelProf(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("flops", ctypes.c_double)]


_lib = None


def load() -> ctypes.CDLL:
    """Load libttgbf.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_2501_07942_gb300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, VP = ctypes.POINTER, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    dp = P(ctypes.c_double)
    lib.ttgbf_workspace_bytes.restype = ctypes.c_size_t
    lib.ttgbf_workspace_bytes.argtypes = [P(Grid), P(Opts)]
    lib.ttgbf_init.argtypes = [P(VP), P(Grid), P(Prior), P(Opts)]
    lib.ttgbf_predict.argtypes = [VP, dp, dp]
    lib.ttgbf_predict_exact.argtypes = [VP, dp, dp]
    lib.ttgbf_update.argtypes = [VP, P(Meas), dp, dp]
    lib.ttgbf_update_dev.argtypes = [VP, P(Meas), dp, VP]
    lib.ttgbf_estimate.argtypes = [VP, dp, dp, dp, dp]
    lib.ttgbf_estimate_dev.argtypes = [VP, VP, VP, VP, VP]
    lib.ttgbf_free.argtypes = [VP]
    lib.ttgbf_strerror.restype = ctypes.c_char_p
    lib.ttgbf_strerror.argtypes = [I]
    lib.ttgbf_ranks.argtypes = [VP, P(ctypes.c_int32)]
    lib.ttgbf_stats.argtypes = [VP, P(StepStats)]
    lib.ttgbf_grid_axes.argtypes = [VP, dp]
    lib.ttgbf_export_cores.argtypes = [VP, ctypes.c_int32, P(ctypes.c_float), ctypes.c_size_t,
                                       P(ctypes.c_int32)]
    lib.ttgbf_import_cores.argtypes = [VP, ctypes.c_int32, P(ctypes.c_float), P(ctypes.c_int32), D]
    lib.ttgbf_densify.argtypes = [VP, ctypes.c_int32, dp, ctypes.c_size_t]
    lib.ttgbf_shear.argtypes = [VP, ctypes.c_int32, ctypes.c_int32, D, ctypes.c_int32]
    lib.ttgbf_scale.argtypes = [VP, ctypes.c_int32, D]
    lib.ttgbf_convolve.argtypes = [VP, dp]
    lib.ttgbf_round.argtypes = [VP]
    lib.ttgbf_normalise.argtypes = [VP]
    lib.ttgbf_profile.argtypes = [VP, ctypes.c_int32]
    lib.ttgbf_profile_read.argtypes = [VP, P(KernelProf), ctypes.c_int32, P(ctypes.c_int32)]
    lib.ttgbf_launch_count.restype = ctypes.c_uint64
    lib.ttgbf_launch_count.argtypes = []
    lib.ttgbf_fg_workspace_bytes.restype = ctypes.c_size_t
    lib.ttgbf_fg_workspace_bytes.argtypes = [P(Grid), ctypes.c_int32]
    lib.ttgbf_fg_init.argtypes = [P(VP), P(Grid), P(Prior), ctypes.c_int32, VP, VP, ctypes.c_size_t]
    lib.ttgbf_fg_predict.argtypes = [VP, dp, dp]
    lib.ttgbf_fg_predict_direct.argtypes = [VP, dp, dp]
    lib.ttgbf_fg_update.argtypes = [VP, P(Meas), dp, dp]
    lib.ttgbf_fg_estimate.argtypes = [VP, dp, dp, dp, dp]
    lib.ttgbf_fg_density.argtypes = [VP, dp, ctypes.c_size_t]
    lib.ttgbf_fg_free.argtypes = [VP]
    lib.ttgbf_group_create.argtypes = [P(VP), P(VP), ctypes.c_int32, VP]
    lib.ttgbf_group_step.argtypes = [VP, P(GroupStepArgs)]
    lib.ttgbf_group_capture.argtypes = [VP, P(GroupStepArgs), ctypes.c_int32]
    lib.ttgbf_group_launch.argtypes = [VP]
    lib.ttgbf_group_graph_kernels.restype = ctypes.c_uint64
    lib.ttgbf_group_graph_kernels.argtypes = [VP]
    lib.ttgbf_group_times.argtypes = [VP, P(ctypes.c_float)]
    lib.ttgbf_group_graph_times.argtypes = [VP, P(ctypes.c_float)]
    lib.ttgbf_group_free.argtypes = [VP]
    lib.ttgbf_autotune.argtypes = [P(Grid), P(Prior), P(Opts), dp, dp, ctypes.c_int32, ctypes.c_char_p,
                                   P(Opts), dp]
    lib.ttgbf_adj_create.argtypes = [P(VP), VP, ctypes.c_int32, ctypes.c_int32]
    for name in ("ttgbf_adj_free", "ttgbf_adj_reset", "ttgbf_adj_backward"):
        getattr(lib, name).argtypes = [VP]
    for name in ("ttgbf_adj_save", "ttgbf_adj_load", "ttgbf_adj_record"):
        getattr(lib, name).argtypes = [VP, ctypes.c_int32]
    lib.ttgbf_adj_grads.argtypes = [VP, dp, dp, dp, ctypes.c_int32]
    lib.ttgbf_ldu_adjoint.argtypes = [ctypes.c_int32, dp, dp, dp, dp, dp]
    lib.ttgbf_design_grid.argtypes = [ctypes.c_int32, ctypes.c_int32, dp, dp, dp, dp, ctypes.c_double, dp, dp]
    lib.ttgbf_regrid.argtypes = [VP, dp, dp]
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load().ttgbf_strerror(int(code)).decode()


def launch_count() -> int:
    """Kernel launches the library made in this process (ttgbf_launch_count)."""
    return int(load().ttgbf_launch_count())


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _check(rc: int, where: str):
    if rc != TTGBF_OK:
        raise TTGBFError(rc, where)


def _grid(lo, hi, n):
    n = np.ascontiguousarray(np.asarray(n, dtype=np.int32))
    lo, hi = _f64(lo), _f64(hi)
    g = Grid(len(n), n.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dptr(lo), _dptr(hi))
    return g, (n, lo, hi)


def workspace_bytes(lo, hi, n, batch=1, rank_cap=16, eps=1e-6, max_shift_span=0,
                    precision="fp32", conv="auto", cross_rank=0) -> int:
    g, keep = _grid(lo, hi, n)
    o = Opts(batch, rank_cap, eps, max_shift_span, None, None, 0, PRECISION[precision], CONV[conv],
             0, 0, 0, int(cross_rank), 0)
    return int(load().ttgbf_workspace_bytes(ctypes.byref(g), ctypes.byref(o)))


class FullGridFilter:
    """The plain full-grid point-mass filter on the GPU (``ttgbf_fg_*``): one
    filter, dense float32 (precision=32) or float64 (precision=64) density."""

    def __init__(self, lo, hi, n, prior_mean, prior_var, precision=32, stream=None, device="cuda"):
        import torch
        self._lib = load()
        self.d = len(n)
        self.n = [int(v) for v in n]
        self.precision = int(precision)
        g, self._gkeep = _grid(lo, hi, n)
        self._stream = torch.cuda.current_stream(device) if stream is None else stream
        nbytes = self._lib.ttgbf_fg_workspace_bytes(ctypes.byref(g), self.precision)
        if nbytes == 0:
            raise TTGBFError(-1, "ttgbf_fg_workspace_bytes")
        self.workspace = torch.empty(int(nbytes), dtype=torch.uint8, device=device)
        pm, pv = _f64(prior_mean), _f64(prior_var)
        pr = Prior(_dptr(pm), _dptr(pv))
        self._ctx = ctypes.c_void_p()
        _check(self._lib.ttgbf_fg_init(ctypes.byref(self._ctx), ctypes.byref(g), ctypes.byref(pr),
                                       self.precision, ctypes.c_void_p(self._stream.cuda_stream),
                                       ctypes.c_void_p(self.workspace.data_ptr()), int(nbytes)),
               "ttgbf_fg_init")

    def predict(self, F, Q):
        F, Q = _f64(F), _f64(Q)
        _check(self._lib.ttgbf_fg_predict(self._ctx, _dptr(F), _dptr(Q)), "ttgbf_fg_predict")

    def predict_direct(self, F, Q):
        F, Q = _f64(F), _f64(Q)
        _check(self._lib.ttgbf_fg_predict_direct(self._ctx, _dptr(F), _dptr(Q)),
               "ttgbf_fg_predict_direct")

    def update(self, comps, R, z):
        """comps: [(modes, device table of float32 / float64 matching precision)]."""
        m, keep = TTFilter._meas(comps)
        R, z = _f64(R), _f64(z)
        _check(self._lib.ttgbf_fg_update(self._ctx, ctypes.byref(m), _dptr(R), _dptr(z)),
               "ttgbf_fg_update")

    def estimate(self):
        mean = np.zeros(self.d)
        cov = np.zeros((self.d, self.d))
        lc = np.zeros(1)
        ll = np.zeros(1)
        _check(self._lib.ttgbf_fg_estimate(self._ctx, _dptr(mean), _dptr(cov), _dptr(lc), _dptr(ll)),
               "ttgbf_fg_estimate")
        return mean, cov, float(lc[0]), float(ll[0])

    def density(self):
        out = np.zeros(int(np.prod(self.n)))
        _check(self._lib.ttgbf_fg_density(self._ctx, _dptr(out), out.size), "ttgbf_fg_density")
        return out.reshape(self.n)

    def free(self):
        if getattr(self, "_ctx", None) is not None and self._ctx.value:
            self._lib.ttgbf_fg_free(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class TTFilter:
    """A batch of TT point-mass filters sharing one grid and model
    (``ttgbf_init``).  Device memory comes from a torch uint8 workspace."""

    def __init__(self, lo, hi, n, prior_mean, prior_var, batch=1, rank_cap=16, eps=1e-6,
                 max_shift_span=0, stream=None, device="cuda", precision="fp32", conv="auto",
                 parts=0, tsqr_slice_blocks=0, svd_threads=0, cross_rank=0, cross_sweeps=0,
                 contraction="fp32"):
        """precision: "fp32" (R factors and SVDs of the rounding in float32) or
        "fp64" (those of the truncating stages in float64), ttgbf_opts.precision.
        conv: "auto", "dense" or "fft", how the Gaussian kernel is applied
        (ttgbf_opts.conv).  parts, tsqr_slice_blocks, svd_threads: the launch
        configuration (0 = the library's default; see ttgbf_autotune).
        cross_rank, cross_sweeps: the TT cross of likelihood factors on several
        modes (ttgbf_opts.cross_rank; 0 = not available).  contraction: "fp32"
        (CUDA cores), "tf32" or "tf32x3" (tensor cores), the arithmetic of the
        core contractions (ttgbf_opts.contraction)."""
        import torch
        self._lib = load()
        self.d = len(n)
        self.n = [int(v) for v in n]
        self.batch = int(batch)
        self.precision = precision
        g, self._gkeep = _grid(lo, hi, n)
        self._stream = torch.cuda.current_stream(device) if stream is None else stream
        o = Opts(self.batch, int(rank_cap), float(eps), int(max_shift_span),
                 ctypes.c_void_p(self._stream.cuda_stream), None, 0, PRECISION[precision],
                 CONV[conv], int(parts), int(tsqr_slice_blocks), int(svd_threads), int(cross_rank),
                 int(cross_sweeps), CONTRACT[contraction])
        nbytes = self._lib.ttgbf_workspace_bytes(ctypes.byref(g), ctypes.byref(o))
        pm, pv = _f64(prior_mean), _f64(prior_var)
        pr = Prior(_dptr(pm), _dptr(pv))
        self._ctx = ctypes.c_void_p()
        if nbytes == 0:
            # ttgbf_init validates every argument on the host before it
            # allocates or launches anything: it names the reason
            rc = self._lib.ttgbf_init(ctypes.byref(self._ctx), ctypes.byref(g), ctypes.byref(pr),
                                      ctypes.byref(o))
            if rc == 0:
                self._lib.ttgbf_free(self._ctx)
                self._ctx = ctypes.c_void_p()
            raise TTGBFError(rc if rc != 0 else -1, "ttgbf_workspace_bytes")
        self.workspace = torch.empty(int(nbytes), dtype=torch.uint8, device=device)
        o.workspace = ctypes.c_void_p(self.workspace.data_ptr())
        o.workspace_bytes = int(nbytes)
        _check(self._lib.ttgbf_init(ctypes.byref(self._ctx), ctypes.byref(g), ctypes.byref(pr),
                                    ctypes.byref(o)), "ttgbf_init")

    # ----------------------------------------------------------- hot path
    def predict(self, F, Q):
        F, Q = _f64(F), _f64(Q)
        _check(self._lib.ttgbf_predict(self._ctx, _dptr(F), _dptr(Q)), "ttgbf_predict")

    def predict_exact(self, F, Q):
        """ttgbf_predict_exact: the textbook transition for an upper
        bidiagonal F (needs cross_rank > 0)."""
        F, Q = _f64(F), _f64(Q)
        _check(self._lib.ttgbf_predict_exact(self._ctx, _dptr(F), _dptr(Q)), "ttgbf_predict_exact")

    @staticmethod
    def _meas(comps):
        arr = (MeasComp * len(comps))()
        for i, (modes, tab, *period) in enumerate(comps):
            arr[i].nmodes = len(modes)
            arr[i].modes[0] = int(modes[0])
            # one mode: -1; a pair: the second; three or more (consecutive): the last
            arr[i].modes[1] = int(modes[-1]) if len(modes) > 1 else -1
            arr[i].htab = ctypes.c_void_p(tab.data_ptr())
            arr[i].period = float(period[0]) if period else 0.0
        return Meas(len(comps), arr), arr

    def update(self, comps, R, z):
        """comps: [(modes, device float32 table[, period])], period > 0 for an
        angle-like component (ttgbf_meas_comp.period); R: (b, b); z: host
        (batch, b)."""
        m, keep = self._meas(comps)
        R, z = _f64(R), _f64(z)
        _check(self._lib.ttgbf_update(self._ctx, ctypes.byref(m), _dptr(R), _dptr(z)), "ttgbf_update")

    def update_dev(self, comps, R, z_dev):
        """z_dev: device float32 tensor (batch, b)."""
        m, keep = self._meas(comps)
        R = _f64(R)
        _check(self._lib.ttgbf_update_dev(self._ctx, ctypes.byref(m), _dptr(R),
                                          ctypes.c_void_p(z_dev.data_ptr())), "ttgbf_update_dev")

    def estimate(self):
        mean = np.zeros((self.batch, self.d))
        cov = np.zeros((self.batch, self.d, self.d))
        lc = np.zeros(self.batch)
        ll = np.zeros(self.batch)
        _check(self._lib.ttgbf_estimate(self._ctx, _dptr(mean), _dptr(cov), _dptr(lc), _dptr(ll)),
               "ttgbf_estimate")
        return mean, cov, lc, ll

    def estimate_dev(self, mean, cov, log_c, log_lik):
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        _check(self._lib.ttgbf_estimate_dev(self._ctx, ptr(mean), ptr(cov), ptr(log_c), ptr(log_lik)),
               "ttgbf_estimate_dev")

    # -------------------------------------------------------- diagnostics
    def ranks(self) -> np.ndarray:
        r = np.zeros((self.batch, self.d + 1), dtype=np.int32)
        _check(self._lib.ttgbf_ranks(self._ctx, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))),
               "ttgbf_ranks")
        return r

    def stats(self):
        arr = (StepStats * self.batch)()
        _check(self._lib.ttgbf_stats(self._ctx, arr), "ttgbf_stats")
        keys = [f[0] for f in StepStats._fields_]
        return [{k: getattr(s, k) for k in keys} for s in arr]

    def grid_axes(self):
        a = np.zeros(sum(self.n))
        _check(self._lib.ttgbf_grid_axes(self._ctx, _dptr(a)), "ttgbf_grid_axes")
        out, at = [], 0
        for nk in self.n:
            out.append(a[at:at + nk].copy())
            at += nk
        return out

    def export_cores(self, f=0):
        r = np.zeros(self.d + 1, dtype=np.int32)
        cap = sum(self.n) * 160 * 160 + 16
        buf = np.zeros(cap, dtype=np.float32)
        _check(self._lib.ttgbf_export_cores(self._ctx, int(f),
                                            buf.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                            cap, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))),
               "ttgbf_export_cores")
        cores, at = [], 0
        for k in range(self.d):
            cnt = int(r[k]) * self.n[k] * int(r[k + 1])
            cores.append(buf[at:at + cnt].reshape(int(r[k]), self.n[k], int(r[k + 1])).copy())
            at += cnt
        return cores

    def densify(self, f=0, cap=None):
        """Filter f's density on the full grid (float64, shape n), contracted
        on the device; small grids only."""
        total = int(np.prod(self.n))
        out = np.zeros(total if cap is None else int(cap), dtype=np.float64)
        _check(self._lib.ttgbf_densify(self._ctx, int(f), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       out.size), "ttgbf_densify")
        return out[:total].reshape(self.n)

    def import_cores(self, f, cores, log_lik=0.0):
        r = np.array([1] + [int(c.shape[2]) for c in cores], dtype=np.int32)
        buf = np.ascontiguousarray(np.concatenate([np.asarray(c, dtype=np.float32).ravel()
                                                   for c in cores]))
        _check(self._lib.ttgbf_import_cores(self._ctx, int(f),
                                            buf.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                            r.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                            float(log_lik)), "ttgbf_import_cores")

    def shear(self, m, n, a, do_round=True):
        _check(self._lib.ttgbf_shear(self._ctx, int(m), int(n), float(a), int(bool(do_round))),
               "ttgbf_shear")

    def scale(self, m, lam):
        _check(self._lib.ttgbf_scale(self._ctx, int(m), float(lam)), "ttgbf_scale")

    def convolve(self, q):
        q = _f64(q)
        _check(self._lib.ttgbf_convolve(self._ctx, _dptr(q)), "ttgbf_convolve")

    def regrid(self, lo, hi):
        """ttgbf_regrid: every filter's density onto the grid [lo, hi] (same cell
        counts), then renormalised (Alg. 4 step 5)."""
        lo, hi = _f64(lo), _f64(hi)
        _check(self._lib.ttgbf_regrid(self._ctx, _dptr(lo), _dptr(hi)), "ttgbf_regrid")

    def round(self):
        _check(self._lib.ttgbf_round(self._ctx), "ttgbf_round")

    def normalise(self):
        _check(self._lib.ttgbf_normalise(self._ctx), "ttgbf_normalise")

    def profile(self, enable=True):
        _check(self._lib.ttgbf_profile(self._ctx, int(bool(enable))), "ttgbf_profile")

    def profile_read(self):
        arr = (KernelProf * 16)()
        cnt = ctypes.c_int32()
        _check(self._lib.ttgbf_profile_read(self._ctx, arr, 16, ctypes.byref(cnt)), "ttgbf_profile_read")
        return {arr[i].name.decode(): {"launches": arr[i].launches, "ms": arr[i].ms, "flops": arr[i].flops}
                for i in range(cnt.value)}

    def free(self):
        if getattr(self, "_ctx", None) is not None and self._ctx.value:
            self._lib.ttgbf_free(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class TTFilterGroup:
    """Several TTFilter batches of different shape stepped together
    (ttgbf_group_*): one call enqueues predict -> update -> estimate of every
    batch with their operations interleaved; a horizon of steps can be
    recorded into a CUDA graph (capture) and launched as a whole (launch)."""

    def __init__(self, filters, stream=None, device="cuda"):
        import torch
        self._lib = load()
        self.filters = list(filters)
        # a created stream: the legacy default stream cannot be recorded into a graph
        self._stream = torch.cuda.Stream(device) if stream is None else stream
        arr = (ctypes.c_void_p * len(self.filters))(*[f._ctx.value for f in self.filters])
        self._g = ctypes.c_void_p()
        _check(self._lib.ttgbf_group_create(ctypes.byref(self._g), arr, len(self.filters),
                                            ctypes.c_void_p(self._stream.cuda_stream)),
               "ttgbf_group_create")

    def _args(self, models):
        """models: per filter (F, Q, comps, R, z_dev, mean, cov, log_c, log_lik)
        with device tensors (or None for outputs)."""
        keep = []
        arr = (GroupStepArgs * len(models))()
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        for i, (F, Q, comps, R, z, mean, cov, lc, ll) in enumerate(models):
            F, Q, R = _f64(F), _f64(Q), _f64(R)
            m, marr = TTFilter._meas(comps)
            keep += [F, Q, R, m, marr]
            arr[i].F, arr[i].Q, arr[i].R = _dptr(F), _dptr(Q), _dptr(R)
            arr[i].h = ctypes.pointer(m)
            arr[i].z_dev, arr[i].mean, arr[i].cov = ptr(z), ptr(mean), ptr(cov)
            arr[i].log_c, arr[i].log_lik = ptr(lc), ptr(ll)
        return arr, keep

    def step(self, models):
        arr, keep = self._args(models)
        _check(self._lib.ttgbf_group_step(self._g, arr), "ttgbf_group_step")

    def capture(self, models, steps):
        arr, keep = self._args(models)
        _check(self._lib.ttgbf_group_capture(self._g, arr, int(steps)), "ttgbf_group_capture")
        self._horizon = int(steps)

    def launch(self):
        _check(self._lib.ttgbf_group_launch(self._g), "ttgbf_group_launch")

    def graph_kernels(self) -> int:
        return int(self._lib.ttgbf_group_graph_kernels(self._g))

    def times(self):
        """Per filter batch: ms from the last step's start to its end."""
        ms = (ctypes.c_float * len(self.filters))()
        _check(self._lib.ttgbf_group_times(self._g, ms), "ttgbf_group_times")
        return list(ms)

    def graph_times(self):
        """Per step of the last graph launch and per filter batch: ms from the
        step's start to the batch's end of it (steps x batches array)."""
        H, n = getattr(self, "_horizon", 0), len(self.filters)
        ms = (ctypes.c_float * max(1, H * n))()
        _check(self._lib.ttgbf_group_graph_times(self._g, ms), "ttgbf_group_graph_times")
        return np.array(ms[:H * n], dtype=np.float64).reshape(H, n)

    def free(self):
        if getattr(self, "_g", None) is not None and self._g.value:
            self._lib.ttgbf_group_free(self._g)
            self._g = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def autotune(lo, hi, n, prior_mean, prior_var, F, Q, batch=1, rank_cap=16, eps=1e-6,
             max_shift_span=0, precision="fp32", conv="auto", steps=3, cache_path=None,
             cache_only=False, contraction="fp32"):
    """ttgbf_autotune: the fastest launch configuration (parts,
    tsqr_slice_blocks, svd_threads) for this batch shape and model, and its
    time per predictive step in ms.  cache_only: look the shape up in
    cache_path without timing anything (LookupError when it is not there)."""
    if cache_only:
        steps = 0
    lib = load()
    g, gkeep = _grid(lo, hi, n)
    pm, pv = _f64(prior_mean), _f64(prior_var)
    pr = Prior(_dptr(pm), _dptr(pv))
    o = Opts(int(batch), int(rank_cap), float(eps), int(max_shift_span), None, None, 0,
             PRECISION[precision], CONV[conv], 0, 0, 0, 0, 0, CONTRACT[contraction])
    best = Opts()
    ms = ctypes.c_double()
    F, Q = _f64(F), _f64(Q)
    cp = cache_path.encode() if cache_path else None
    rc = lib.ttgbf_autotune(ctypes.byref(g), ctypes.byref(pr), ctypes.byref(o), _dptr(F), _dptr(Q),
                            int(steps), cp, ctypes.byref(best), ctypes.byref(ms))
    if cache_only and rc == -1:
        raise LookupError("shape not in the autotuner's cache")
    _check(rc, "ttgbf_autotune")
    return {"parts": best.parts, "tsqr_slice_blocks": best.tsqr_slice_blocks,
            "svd_threads": best.svd_threads}, ms.value


def ldu_adjoint(F, GL, GD, GU):
    """ttgbf_ldu_adjoint (host only): dl/dF from the gradients with respect to
    the strictly lower L, the diagonal D and the strictly upper U of F = L D U."""
    F, GL, GD, GU = _f64(F), _f64(GL), _f64(GD), _f64(GU)
    d = F.shape[0]
    out = np.zeros((d, d))
    _check(load().ttgbf_ldu_adjoint(d, _dptr(F), _dptr(GL), _dptr(GD), _dptr(GU), _dptr(out)),
           "ttgbf_ldu_adjoint")
    return out


class Adjoint:
    """Reverse pass of a TTFilter batch (``ttgbf_adj_*``): checkpoints of the
    filter state, recording of segments of steps and the backward sweep (the
    adjoint recursion of the filter equations with the adjoint density as a
    rounded tensor train)."""

    def __init__(self, filt, steps, slots):
        self._lib = load()
        self.filt = filt
        self._a = ctypes.c_void_p()
        _check(self._lib.ttgbf_adj_create(ctypes.byref(self._a), filt._ctx, int(steps), int(slots)),
               "ttgbf_adj_create")

    def reset(self):
        _check(self._lib.ttgbf_adj_reset(self._a), "ttgbf_adj_reset")

    def save(self, slot):
        _check(self._lib.ttgbf_adj_save(self._a, int(slot)), "ttgbf_adj_save")

    def load(self, slot):
        _check(self._lib.ttgbf_adj_load(self._a, int(slot)), "ttgbf_adj_load")

    def record(self, on):
        _check(self._lib.ttgbf_adj_record(self._a, 1 if on else 0), "ttgbf_adj_record")

    def backward(self):
        _check(self._lib.ttgbf_adj_backward(self._a), "ttgbf_adj_backward")

    def grads(self, n_r):
        B, d = self.filt.batch, self.filt.d
        dF = np.zeros((B, d, d))
        dQ = np.zeros((B, d))
        dR = np.zeros((B, max(1, n_r)))
        _check(self._lib.ttgbf_adj_grads(self._a, _dptr(dF), _dptr(dQ), _dptr(dR), int(n_r)),
               "ttgbf_adj_grads")
        return dF, dQ, dR[:, :n_r]

    def free(self):
        if getattr(self, "_a", None) is not None and self._a.value:
            self._lib.ttgbf_adj_free(self._a)
            self._a = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _run_segment(filt, F, Q, comps, R, z_dev, k0, k1):
    for k in range(k0, k1):
        filt.predict(F, Q)
        filt.update_dev(comps, R, z_dev[k])


def _make_loglik_function():
    import torch

    class _LogLik(torch.autograd.Function):
        """l_b = sum_k log c_k of every filter of a batch run from its prior
        over the measurements z (steps, batch, b), as a function of F, q =
        diag(Q) and r = diag(R); the backward pass is ttgbf_adj_* with
        checkpoints every `every` steps (each segment recomputed once)."""

        @staticmethod
        def forward(ctx, F, q, r, spec):
            Fn = F.detach().cpu().double().numpy()
            Qn = np.diag(q.detach().cpu().double().numpy())
            Rn = np.diag(r.detach().cpu().double().numpy())
            filt = spec["make_filter"]()
            K, every = spec["z"].shape[0], spec["every"]
            nseg = -(-K // every)
            adj = Adjoint(filt, every, nseg)
            for s in range(nseg):
                adj.save(s)
                _run_segment(filt, Fn, Qn, spec["comps"], Rn, spec["z"], s * every, min(K, (s + 1) * every))
            ll = filt.estimate()[3]
            ctx.state = (filt, adj, Fn, Qn, Rn, spec, nseg)
            return torch.tensor(ll, dtype=torch.float64)

        @staticmethod
        def backward(ctx, g):
            filt, adj, Fn, Qn, Rn, spec, nseg = ctx.state
            K, every = spec["z"].shape[0], spec["every"]
            adj.reset()
            for s in range(nseg - 1, -1, -1):
                adj.load(s)
                adj.record(True)
                _run_segment(filt, Fn, Qn, spec["comps"], Rn, spec["z"], s * every, min(K, (s + 1) * every))
                adj.record(False)
                adj.backward()
            dF, dQ, dR = adj.grads(len(spec["comps"]))
            w = g.detach().cpu().double().numpy()
            gF = torch.tensor(np.einsum("b,bij->ij", w, dF))
            gq = torch.tensor(np.einsum("b,bi->i", w, dQ))
            gr = torch.tensor(np.einsum("b,bi->i", w, dR))
            adj.free()
            filt.free()
            ctx.state = None
            return gF, gq, gr, None

    return _LogLik


_LOGLIK = None


def log_likelihood(F, q, r, *, lo, hi, n, prior_mean, prior_var, comps, z, rank_cap=16, eps=1e-6,
                   max_shift_span=0, precision="fp32", conv="dense", checkpoint_every=20,
                   device="cuda"):
    """Differentiable log-likelihood of the TT filter: l_b = sum_k log c_k
    (Eq. pmf_filtrace_b) of a batch of filters run from the prior over the
    measurements z (device float32, steps x batch x b), as a torch function of
    F (d x d), q = diag(Q) and r = diag(R) (float64 CPU tensors).  The
    gradient comes from the reverse pass (ttgbf_adj_*: the adjoint recursion
    of the filter equations in TT form) with per-segment checkpoints every
    `checkpoint_every` steps (each segment is run a second time, recorded,
    in the backward pass)."""
    global _LOGLIK
    if _LOGLIK is None:
        _LOGLIK = _make_loglik_function()
    B = int(z.shape[1])

    def make_filter():
        return TTFilter(lo, hi, n, prior_mean, prior_var, batch=B, rank_cap=rank_cap, eps=eps,
                        max_shift_span=max_shift_span, device=device, precision=precision, conv=conv,
                        parts=1)

    spec = {"make_filter": make_filter, "comps": comps, "z": z, "every": int(checkpoint_every)}
    return _LOGLIK.apply(F, q, r, spec)


def design_grid(F, Q, means, covs, kappa=5.0):
    """ttgbf_design_grid (host only): the grid box of Alg. 4 for a batch from
    its filtering means (batch, d) and covariances (batch, d, d): returns
    (lo, hi)."""
    F, Q = _f64(F), _f64(Q)
    means = _f64(np.atleast_2d(means))
    covs = _f64(np.asarray(covs, dtype=np.float64).reshape(means.shape[0], F.shape[0], F.shape[0]))
    d, B = F.shape[0], means.shape[0]
    lo, hi = np.zeros(d), np.zeros(d)
    _check(load().ttgbf_design_grid(d, B, _dptr(F), _dptr(Q), _dptr(means), _dptr(covs), float(kappa),
                                    _dptr(lo), _dptr(hi)), "ttgbf_design_grid")
    return lo, hi
