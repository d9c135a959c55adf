"""The allocation-free entry point ttgbf_moments_noalloc, called through the C
ABI, must give the moments that ttgbf_estimate gives for the same TT
densities.  It exists for callers that cannot call cudaMalloc (allocation is
forbidden while a framework records a CUDA graph, or the caller runs with a
fixed memory budget); its scratch is a static device array inside the
library.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import synth

from gpu_util import device_tables, lib_module, make_filter

pytestmark = pytest.mark.gpu

MOMENT_ATOL = 1e-6  # the moment tolerance of the other GPU tests


def _bind(lib, G):
    fn = lib.ttgbf_moments_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int32, ctypes.POINTER(G.Grid), ctypes.POINTER(ctypes.c_void_p),
                   ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p, ctypes.c_int32,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return fn


def test_noalloc_moments_match_estimate():
    import torch
    G = lib_module()
    lib = G.load()
    fn = _bind(lib, G)
    model = synth.config2(n=24)
    B, d = 3, model.d
    f = make_filter(G, model, batch=B)
    comps = device_tables(model, f.grid_axes())
    zs = np.stack([synth.simulate(model, mc, steps=2)[1] for mc in (11, 12, 13)], axis=1)
    for k in range(2):
        f.predict(model.F, model.Q)
        f.update(comps, model.R, zs[k])
    mean_ref, cov_ref, _, _ = f.estimate()
    ranks = f.ranks()
    rmax = int(ranks.max())
    # the caller's own copy of the cores: core k of filter b at base_k + b * stride_k
    strides = [max(int(ranks[b, k] * model.n[k] * ranks[b, k + 1]) for b in range(B)) for k in range(d)]
    bufs = [torch.zeros(B, strides[k], dtype=torch.float32, device="cuda") for k in range(d)]
    for b in range(B):
        for k, core in enumerate(f.export_cores(b)):
            bufs[k][b, :core.size] = torch.from_numpy(core.ravel()).cuda()
    ranks_dev = torch.tensor(ranks, dtype=torch.int32, device="cuda")
    mass = torch.empty(B, dtype=torch.float64, device="cuda")
    mean = torch.empty(B, d, dtype=torch.float64, device="cuda")
    cov = torch.empty(B, d, d, dtype=torch.float64, device="cuda")
    g, keep = G._grid(model.lo, model.hi, model.n)
    cores_arr = (ctypes.c_void_p * d)(*[t.data_ptr() for t in bufs])
    stride_arr = (ctypes.c_int64 * d)(*strides)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):  # two calls in a row share the static scratch array
        mass.fill_(float("nan"))
        mean.fill_(float("nan"))
        cov.fill_(float("nan"))
        rc = fn(B, ctypes.byref(g), cores_arr, stride_arr, ranks_dev.data_ptr(), rmax, mass.data_ptr(),
                mean.data_ptr(), cov.data_ptr(), stream)
        assert rc == 0, G.strerror(rc)
        torch.cuda.synchronize()
        np.testing.assert_allclose(mean.cpu().numpy(), mean_ref, rtol=0, atol=MOMENT_ATOL)
        np.testing.assert_allclose(cov.cpu().numpy(), cov_ref, rtol=0, atol=MOMENT_ATOL)
        np.testing.assert_allclose(mass.cpu().numpy(), 1.0, rtol=0, atol=1e-5)
    # sizes beyond the static array are rejected before any launch
    assert fn(B, ctypes.byref(g), cores_arr, stride_arr, ranks_dev.data_ptr(), 65, mass.data_ptr(),
              mean.data_ptr(), cov.data_ptr(), stream) == -5
    assert fn(100000, ctypes.byref(g), cores_arr, stride_arr, ranks_dev.data_ptr(), 64,
              mass.data_ptr(), mean.data_ptr(), cov.data_ptr(), stream) == -5
