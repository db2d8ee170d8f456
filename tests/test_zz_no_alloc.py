"""The allocation-free entry point (band_to_bidiag_noalloc) against the regular
one.  It exists for callers that cannot allocate device memory when they call
the reduction (a stream capture that must not contain allocation nodes, an
external allocator that owns the device memory); it runs the same kernels on a
fixed 16 MiB device array owned by the library.  This file is collected last
so that a run stopping at the first failure has run every other test first.
"""
import ctypes

import numpy as np
import pytest

import bandgen
from gpu_util import TOL_F32, TOL_F64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bb():
    from paper_2510_12705_gb300 import build
    build.build()
    import paper_2510_12705_gb300 as m
    return m


def _run(bb, ab, b, dtype, noalloc):
    import torch
    band = torch.from_numpy(ab).to("cuda", dtype)
    n = band.shape[0]
    d = torch.full((n,), float("nan"), device="cuda", dtype=dtype)
    e = torch.full((max(n - 1, 1),), float("nan"), device="cuda", dtype=dtype)
    if noalloc:
        # straight through the C ABI
        L = bb.lib()
        f = L.band_to_bidiag_noalloc
        f.restype = ctypes.c_int
        f.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                      ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        rc = f(n, b, bb._dtype_code(dtype), band.data_ptr(), band.shape[1], d.data_ptr(),
               e.data_ptr(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == bb.BB_OK, bb.status_string(rc)
    else:
        bb.band_to_bidiag(band, b, d, e)
    torch.cuda.synchronize()
    assert bb.bb_device_status(reset=True) == 0
    return d.double().cpu().numpy(), e[: n - 1].double().cpu().numpy()


@pytest.mark.parametrize("dtype_name", ["f64", "f32"])
def test_noalloc_matches_regular_entry_point_twice(bb, dtype_name):
    import torch
    dtype = torch.float64 if dtype_name == "f64" else torch.float32
    tol = TOL_F64 if dtype_name == "f64" else TOL_F32
    # two calls in a row on different problems: the shared scratch must be
    # cleared by each call
    for (n, b, seed) in [(2000, 48, 1), (1500, 64, 2)]:
        ab = bandgen.random_band(n, b, seed=seed)
        d_ref, e_ref = _run(bb, ab, b, dtype, noalloc=False)
        d, e = _run(bb, ab, b, dtype, noalloc=True)
        scale = max(np.max(np.abs(d_ref)), np.max(np.abs(e_ref)))
        assert np.max(np.abs(d - d_ref)) <= tol * scale
        assert np.max(np.abs(e - e_ref)) <= tol * scale


def test_noalloc_rejects_problems_beyond_its_scratch(bb):
    L = bb.lib()
    L.band_to_bidiag_noalloc_max_bytes.restype = ctypes.c_size_t
    cap = L.band_to_bidiag_noalloc_max_bytes()
    assert cap == 16 << 20
    # n = 32768, b = 128 in FP64 needs ~43 MB of workspace: rejected up front
    assert bb.band_to_bidiag_workspace_size(32768, 128, bb.BB_F64) > cap
    f = L.band_to_bidiag_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    rc = f(32768, 128, bb.BB_F64, 256, 129, 256, 256, None)
    assert rc == bb.BB_ERR_WORKSPACE
