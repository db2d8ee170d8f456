"""Helpers for the GPU tests: run the CUDA path through the C-ABI binding and
compare its bidiagonal with the oracle's as singular values."""
import numpy as np

import oracle

# tolerances on singular values, relative to ||A||_2 = sigma_max
TOL_F64 = 1e-11
TOL_F32 = 2e-4


def run_gpu(ab: np.ndarray, b: int, dtype: str = "f64", tuning=None, stream=None):
    import torch
    import paper_2510_12705_gb300 as bb
    tdt = torch.float64 if dtype == "f64" else torch.float32
    band = torch.from_numpy(np.ascontiguousarray(ab)).to(device="cuda", dtype=tdt)
    n = band.shape[0]
    d = torch.empty(n, device="cuda", dtype=tdt)
    e = torch.empty(max(n - 1, 1), device="cuda", dtype=tdt)
    if tuning is None:
        bb.band_to_bidiag(band, b, d, e, stream=stream)
    else:
        bb.band_to_bidiag_ex(band, b, d, e, tuning=tuning, stream=stream)
    status = bb.bb_device_status(stream, reset=True)
    return (d.double().cpu().numpy(), e[: n - 1].double().cpu().numpy(), status)


def sigma_err(d, e, sigma_ref):
    s = oracle.bidiag_sigma(np.asarray(d, np.float64), np.asarray(e, np.float64))
    return float(np.max(np.abs(s - sigma_ref)) / max(sigma_ref[0], 1e-300)), s
