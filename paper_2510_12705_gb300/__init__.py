"""GB300 (sm_103a) band -> bidiagonal reduction: thin binding over the C ABI.

Every step of the reduction runs in the CUDA kernels of ``libbandbidiag.so``
(``include/band_bidiag.h``); this module only marshals arguments.  PyTorch is
used for device memory and streams.  The functions keep the C names:

    band_to_bidiag(band, b, d_out, e_out, stream=None)
    band_to_bidiag_ex(band, b, d_out, e_out, tuning=None, workspace=None, stream=None)
    band_to_bidiag_host(band_np, b, tuning=None) -> (d, e)
    band_to_bidiag_workspace_size(n, b, dtype, tuning=None)
    BatchPlan(problems, dtype, tuning)       # bb_batch_plan_*
    band_to_bidiag_batched(problems, stream=None)
    bb_device_status(stream=None, reset=True), bb_last_device_status(stream=None)
    bb_schedule_counts(n, b, tw), bb_default_tuning(n, b, dtype)
    bb_measure_l2_bandwidth(bytes, reps), bb_measure_fma_peak(dtype)

Band tensors use LAPACK 'U' band storage seen as a row-major (n, ldab)
array: row j holds column j of the band, A[i, j] = band[j, b + i - j].
There is no CPU fallback: without the compiled library every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbandbidiag.so")

BB_OK = 0
BB_ERR_ARG = 1
BB_ERR_ALLOC = 2
BB_ERR_LAUNCH = 3
BB_ERR_TIMEOUT = 4
BB_ERR_NONFINITE = 5
BB_ERR_WORKSPACE = 6
BB_ERR_UNSUPPORTED = 7
BB_F32 = 0
BB_F64 = 1
BB_F16 = 2
BB_BF16 = 3
BB_FLAG_INJECT_STALL = 0x100

_lib = None


class BBError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {status_string(code)} ({code})" if what else status_string(code))


class Tuning(ctypes.Structure):
    _fields_ = [("tw", ctypes.c_int), ("tpb", ctypes.c_int), ("sweeps_in_flight", ctypes.c_int),
                ("flags", ctypes.c_int), ("timeout_s", ctypes.c_double),
                ("ev_start", ctypes.c_void_p), ("ev_stop", ctypes.c_void_p), ("group", ctypes.c_int),
                ("teams", ctypes.c_int), ("ev_launch", ctypes.c_void_p), ("ev_count", ctypes.c_int),
                ("launch_log", ctypes.c_void_p)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("b", ctypes.c_int64), ("band", ctypes.c_void_p),
                ("ldab", ctypes.c_int64), ("d_out", ctypes.c_void_p), ("e_out", ctypes.c_void_p)]


def lib():
    """Load the compiled library; raise if it is missing (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2510_12705_gb300.build` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        i64, vp, ci, sz = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        tp = ctypes.POINTER(Tuning)
        sig = {
            "band_to_bidiag": (ci, [i64, i64, ci, vp, i64, vp, vp, vp]),
            "band_to_bidiag_ex": (ci, [i64, i64, ci, vp, i64, vp, vp, tp, vp, sz, vp]),
            "band_to_bidiag_workspace_size": (sz, [i64, i64, ci, tp]),
            "bb_shared_bytes": (sz, [i64, i64, ci, tp]),
            "band_to_bidiag_host": (ci, [i64, i64, ci, vp, i64, vp, vp, tp, vp]),
            "bb_batch_plan_create": (vp, [ci, ctypes.POINTER(Problem), ci, tp]),
            "bb_batch_plan_workspace_size": (sz, [vp]),
            "bb_batch_execute": (ci, [vp, vp, sz, vp]),
            "bb_batch_plan_destroy": (None, [vp]),
            "bb_device_status": (ci, [vp, ci]),
            "bb_last_device_status": (ci, [vp]),
            "band_to_bidiag_batched": (ci, [ci, ctypes.POINTER(Problem), ci, vp]),
            "bb_status_string": (ctypes.c_char_p, [ci]),
            "bb_schedule_counts": (ci, [i64, i64, ci, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                        ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double)]),
            "bb_default_tuning": (ci, [i64, i64, ci, tp]),
            "bb_stage_counts": (ci, [i64, i64, ci, ci, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
            "bb_reflector_index": (ci, [i64, i64, ci, ci, i64, i64, ctypes.POINTER(i64)]),
            "bb_measure_l2_bandwidth": (ctypes.c_double, [sz, ci, vp]),
            "bb_measure_fma_peak": (ctypes.c_double, [ci, vp]),
            "bb_autotune": (ci, [i64, i64, ci, vp, i64, vp, vp, tp, ci, ci,
                                 ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ci), vp]),
            "bb_bidiag_sigma_workspace_size": (sz, [i64]),
            "dense_to_band_workspace_size": (sz, [i64, i64, ci]),
            "band_to_bidiag_vectors_workspace_size": (sz, [i64, i64, ci, tp]),
            "band_to_bidiag_vectors": (ci, [i64, i64, ci, vp, i64, vp, vp, vp, i64, vp, i64, tp, vp, sz, vp]),
            "dense_to_band": (ci, [i64, i64, ci, vp, i64, vp, i64, vp, sz, vp]),
            "dense_to_band_qp": (ci, [i64, i64, ci, vp, i64, vp, i64, vp, i64, vp, i64, vp, sz, vp]),
            "bb_bidiag_sigma": (ci, [i64, ci, vp, vp, vp, vp, sz, vp]),
            "bb_mlp_param_count": (sz, [ci, ci]),
            "bb_mlp_backward_scratch": (sz, [ci, ci]),
            "bb_mlp_forward": (ci, [ci, ci, vp, vp, ci, vp, vp, vp, vp]),
            "bb_mlp_backward": (ci, [ci, ci, vp, vp, vp, vp, vp, vp, ci, vp, vp, vp]),
            "bb_mlp_adam": (ci, [ci, vp, vp, vp, vp, ci, ctypes.c_float, ctypes.c_float,
                                 ctypes.c_float, ctypes.c_float, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def status_string(code: int) -> str:
    return lib().bb_status_string(int(code)).decode()


def _check(code: int, what: str):
    if code != BB_OK:
        raise BBError(code, what)


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dtype_code(t) -> int:
    import torch
    if t == torch.float64:
        return BB_F64
    if t == torch.float32:
        return BB_F32
    if t == torch.float16:
        return BB_F16
    if t == torch.bfloat16:
        return BB_BF16
    raise TypeError(f"unsupported dtype {t}")


def _tuning_ptr(tuning):
    if tuning is None:
        return None
    if isinstance(tuning, dict):
        t = Tuning()
        for k, v in tuning.items():
            setattr(t, k, v)
        tuning = t
    return ctypes.byref(tuning)


def _device_buffer(x, name, like=None, min_bytes=0):
    """(pointer, bytes) of a tensor the kernels read or write: it must be a
    contiguous CUDA tensor on `like`'s device with at least `min_bytes`
    bytes.  A host tensor's pointer would reach a kernel as a device address,
    so it is refused here, before any library call."""
    if x is None or not x.is_cuda or not x.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor")
    if like is not None and x.device != like.device:
        raise ValueError(f"{name} must be on {like.device}, not {x.device}")
    nbytes = x.numel() * x.element_size()
    if nbytes < min_bytes:
        raise ValueError(f"{name} holds {nbytes} bytes; {min_bytes} needed")
    return x.data_ptr(), nbytes


def _workspace_args(workspace, like):
    """(pointer, bytes) of an optional caller workspace; (None, 0) lets the
    library allocate its own (the library checks the size)."""
    if workspace is None:
        return None, 0
    return _device_buffer(workspace, "workspace", like)


def _check_band(band, d_out, e_out):
    if band.dim() != 2:
        raise ValueError("band must be a 2-D tensor (n, ldab)")
    n, ldab = band.shape
    if not (band.is_cuda and d_out.is_cuda and (n == 1 or e_out.is_cuda)):
        raise ValueError("band, d_out and e_out must be CUDA tensors")
    if not band.is_contiguous():
        raise ValueError("band must be contiguous (n, ldab)")
    if not d_out.is_contiguous() or (n > 1 and not e_out.is_contiguous()):
        raise ValueError("d_out and e_out must be contiguous")
    if d_out.device != band.device or (n > 1 and e_out.device != band.device):
        raise ValueError("band, d_out and e_out must be on one device")
    if d_out.dtype != band.dtype or (n > 1 and e_out.dtype != band.dtype):
        raise ValueError("d_out / e_out must have the band's dtype")
    if d_out.numel() < n or (n > 1 and e_out.numel() < n - 1):
        raise ValueError("d_out needs n and e_out n-1 elements")
    return n, ldab


def band_to_bidiag(band, b: int, d_out, e_out, stream=None) -> None:
    """Reduce ``band`` (CUDA tensor (n, ldab), float32/float64) into d_out, e_out."""
    n, ldab = _check_band(band, d_out, e_out)
    rc = lib().band_to_bidiag(n, b, _dtype_code(band.dtype), band.data_ptr(), ldab,
                              d_out.data_ptr(), e_out.data_ptr() if n > 1 else None,
                              _stream_handle(stream))
    _check(rc, "band_to_bidiag")


def band_to_bidiag_ex(band, b: int, d_out, e_out, tuning=None, workspace=None, stream=None):
    n, ldab = _check_band(band, d_out, e_out)
    ws_ptr, ws_bytes = _workspace_args(workspace, band)
    rc = lib().band_to_bidiag_ex(n, b, _dtype_code(band.dtype), band.data_ptr(), ldab,
                                 d_out.data_ptr(), e_out.data_ptr() if n > 1 else None,
                                 _tuning_ptr(tuning), ws_ptr, ws_bytes, _stream_handle(stream))
    _check(rc, "band_to_bidiag_ex")


def band_to_bidiag_workspace_size(n: int, b: int, dtype: int, tuning=None) -> int:
    return int(lib().band_to_bidiag_workspace_size(n, b, dtype, _tuning_ptr(tuning)))


def bb_shared_bytes(n: int, b: int, dtype: int, tuning=None) -> int:
    """Dynamic shared memory per CTA of the bulge kernel (0 = invalid)."""
    return int(lib().bb_shared_bytes(n, b, dtype, _tuning_ptr(tuning)))


def band_to_bidiag_host(band, b: int, tuning=None, stream=None, out=None):
    """End-to-end call on host numpy arrays (pinned if possible): returns (d, e)."""
    import numpy as np
    band = np.ascontiguousarray(band)
    n, ldab = band.shape
    code = {np.dtype(np.float64): BB_F64, np.dtype(np.float32): BB_F32,
            np.dtype(np.float16): BB_F16}.get(band.dtype)
    if code is None:
        raise TypeError(f"unsupported dtype {band.dtype} (float64, float32, float16)")
    if out is None:
        d = np.empty(n, dtype=band.dtype)
        e = np.empty(max(n - 1, 1), dtype=band.dtype)
    else:
        d, e = out
    rc = lib().band_to_bidiag_host(n, b, code, band.ctypes.data, ldab, d.ctypes.data,
                                   e.ctypes.data, _tuning_ptr(tuning), _stream_handle(stream))
    _check(rc, "band_to_bidiag_host")
    return d, e[: n - 1]


def band_to_bidiag_host_ptr(n: int, b: int, dtype: int, band_ptr: int, ldab: int, d_ptr: int,
                            e_ptr: int, tuning=None, stream=None) -> int:
    """Raw-pointer form of band_to_bidiag_host (e.g. pinned torch CPU tensors)."""
    return lib().band_to_bidiag_host(n, b, dtype, band_ptr, ldab, d_ptr, e_ptr,
                                     _tuning_ptr(tuning), _stream_handle(stream))


def bb_device_status(stream=None, reset: bool = True) -> int:
    return int(lib().bb_device_status(_stream_handle(stream), 1 if reset else 0))


def status_bits(word: int) -> list[int]:
    return [c for c in range(1, 16) if word & (1 << c)]


def bb_default_tuning(n: int, b: int, dtype: int) -> Tuning:
    t = Tuning()
    _check(lib().bb_default_tuning(n, b, dtype, ctypes.byref(t)), "bb_default_tuning")
    return t


@dataclass
class ScheduleCounts:
    stages: int
    steps: int
    flops: float
    elements: float

    def bytes(self, elem_size: int) -> float:
        """Algorithmic bytes: every touched element read once and written once."""
        return 2.0 * self.elements * elem_size


def bb_stage_counts(n: int, b: int, tw: int, stage: int) -> ScheduleCounts:
    """Work model of one stage (``stages`` is the total number of stages)."""
    st, sp = ctypes.c_int64(), ctypes.c_int64()
    fl, el = ctypes.c_double(), ctypes.c_double()
    _check(lib().bb_stage_counts(n, b, tw, stage, ctypes.byref(st), ctypes.byref(sp),
                                 ctypes.byref(fl), ctypes.byref(el)), "bb_stage_counts")
    return ScheduleCounts(st.value, sp.value, fl.value, el.value)


def bb_schedule_counts(n: int, b: int, tw: int) -> ScheduleCounts:
    st, sp = ctypes.c_int64(), ctypes.c_int64()
    fl, el = ctypes.c_double(), ctypes.c_double()
    _check(lib().bb_schedule_counts(n, b, tw, ctypes.byref(st), ctypes.byref(sp),
                                    ctypes.byref(fl), ctypes.byref(el)), "bb_schedule_counts")
    return ScheduleCounts(st.value, sp.value, fl.value, el.value)


def bb_reflector_index(n: int, b: int, tw: int, stage: int, R: int, s: int) -> int:
    """Row-bulge ordinal k of step s of sweep R in stage `stage`: its right and
    left reflectors sit in slots 2k and 2k + 1 of the reflector store (host
    only; raises BBError with BB_ERR_ARG for a row-bulge that does not exist)."""
    k = ctypes.c_int64()
    _check(lib().bb_reflector_index(n, b, tw, stage, R, s, ctypes.byref(k)), "bb_reflector_index")
    return k.value


def bb_measure_l2_bandwidth(nbytes: int = 32 << 20, reps: int = 200, stream=None) -> float:
    return float(lib().bb_measure_l2_bandwidth(nbytes, reps, _stream_handle(stream)))


def bb_measure_fma_peak(dtype: int, stream=None) -> float:
    return float(lib().bb_measure_fma_peak(dtype, _stream_handle(stream)))


def dense_to_band(a, b: int, band_out, workspace=None, stream=None) -> None:
    """Stage 1 (dense_to_band): the dense CUDA matrix ``a`` (n x n, float32 or
    float64; read, never written) to upper band form with bandwidth b, written
    to ``band_out`` in the layout band_to_bidiag takes (a CUDA tensor (n, ldab),
    ldab >= b + 1, row j holding column j of the band).  ``a`` is seen
    column-major: a row-major tensor passes its transpose, which has the same
    singular values (use ``a.t().contiguous()`` for A itself)."""
    n = a.shape[0]
    if a.dim() != 2 or a.shape[1] != n or not a.is_cuda or not a.is_contiguous():
        raise ValueError("a must be a contiguous square CUDA tensor")
    if not band_out.is_cuda or band_out.dim() != 2 or band_out.shape[0] != n or band_out.dtype != a.dtype \
            or not band_out.is_contiguous() or band_out.device != a.device:
        raise ValueError("band_out must be a contiguous CUDA tensor (n, ldab) of a's dtype on a's device")
    code = _dtype_code(a.dtype)
    ws_ptr, ws_bytes = _workspace_args(workspace, a)
    rc = lib().dense_to_band(n, b, code, a.data_ptr(), n, band_out.data_ptr(), band_out.shape[1],
                             ws_ptr, ws_bytes, _stream_handle(stream))
    _check(rc, "dense_to_band")


def band_to_bidiag_vectors(band, b: int, d_out, e_out, q_out, p_out, tuning=None, workspace=None,
                           stream=None) -> None:
    """band_to_bidiag plus the orthogonal factors: Q (q_out) and P (p_out), CUDA
    tensors (n, n) of the band's dtype holding the column-major factors, so
    that Q^T A P = bidiag(d, e); as row-major tensors they read as Q^T and P^T."""
    n, ldab = _check_band(band, d_out, e_out)
    for x in (q_out, p_out):
        if not x.is_cuda or x.dtype != band.dtype or x.shape != (n, n) or not x.is_contiguous() \
                or x.device != band.device:
            raise ValueError("q_out and p_out must be contiguous (n, n) CUDA tensors of the band's dtype")
    ws_ptr, ws_bytes = _workspace_args(workspace, band)
    rc = lib().band_to_bidiag_vectors(n, b, _dtype_code(band.dtype), band.data_ptr(), ldab, d_out.data_ptr(),
                                      e_out.data_ptr() if n > 1 else None, q_out.data_ptr(), n,
                                      p_out.data_ptr(), n, _tuning_ptr(tuning), ws_ptr, ws_bytes,
                                      _stream_handle(stream))
    _check(rc, "band_to_bidiag_vectors")


def dense_to_band_qp(a, b: int, band_out, q_out, p_out, workspace=None, stream=None) -> None:
    """dense_to_band plus its orthogonal factors: Q (q_out) and P (p_out), CUDA
    tensors (n, n) of a's dtype holding the column-major factors (as row-major
    tensors they read as Q^T and P^T), with Q^T A P = B for the column-major A."""
    n = a.shape[0]
    if a.dim() != 2 or a.shape[1] != n or not a.is_cuda or not a.is_contiguous():
        raise ValueError("a must be a contiguous square CUDA tensor")
    for x in (q_out, p_out):
        if not x.is_cuda or x.dtype != a.dtype or x.shape != (n, n) or not x.is_contiguous() \
                or x.device != a.device:
            raise ValueError("q_out and p_out must be contiguous (n, n) CUDA tensors of a's dtype")
    if not band_out.is_cuda or band_out.dim() != 2 or band_out.shape[0] != n or band_out.dtype != a.dtype \
            or not band_out.is_contiguous() or band_out.device != a.device:
        raise ValueError("band_out must be a contiguous CUDA tensor (n, ldab) of a's dtype on a's device")
    ws_ptr, ws_bytes = _workspace_args(workspace, a)
    rc = lib().dense_to_band_qp(n, b, _dtype_code(a.dtype), a.data_ptr(), n, band_out.data_ptr(), band_out.shape[1],
                                q_out.data_ptr(), n, p_out.data_ptr(), n, ws_ptr, ws_bytes, _stream_handle(stream))
    _check(rc, "dense_to_band_qp")


def dense_to_band_workspace_size(n: int, b: int, dtype: int) -> int:
    return int(lib().dense_to_band_workspace_size(n, b, dtype))


class BatchPlan:
    """bb_batch_plan: many band problems reduced together, one persistent launch
    per stage for all of them.

    ``problems``: list of (band, b, d_out, e_out) CUDA tensors of one dtype.
    ``execute(workspace, stream)`` only enqueues stream work, so it can be
    captured into a CUDA graph (``torch.cuda.CUDAGraph``) and replayed.
    """

    def __init__(self, problems, tuning=None):
        self._keep = problems
        dt = problems[0][0].dtype
        self.dtype = _dtype_code(dt)
        arr = (Problem * len(problems))()
        for i, (band, b, d, e) in enumerate(problems):
            n, ldab = _check_band(band, d, e)
            if band.dtype != dt:
                raise ValueError("all problems of a batch share one dtype")
            arr[i] = Problem(n, b, band.data_ptr(), ldab, d.data_ptr(),
                             e.data_ptr() if n > 1 else None)
        self._arr = arr
        self._plan = lib().bb_batch_plan_create(len(problems), arr, self.dtype, _tuning_ptr(tuning))
        if not self._plan:
            raise BBError(BB_ERR_ARG, "bb_batch_plan_create")
        self.workspace_bytes = int(lib().bb_batch_plan_workspace_size(self._plan))

    def execute(self, workspace, stream=None):
        ws_ptr, ws_bytes = _device_buffer(workspace, "workspace", self._keep[0][0])
        rc = lib().bb_batch_execute(self._plan, ws_ptr, ws_bytes, _stream_handle(stream))
        _check(rc, "bb_batch_execute")

    def __del__(self):
        p = getattr(self, "_plan", None)
        if p and _lib is not None:
            _lib.bb_batch_plan_destroy(p)
            self._plan = None


def band_to_bidiag_batched(problems, stream=None) -> None:
    """One call for a batch: ``problems`` is a list of (band, b, d_out, e_out)
    CUDA tensors of one dtype; the workspace comes from the stream-ordered
    allocator (see BatchPlan for a reusable, graph-capturable plan)."""
    dt = problems[0][0].dtype
    arr = (Problem * len(problems))()
    for i, (band, b, d, e) in enumerate(problems):
        n, ldab = _check_band(band, d, e)
        if band.dtype != dt:
            raise ValueError("all problems of a batch share one dtype")
        arr[i] = Problem(n, b, band.data_ptr(), ldab, d.data_ptr(), e.data_ptr() if n > 1 else None)
    _check(lib().band_to_bidiag_batched(len(problems), arr, _dtype_code(dt), _stream_handle(stream)),
           "band_to_bidiag_batched")


def bb_last_device_status(stream=None) -> int:
    """bb_device_status(stream, reset=True)."""
    return int(lib().bb_last_device_status(_stream_handle(stream)))


def band_to_bidiag_noalloc(band, b: int, d_out, e_out, stream=None) -> None:
    """Allocation-free reduction: like band_to_bidiag, but the library's fixed
    16 MiB device scratch array is used instead of any allocation.  For callers
    that cannot allocate device memory at call time (stream capture without
    allocation nodes, an external allocator owning all memory).  Calls that may
    overlap on the GPU share that array and race; keep them on one stream.
    Raises BBError(BB_ERR_WORKSPACE) when the problem does not fit."""
    L = lib()
    f = L.band_to_bidiag_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    n, ldab = _check_band(band, d_out, e_out)
    rc = f(n, b, _dtype_code(band.dtype), band.data_ptr(), ldab, d_out.data_ptr(),
           e_out.data_ptr() if n > 1 else None, _stream_handle(stream))
    _check(rc, "band_to_bidiag_noalloc")


def bb_autotune(band, b: int, d_out, e_out, candidates, reps: int = 1, stream=None):
    """Exhaustive search: time every Tuning in ``candidates`` on this problem
    (median of ``reps`` runs after one untimed run); returns (times_ms, best)."""
    n, ldab = _check_band(band, d_out, e_out)
    arr = (Tuning * len(candidates))(*candidates)
    times = (ctypes.c_float * len(candidates))()
    best = ctypes.c_int(-1)
    rc = lib().bb_autotune(n, b, _dtype_code(band.dtype), band.data_ptr(), ldab, d_out.data_ptr(),
                           e_out.data_ptr() if n > 1 else None, arr, len(candidates), reps, times,
                           ctypes.byref(best), _stream_handle(stream))
    _check(rc, "bb_autotune")
    return [float(t) for t in times], int(best.value)


def bb_mlp_param_count(in_dim: int, hidden: int) -> int:
    return int(lib().bb_mlp_param_count(in_dim, hidden))


def bb_mlp_backward_scratch(hidden: int, N: int) -> int:
    return int(lib().bb_mlp_backward_scratch(hidden, N))


def _mlp_buffers(in_dim: int, hidden: int, X, named):
    """Pointers of the MLP kernels' FP32 buffers after checking that each is a
    contiguous CUDA tensor on X's device holding what the kernels touch:
    ``named`` maps a name to (tensor, floats needed)."""
    import torch
    if X.dim() != 2 or X.shape[1] != in_dim:
        raise ValueError(f"X must be (N, {in_dim})")
    ptrs = {}
    for name, (t, floats) in named.items():
        if t.dtype != torch.float32:
            raise ValueError(f"{name} must be float32")
        ptrs[name] = _device_buffer(t, name, X, 4 * floats)[0]
    return ptrs


def bb_mlp_forward(in_dim: int, hidden: int, params, X, Y, H1, H2, stream=None) -> None:
    """Y[N], H1[N][hidden], H2[N][hidden] from X[N][in_dim] (FP32 CUDA tensors)."""
    N, P = X.shape[0], bb_mlp_param_count(in_dim, hidden)
    p = _mlp_buffers(in_dim, hidden, X, {"params": (params, P), "X": (X, N * in_dim), "Y": (Y, N),
                                         "H1": (H1, N * hidden), "H2": (H2, N * hidden)})
    rc = lib().bb_mlp_forward(in_dim, hidden, p["params"], p["X"], N, p["Y"], p["H1"], p["H2"],
                              _stream_handle(stream))
    _check(rc, "bb_mlp_forward")


def bb_mlp_backward(in_dim: int, hidden: int, params, X, H1, H2, Y, T, grads, scratch,
                    stream=None) -> None:
    """Gradient of mean((Y - T)^2) with respect to the flat parameters."""
    N, P = X.shape[0], bb_mlp_param_count(in_dim, hidden)
    p = _mlp_buffers(in_dim, hidden, X, {
        "params": (params, P), "X": (X, N * in_dim), "H1": (H1, N * hidden), "H2": (H2, N * hidden),
        "Y": (Y, N), "T": (T, N), "grads": (grads, P),
        "scratch": (scratch, bb_mlp_backward_scratch(hidden, N))})
    rc = lib().bb_mlp_backward(in_dim, hidden, p["params"], p["X"], p["H1"], p["H2"], p["Y"], p["T"], N,
                               p["grads"], p["scratch"], _stream_handle(stream))
    _check(rc, "bb_mlp_backward")


def bb_mlp_adam(params, grads, m, v, step: int, lr: float, beta1: float = 0.9,
                beta2: float = 0.999, eps: float = 1e-8, stream=None) -> None:
    import torch
    count = params.numel()
    ptrs = []
    for name, t in (("params", params), ("grads", grads), ("m", m), ("v", v)):
        if t.dtype != torch.float32:
            raise ValueError(f"{name} must be float32")
        ptrs.append(_device_buffer(t, name, params, 4 * count)[0])
    rc = lib().bb_mlp_adam(count, *ptrs, step, lr, beta1, beta2, eps, _stream_handle(stream))
    _check(rc, "bb_mlp_adam")


def bb_bidiag_sigma(d, e, sigma_out=None, workspace=None, stream=None):
    """Singular values (FP64, descending, on the GPU) of the upper bidiagonal
    with diagonal d (n) and superdiagonal e (n-1), CUDA tensors of one dtype."""
    import torch
    n = d.numel()
    if e.dtype != d.dtype or (n > 1 and e.numel() < n - 1):
        raise ValueError("d and e: one dtype, len(e) >= len(d) - 1")
    d_ptr, _ = _device_buffer(d, "d")
    e_ptr = _device_buffer(e, "e", d)[0] if n > 1 else None
    if sigma_out is None:
        sigma_out = torch.empty(n, dtype=torch.float64, device=d.device)
    if sigma_out.dtype != torch.float64:
        raise ValueError("sigma_out must be float64")
    s_ptr, _ = _device_buffer(sigma_out, "sigma_out", d, 8 * n)
    if workspace is None:
        workspace = torch.empty(int(lib().bb_bidiag_sigma_workspace_size(n)), dtype=torch.uint8,
                                device=d.device)
    ws_ptr, ws_bytes = _device_buffer(workspace, "workspace", d)
    rc = lib().bb_bidiag_sigma(n, _dtype_code(d.dtype), d_ptr, e_ptr, s_ptr, ws_ptr, ws_bytes,
                               _stream_handle(stream))
    _check(rc, "bb_bidiag_sigma")
    return sigma_out
