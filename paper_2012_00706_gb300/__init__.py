"""GB300 column interpolative decomposition: thin Python binding over libgb300id.

The column ID of Dunton & Fox (Sec. 1.1) approximates A (m x n) by k of its
own columns, A ~= A(:, J[:k]) P with P(:, J[:k]) = I and P(:, J[k:]) = T.  All
arithmetic runs in the hand-written sm_103a kernels of ``libgb300id.so``; this
module only marshals torch tensors (device memory, the current stream, a
workspace buffer) into the C ABI declared in ``include/gb300_id.h``.  There is
no CPU fallback: if the native library is missing or there is no GPU, every
call raises.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

import torch

__all__ = [
    "PRECISIONS", "IDResult", "load", "id_factor", "id_sketch", "id_scale_cast", "id_workspace_size",
    "status_string", "lib_path", "set_stage_events", "id_backward", "id_reconstruct", "IDFunction",
    "BatchPlan", "shard_batch", "probe_fma_peak", "check_widen", "low_cast", "reconstruct", "id_factor_adaptive",
    "id_factor_rows", "id_factor_two_sided",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_NAME = "libgb300id.so"
_lib = None
_lock = threading.Lock()

PRECISIONS = {
    "plain_f64": 0, "plain_f32": 1, "mixed_bf16": 2, "mixed_f16": 3, "mixed_bf16x2": 4, "mixed_bf16x3": 5,
    "low_bf16": 6, "low_f16": 7,
}
_DTYPE = {torch.float64: 0, torch.float32: 1}
ID_SCALE_BLOCK_ROWS = 64
ID_MAX_ELL = 256


class IDOpts(ctypes.Structure):
    _fields_ = [
        ("k", ctypes.c_int32), ("rel_tol", ctypes.c_double), ("k_max", ctypes.c_int32),
        ("sketch", ctypes.c_int32), ("ell", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("omega", ctypes.c_void_p), ("omega_ld", ctypes.c_int64), ("refine_steps", ctypes.c_int32),
        ("estimate_error", ctypes.c_int32), ("watchdog_ms", ctypes.c_int64),
    ]


class BatchOpts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32), ("oversample", ctypes.c_int32), ("refine_steps", ctypes.c_int32),
        ("rel_tol", ctypes.c_double), ("watchdog_ms", ctypes.c_int64), ("slab_chunks", ctypes.c_int32),
        ("cpqr_tpc", ctypes.c_int32), ("solve_warps", ctypes.c_int32), ("solve_cols", ctypes.c_int32),
        ("tune_cache", ctypes.c_char_p),
    ]


class IDError(RuntimeError):
    pass


def lib_path() -> str:
    return os.path.join(_HERE, _LIB_NAME)


def load():
    """Load (building first if needed) the native library; raise if that fails."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        from . import build as _build
        if not _build.up_to_date():
            _build.build()
        lib = ctypes.CDLL(path)
        p, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        lib.id_opts_default.argtypes = [ctypes.POINTER(IDOpts)]
        lib.id_status_string.argtypes = [ctypes.c_int]
        lib.id_status_string.restype = ctypes.c_char_p
        lib.id_version.restype = ctypes.c_char_p
        lib.id_workspace_size.argtypes = [ctypes.c_int, i64, i64, ctypes.POINTER(IDOpts), ctypes.POINTER(sz)]
        lib.id_factor.argtypes = [p, ctypes.c_int, i64, i64, i64, ctypes.POINTER(IDOpts), p, p, i64, p, p, p,
                                  p, sz, p]
        lib.id_sketch_workspace_size.argtypes = [ctypes.c_int, i64, i64, i32, i32, ctypes.POINTER(sz)]
        lib.id_sketch.argtypes = [p, ctypes.c_int, i64, i64, i64, p, i64, i32, i32, p, i64, p, p, sz, p]
        lib.id_scale_cast.argtypes = [p, ctypes.c_int, i64, i64, i64, i32, p, p, p, p]
        lib.id_set_stage_events.argtypes = [ctypes.POINTER(ctypes.c_void_p), i32]
        lib.id_backward_workspace_size.argtypes = [i64, i64, i64, i32, ctypes.POINTER(sz)]
        lib.id_backward.argtypes = [i64, p, i64, i64, i64, i64, p, i64, i32, p, i64, i64, p, i64, i64, p, i64, i64,
                                    p, i64, i64, p, sz, p]
        lib.id_reconstruct_workspace_size.argtypes = [i64, i64, i32, ctypes.POINTER(sz)]
        lib.id_reconstruct.argtypes = [i64, p, i64, i64, i64, i64, p, i64, i32, p, i64, i64, p, i64, i64, p, sz, p]
        for name in ("id_backward_workspace_size", "id_backward", "id_reconstruct_workspace_size", "id_reconstruct"):
            getattr(lib, name).restype = ctypes.c_int
        lib.id_batch_opts_default.restype = BatchOpts
        lib.id_batch_plan_create.argtypes = [i32, ctypes.c_int, p, p, p, p, ctypes.POINTER(BatchOpts),
                                             ctypes.POINTER(ctypes.c_void_p)]
        lib.id_batch_plan_destroy.argtypes = [p]
        lib.id_batch_plan_destroy.restype = None
        lib.id_batch_plan_query.argtypes = [p, ctypes.POINTER(sz), p, p, ctypes.POINTER(i32), ctypes.POINTER(i64)]
        lib.id_batch_plan_describe.argtypes = [p, ctypes.c_char_p, i64]
        lib.id_batch_plan_describe.restype = i64
        lib.id_batch_workspace_size.argtypes = [p, ctypes.POINTER(sz)]
        lib.id_batch_bind.argtypes = [p, ctypes.POINTER(ctypes.c_void_p), p, sz, p]
        lib.id_factor_batched.argtypes = [p, p, i64, p, p, p, p, p, sz, p]
        lib.id_batch_autotune.argtypes = [p, p, i64, p, p, p, p, p, sz, p, i32, ctypes.c_char_p,
                                          ctypes.POINTER(ctypes.c_double)]
        lib.id_batch_shard.argtypes = [i32, p, p, p, i32, i32, p, p]
        lib.id_probe_fma_peak.argtypes = [i32, ctypes.POINTER(ctypes.c_double), p]
        lib.id_probe_fma_peak.restype = ctypes.c_int
        lib.id_check_widen.argtypes = [ctypes.POINTER(ctypes.c_uint64), p]
        lib.id_check_widen.restype = ctypes.c_int
        lib.id_adaptive_workspace_size.argtypes = [ctypes.c_int, i64, i64, ctypes.POINTER(IDOpts), i32, i32,
                                                   ctypes.POINTER(sz)]
        lib.id_adaptive_workspace_size.restype = ctypes.c_int
        lib.id_factor_adaptive.argtypes = [p, ctypes.c_int, i64, i64, i64, ctypes.POINTER(IDOpts), i32, i32, p, p,
                                           i64, p, p, p, ctypes.POINTER(i32), p, sz, p]
        lib.id_factor_adaptive.restype = ctypes.c_int
        lib.id_rows_workspace_size.argtypes = [ctypes.c_int, i64, i64, ctypes.POINTER(IDOpts), ctypes.POINTER(sz)]
        lib.id_factor_rows.argtypes = [p, ctypes.c_int, i64, i64, i64, ctypes.POINTER(IDOpts), p, p, i64, p, p, p,
                                       p, sz, p]
        lib.id_two_sided_workspace_size.argtypes = [ctypes.c_int, i64, i64, ctypes.POINTER(IDOpts),
                                                    ctypes.POINTER(sz)]
        lib.id_factor_two_sided.argtypes = [p, ctypes.c_int, i64, i64, i64, ctypes.POINTER(IDOpts), p, p, i64, p, p,
                                            i64, p, p, p, sz, p]
        for name in ("id_rows_workspace_size", "id_factor_rows", "id_two_sided_workspace_size",
                     "id_factor_two_sided"):
            getattr(lib, name).restype = ctypes.c_int
        lib.id_low_cast.argtypes = [p, ctypes.c_int, i64, i64, i64, i32, p, i64, p, p]
        lib.id_low_cast.restype = ctypes.c_int
        lib.id_reconstruct_one.argtypes = [p, ctypes.c_int, i64, i64, i64, p, i32, p, i64, p, i64, p]
        lib.id_reconstruct_one.restype = ctypes.c_int
        for name in ("id_batch_plan_create", "id_batch_plan_query", "id_batch_workspace_size", "id_batch_bind",
                     "id_factor_batched", "id_batch_autotune", "id_batch_shard"):
            getattr(lib, name).restype = ctypes.c_int
        for name in ("id_workspace_size", "id_factor", "id_sketch_workspace_size", "id_sketch",
                     "id_scale_cast", "id_set_stage_events"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def status_string(code: int) -> str:
    return load().id_status_string(code).decode()


def _check(code: int, what: str):
    if code != 0:
        raise IDError(f"{what}: {status_string(code)}")


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _colmajor(a: torch.Tensor):
    """(tensor, ld) with column-major storage of the (m, n) matrix a."""
    if a.dim() != 2:
        raise ValueError("expected a 2-D matrix")
    m, n = a.shape
    if a.stride(0) == 1 and (n == 1 or a.stride(1) >= max(m, 1)):
        return a, max(a.stride(1), m) if n > 1 else m
    return a.t().contiguous().t(), m


def _require_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("the GB300 ID library works on CUDA tensors only")


@dataclasses.dataclass
class IDResult:
    J: torch.Tensor        # (n,) int32: skeleton J[:k] in pivot order, then the rest ascending
    T: torch.Tensor        # (k, n - k) float64 interpolation coefficients
    k: int                 # rank used
    info: int              # 0 ok, j > 0 rank reduced, -1 non-finite input, -2 watchdog
    err: float | None      # relative Frobenius residual when requested


def _opts(k, tol, k_max, precision, sketch, ell, omega, omega_ld, refine_steps, estimate_error, watchdog_ms):
    o = IDOpts()
    load().id_opts_default(ctypes.byref(o))
    o.k = int(k or 0)
    o.rel_tol = float(tol or 0.0)
    o.k_max = int(k_max or 0)
    o.sketch = 1 if sketch else 0
    o.ell = int(ell or 0)
    o.precision = PRECISIONS[precision]
    o.omega = omega.data_ptr() if omega is not None else None
    o.omega_ld = int(omega_ld or 0)
    o.refine_steps = int(refine_steps)
    o.estimate_error = 1 if estimate_error else 0
    o.watchdog_ms = int(watchdog_ms or 0)
    return o


def _omega_ld(omega):
    if omega is None:
        return 0
    if omega.dim() != 2 or omega.stride(1) != 1:
        raise ValueError("omega must be a row-major (ell, m) tensor")
    return omega.stride(0)


def id_workspace_size(m, n, dtype=torch.float64, **kw) -> int:
    o = _opts(kw.get("k"), kw.get("tol"), kw.get("k_max"), kw.get("precision", "plain_f64"),
              kw.get("sketch", False), kw.get("ell"), kw.get("omega"), _omega_ld(kw.get("omega")),
              kw.get("refine_steps", 1), kw.get("estimate_error", False), 0)
    nb = ctypes.c_size_t(0)
    _check(load().id_workspace_size(_DTYPE[dtype], m, n, ctypes.byref(o), ctypes.byref(nb)), "id_workspace_size")
    return nb.value


def id_factor(A: torch.Tensor, k: int | None = None, *, tol: float | None = None, k_max: int | None = None,
              precision: str = "plain_f64", omega: torch.Tensor | None = None, refine_steps: int = 1,
              estimate_error: bool = False, watchdog_ms: int = 0, stream=None, workspace=None,
              out=None, sync: bool = True) -> IDResult:
    """Column ID of the CUDA matrix A (m, n); sketched when ``omega`` (ell, m) is given.

    ``precision``: plain_f64 | plain_f32 | mixed_bf16 | mixed_f16 | mixed_bf16x2 | mixed_bf16x3 |
    low_bf16 | low_f16 (mixed precisions need ``omega`` in bfloat16/half; plain_f64 sketches with
    a float64 omega; low_* pivot the cast A_L of the whole matrix, no omega).
    With ``sync=False`` the result tensors are returned without waiting; k and info are then -1.
    """
    _require_cuda(A, omega)
    if A.dtype not in _DTYPE:
        raise ValueError("A must be float64 or float32")
    a, lda = _colmajor(A)
    m, n = a.shape
    sketch = omega is not None
    ell = omega.shape[0] if sketch else 0
    if tol is None and k is None:
        raise ValueError("give a rank k or a tolerance tol")
    kcap = int(k_max if tol is not None else k)
    o = _opts(k, tol, k_max, precision, sketch, ell, omega, _omega_ld(omega), refine_steps, estimate_error,
              watchdog_ms)
    lib = load()
    nb = ctypes.c_size_t(0)
    _check(lib.id_workspace_size(_DTYPE[A.dtype], m, n, ctypes.byref(o), ctypes.byref(nb)), "id_workspace_size")
    dev = a.device
    if workspace is None or workspace.numel() < nb.value:
        workspace = torch.empty(nb.value, dtype=torch.uint8, device=dev)
    if out is None:
        J = torch.empty(n, dtype=torch.int32, device=dev)
        T = torch.empty((max(n - 1, 1), kcap), dtype=torch.float64, device=dev).t()   # column-major, ld = kcap
        small = torch.zeros(2, dtype=torch.int32, device=dev)
        err = torch.zeros(1, dtype=torch.float64, device=dev)
    else:
        J, T, small, err = out
    code = lib.id_factor(a.data_ptr(), _DTYPE[A.dtype], m, n, lda, ctypes.byref(o), J.data_ptr(), T.data_ptr(),
                         kcap, small.data_ptr(), small.data_ptr() + 4, err.data_ptr() if estimate_error else None,
                         workspace.data_ptr(), workspace.numel(), _stream_ptr(stream))
    _check(code, "id_factor")
    if not sync:
        return IDResult(J, T, -1, -1, None)
    kk, info = (int(v) for v in small.cpu())
    return IDResult(J, T[:kk, : n - kk], kk, info, float(err.item()) if estimate_error else None)


def probe_fma_peak(which: str = "fp32", stream=None) -> float:
    """Measured FFMA ("fp32") or DFMA ("fp64") rate of the current GPU in TFLOP/s
    (a profiling aid: the peak the ALU-bound kernels' rooflines use).  Synchronises."""
    t = ctypes.c_double(0.0)
    _check(load().id_probe_fma_peak({"fp32": 0, "fp64": 1}[which], ctypes.byref(t), _stream_ptr(stream)),
           "id_probe_fma_peak")
    return t.value


def check_widen(stream=None) -> int:
    """Number of FP32 bit patterns (of all 2^32) whose integer widening to FP64, the one
    the FP32 pivoted-QR kernels store R with, differs from the hardware conversion
    (a self-check; 0 expected).  Synchronises."""
    n = ctypes.c_uint64(0)
    _check(load().id_check_widen(ctypes.byref(n), _stream_ptr(stream)), "id_check_widen")
    return int(n.value)


def id_factor_adaptive(A: torch.Tensor, tol: float, k_max: int, omega: torch.Tensor, *, block: int = 16,
                       oversample: int = 10, precision: str = "mixed_bf16x3", refine_steps: int = 1,
                       watchdog_ms: int = 0, stream=None, workspace=None):
    """Rank-adaptive randomized ID: the sketch grows by ``block`` rows of ``omega`` (ell_max x m)
    and the rank with it (k = ell - oversample, at most k_max) until the FP64 relative
    Frobenius residual on A is <= tol.  Returns (IDResult with err, ell used).  Synchronises."""
    _require_cuda(A, omega)
    a, lda = _colmajor(A)
    m, n = a.shape
    o = _opts(None, tol, k_max, precision, True, omega.shape[0], omega, _omega_ld(omega), refine_steps, True,
              watchdog_ms)
    lib = load()
    nb = ctypes.c_size_t(0)
    _check(lib.id_adaptive_workspace_size(_DTYPE[A.dtype], m, n, ctypes.byref(o), block, oversample,
                                          ctypes.byref(nb)), "id_adaptive_workspace_size")
    dev = a.device
    if workspace is None or workspace.numel() < nb.value:
        workspace = torch.empty(nb.value, dtype=torch.uint8, device=dev)
    J = torch.empty(n, dtype=torch.int32, device=dev)
    T = torch.empty((max(n - 1, 1), k_max), dtype=torch.float64, device=dev).t()
    small = torch.zeros(2, dtype=torch.int32, device=dev)
    err = torch.zeros(1, dtype=torch.float64, device=dev)
    ell = ctypes.c_int32(0)
    _check(lib.id_factor_adaptive(a.data_ptr(), _DTYPE[A.dtype], m, n, lda, ctypes.byref(o), block, oversample,
                                  J.data_ptr(), T.data_ptr(), k_max, small.data_ptr(), small.data_ptr() + 4,
                                  err.data_ptr(), ctypes.byref(ell), workspace.data_ptr(), workspace.numel(),
                                  _stream_ptr(stream)), "id_factor_adaptive")
    kk, info = (int(v) for v in small.cpu())
    return IDResult(J, T[:kk, : n - kk], kk, info, float(err.item())), ell.value


def id_factor_rows(A: torch.Tensor, k: int, *, precision: str = "plain_f64", omega: torch.Tensor | None = None,
                   refine_steps: int = 1, estimate_error: bool = False, stream=None) -> IDResult:
    """Row ID A ~= X A(I[:k], :) of the CUDA matrix A (m, n): the column ID of A^T (``omega``,
    if given, is (ell, n)).  Returns IDResult with J = I (m row indices) and T (k, m - k):
    row I[k + c] of A ~= sum_b T[b, c] row I[b].  Synchronises."""
    _require_cuda(A, omega)
    a, lda = _colmajor(A)
    m, n = a.shape
    sketch = omega is not None
    o = _opts(k, None, None, precision, sketch, omega.shape[0] if sketch else 0, omega, _omega_ld(omega),
              refine_steps, estimate_error, 0)
    lib = load()
    nb = ctypes.c_size_t(0)
    _check(lib.id_rows_workspace_size(_DTYPE[A.dtype], m, n, ctypes.byref(o), ctypes.byref(nb)),
           "id_rows_workspace_size")
    dev = a.device
    work = torch.empty(nb.value, dtype=torch.uint8, device=dev)
    I = torch.empty(m, dtype=torch.int32, device=dev)
    T = torch.empty((max(m - 1, 1), k), dtype=torch.float64, device=dev).t()
    small = torch.zeros(2, dtype=torch.int32, device=dev)
    err = torch.zeros(1, dtype=torch.float64, device=dev)
    _check(lib.id_factor_rows(a.data_ptr(), _DTYPE[A.dtype], m, n, lda, ctypes.byref(o), I.data_ptr(), T.data_ptr(),
                              k, small.data_ptr(), small.data_ptr() + 4, err.data_ptr() if estimate_error else None,
                              work.data_ptr(), work.numel(), _stream_ptr(stream)), "id_factor_rows")
    kk, info = (int(v) for v in small.cpu())
    return IDResult(I, T[:kk, : m - kk], kk, info, float(err.item()) if estimate_error else None)


def id_factor_two_sided(A: torch.Tensor, k: int, *, precision: str = "plain_f64", omega: torch.Tensor | None = None,
                        refine_steps: int = 1, stream=None):
    """Two-sided ID A ~= X A(I[:k], J[:k]) P at rank k: the column ID (J, Tc) of A, then the
    rank-k row ID (I, Tr) of A(:, J[:k]).  Returns (col IDResult, row IDResult).  Synchronises."""
    _require_cuda(A, omega)
    a, lda = _colmajor(A)
    m, n = a.shape
    sketch = omega is not None
    o = _opts(k, None, None, precision, sketch, omega.shape[0] if sketch else 0, omega, _omega_ld(omega),
              refine_steps, False, 0)
    lib = load()
    nb = ctypes.c_size_t(0)
    _check(lib.id_two_sided_workspace_size(_DTYPE[A.dtype], m, n, ctypes.byref(o), ctypes.byref(nb)),
           "id_two_sided_workspace_size")
    dev = a.device
    work = torch.empty(nb.value, dtype=torch.uint8, device=dev)
    J = torch.empty(n, dtype=torch.int32, device=dev)
    Tc = torch.empty((max(n - 1, 1), k), dtype=torch.float64, device=dev).t()
    I = torch.empty(m, dtype=torch.int32, device=dev)
    Tr = torch.empty((max(m - 1, 1), k), dtype=torch.float64, device=dev).t()
    ks = torch.zeros(2, dtype=torch.int32, device=dev)
    infos = torch.zeros(2, dtype=torch.int32, device=dev)
    _check(lib.id_factor_two_sided(a.data_ptr(), _DTYPE[A.dtype], m, n, lda, ctypes.byref(o), J.data_ptr(),
                                   Tc.data_ptr(), k, I.data_ptr(), Tr.data_ptr(), k, ks.data_ptr(), infos.data_ptr(),
                                   work.data_ptr(), work.numel(), _stream_ptr(stream)), "id_factor_two_sided")
    (kc, kr), (ic, ir) = ks.cpu().tolist(), infos.cpu().tolist()
    return (IDResult(J, Tc[:kc, : n - kc], kc, ic, None), IDResult(I, Tr[:kr, : m - kr], kr, ir, None))


def set_stage_events(events) -> None:
    """Record these torch.cuda.Event objects at id_factor's stage boundaries (None: stop)."""
    lib = load()
    if not events:
        lib.id_set_stage_events(None, 0)
        return
    for e in events:
        if not e.cuda_event:        # torch creates the CUDA event at its first record
            e.record()
    arr = (ctypes.c_void_p * len(events))(*[ctypes.c_void_p(e.cuda_event) for e in events])
    lib.id_set_stage_events(arr, len(events))


def id_sketch(A: torch.Tensor, omega: torch.Tensor, precision: str = "mixed_bf16", stream=None,
              return_info: bool = False):
    """Y = Omega A (ell, n): float32 for the mixed precisions, float64 for plain_f64.
    With return_info, (Y, info): info a one-element device int32 tensor, -1 when A holds
    a non-finite value or an entry of Y is not finite, else 0."""
    _require_cuda(A, omega)
    a, lda = _colmajor(A)
    m, n = a.shape
    ell = omega.shape[0]
    lib = load()
    nb = ctypes.c_size_t(0)
    _check(lib.id_sketch_workspace_size(_DTYPE[A.dtype], m, n, ell, PRECISIONS[precision], ctypes.byref(nb)),
           "id_sketch_workspace_size")
    work = torch.empty(nb.value, dtype=torch.uint8, device=a.device)
    ydt = torch.float64 if precision == "plain_f64" else torch.float32
    Y = torch.empty((n, ell), dtype=ydt, device=a.device).t()      # column-major (ell, n)
    info = torch.zeros(1, dtype=torch.int32, device=a.device)
    _check(lib.id_sketch(a.data_ptr(), _DTYPE[A.dtype], m, n, lda, omega.data_ptr(), _omega_ld(omega), ell,
                         PRECISIONS[precision], Y.data_ptr(), ell, info.data_ptr(), work.data_ptr(), work.numel(),
                         _stream_ptr(stream)), "id_sketch")
    return (Y, info) if return_info else Y


def id_scale_cast(A: torch.Tensor, precision: str = "mixed_bf16", stream=None):
    """The sketch's scaled cast on its own: (pieces (nsplit, m, n) uint16 bits, shifts (nblocks, n), info)."""
    _require_cuda(A)
    a, lda = _colmajor(A)
    m, n = a.shape
    nsplit = {"mixed_bf16": 1, "mixed_f16": 1, "mixed_bf16x2": 2, "mixed_bf16x3": 3}[precision]
    nb = (m + ID_SCALE_BLOCK_ROWS - 1) // ID_SCALE_BLOCK_ROWS
    pieces = torch.empty((nsplit, n, m), dtype=torch.int16, device=a.device)
    shifts = torch.empty((n, nb), dtype=torch.int32, device=a.device)
    info = torch.zeros(1, dtype=torch.int32, device=a.device)
    _check(load().id_scale_cast(a.data_ptr(), _DTYPE[A.dtype], m, n, lda, PRECISIONS[precision],
                                pieces.data_ptr(), shifts.data_ptr(), info.data_ptr(), _stream_ptr(stream)),
           "id_scale_cast")
    return pieces.transpose(1, 2), shifts.t(), info


def low_cast(A: torch.Tensor, precision: str = "low_f16", stream=None, return_info: bool = False):
    """A_L of Algorithm 2 as a float32 (m, n) tensor: 2^s fl_low(x 2^-s) per (64-row block,
    column), the matrix the low_* precisions pivot (low_bf16 / mixed_bf16*: bfloat16,
    low_f16 / mixed_f16: half)."""
    _require_cuda(A)
    a, lda = _colmajor(A)
    m, n = a.shape
    out = torch.empty((n, m), dtype=torch.float32, device=a.device).t()
    info = torch.zeros(1, dtype=torch.int32, device=a.device)
    _check(load().id_low_cast(a.data_ptr(), _DTYPE[A.dtype], m, n, lda, PRECISIONS[precision], out.data_ptr(), m,
                              info.data_ptr(), _stream_ptr(stream)), "id_low_cast")
    return (out, info) if return_info else out


def reconstruct(A: torch.Tensor, J: torch.Tensor, T: torch.Tensor, k: int, stream=None) -> torch.Tensor:
    """A_hat = A(:, J[:k]) P of one (m, n) float64 or float32 matrix (FP64 accumulation):
    with A = A_D the ID's approximation (the mixed ID for low/mixed precisions), with
    A = low_cast(A_D) the low ID of Algorithm 2."""
    _require_cuda(A, J, T)
    a, lda = _colmajor(A)
    m, n = a.shape
    j = J.reshape(n).to(torch.int32).contiguous()
    out = torch.empty((n, m), dtype=A.dtype, device=a.device).t()
    if k < n:
        t = T[:k, : n - k]
        if not (t.stride(0) == 1 and t.stride(1) >= k):
            t = t.t().contiguous().t()
        tptr, ldt = t.data_ptr(), max(t.stride(1), k)
    else:
        tptr, ldt = None, k
    _check(load().id_reconstruct_one(a.data_ptr(), _DTYPE[A.dtype], m, n, lda, j.data_ptr(), k, tptr, ldt,
                                     out.data_ptr(), m, _stream_ptr(stream)), "id_reconstruct_one")
    return out


# ------------------------------------------------------------------ fixed-pivot adjoint

def _batched_colmajor(x: torch.Tensor, rows: int):
    """(batch, rows, cols) view with column-major matrices: returns (tensor, ld, batch stride)."""
    if x.dim() == 2:
        x = x.unsqueeze(0)
    b, r, c = x.shape
    if not (x.stride(1) == 1 and (c == 1 or x.stride(2) >= r)):
        x = x.transpose(1, 2).contiguous().transpose(1, 2)
    return x, x.stride(2) if c > 1 else r, x.stride(0)


def id_reconstruct(A: torch.Tensor, J: torch.Tensor, T: torch.Tensor, k: int, stream=None) -> torch.Tensor:
    """A_hat = A(:, J[:k]) P for float32 A of shape (m, n) or (batch, m, n); T (.., k, n-k) float64."""
    _require_cuda(A, J, T)
    squeeze = A.dim() == 2
    a, lda, sa = _batched_colmajor(A, A.shape[-2])
    batch, m, n = a.shape
    j = J.reshape(batch, n).contiguous()
    t, ldt, st = _batched_colmajor(T.reshape(batch, k, n - k), k)
    out = torch.empty((batch, n, m), dtype=torch.float32, device=a.device).transpose(1, 2)
    lib = load()
    nb = ctypes.c_size_t(0)
    _check(lib.id_reconstruct_workspace_size(batch, n, k, ctypes.byref(nb)), "id_reconstruct_workspace_size")
    work = torch.empty(nb.value, dtype=torch.uint8, device=a.device)
    _check(lib.id_reconstruct(batch, a.data_ptr(), m, n, lda, sa, j.data_ptr(), n, k, t.data_ptr(), ldt, st,
                              out.data_ptr(), m, m * n, work.data_ptr(), work.numel(), _stream_ptr(stream)),
           "id_reconstruct")
    return out[0] if squeeze else out


def id_backward(A: torch.Tensor, J: torch.Tensor, T: torch.Tensor, k: int, dAhat: torch.Tensor | None = None,
                dT: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """dL/dA of the fixed-pivot ID for float32 A (m, n) or (batch, m, n), given dL/dA_hat and/or dL/dT."""
    _require_cuda(A, J, T, dAhat, dT)
    squeeze = A.dim() == 2
    a, lda, sa = _batched_colmajor(A, A.shape[-2])
    batch, m, n = a.shape
    j = J.reshape(batch, n).contiguous()
    t, ldt, st = _batched_colmajor(T.reshape(batch, k, n - k), k)
    g = ldg = sg = None
    if dAhat is not None:
        g, ldg, sg = _batched_colmajor(dAhat.reshape(batch, m, n).float(), m)
    tb = ldtb = stb = None
    if dT is not None:
        tb, ldtb, stb = _batched_colmajor(dT.reshape(batch, k, n - k).double(), k)
    out = torch.empty((batch, n, m), dtype=torch.float32, device=a.device).transpose(1, 2)
    lib = load()
    nb = ctypes.c_size_t(0)
    _check(lib.id_backward_workspace_size(batch, m, n, k, ctypes.byref(nb)), "id_backward_workspace_size")
    work = torch.empty(nb.value, dtype=torch.uint8, device=a.device)
    _check(lib.id_backward(batch, a.data_ptr(), m, n, lda, sa, j.data_ptr(), n, k, t.data_ptr(), ldt, st,
                           g.data_ptr() if g is not None else None, ldg or m, sg or 0,
                           tb.data_ptr() if tb is not None else None, ldtb or k, stb or 0,
                           out.data_ptr(), m, m * n, work.data_ptr(), work.numel(), _stream_ptr(stream)),
           "id_backward")
    return out[0] if squeeze else out


_PLAN_CACHE: "dict" = {}
_PLAN_CACHE_SIZE = 4


def _forward_plan(ac: torch.Tensor, k: int, lda: int) -> "BatchPlan":
    """The bound PLAIN_F32 batch plan of IDFunction's forward for these matrices, kept for
    the most recent few (shape, rank, strides, address): a repeated forward on the same
    buffers only launches (no host tables, no table upload).  The plan keeps the matrices'
    addresses only (they are part of the key), not the tensors, so the cache holds no
    caller memory alive; the caller copies J and T out before the plan can run again."""
    batch, m, n = ac.shape
    key = (batch, m, n, k, lda, tuple(ac.stride()), ac.data_ptr(), ac.dtype, str(ac.device))
    plan = _PLAN_CACHE.pop(key, None)
    if plan is None:
        plan = BatchPlan([(m, n)] * batch, [k] * batch, dtype=ac.dtype, precision="plain_f32",
                         lda=[lda] * batch, device=ac.device)
        plan.bind([ac[b] for b in range(batch)])
        plan.mats = None
    _PLAN_CACHE[key] = plan
    while len(_PLAN_CACHE) > _PLAN_CACHE_SIZE:
        _PLAN_CACHE.pop(next(iter(_PLAN_CACHE)))
    return plan


class IDFunction(torch.autograd.Function):
    """Differentiable column ID with the pivots held fixed.

    ``IDFunction.apply(A, k)`` for float32 A (m, n) or (batch, m, n) returns
    ``(A_hat, T, J)``: the reconstruction A(:, J[:k]) P, the coefficients T (float64,
    k x (n-k)) and the pivots (not differentiable).  The pivots and T come from the
    column-pivoted QR of A (``precision='plain_f32'``), whose T = R11^-1 R12 is the
    least-squares X^+ C that the adjoint differentiates.
    """

    @staticmethod
    def forward(ctx, A, k):
        squeeze = A.dim() == 2
        a = A.unsqueeze(0) if squeeze else A
        batch, m, n = a.shape
        dev = a.device
        if batch > 1:
            # the whole batch in one launch sequence: grouped pivoted QRs in waves, then
            # one batched solve; the ranks are read back once
            ac, lda, _ = _batched_colmajor(a, m)
            plan = _forward_plan(ac, k, lda)
            plan.run()
            kinfo = torch.stack([plan.k_out, plan.info], dim=1).cpu()
            Jt = plan.J[: batch * n].view(batch, n).clone()
            Tt = plan.T[: batch * k * (n - k)].view(batch, n - k, k).clone().transpose(1, 2)
        else:
            ws = torch.empty(id_workspace_size(m, n, a.dtype, k=k, precision="plain_f32"), dtype=torch.uint8,
                             device=dev)
            Jt = torch.empty((batch, n), dtype=torch.int32, device=dev)
            Tall = torch.empty((batch, max(n - k, 1), k), dtype=torch.float64, device=dev)
            small = torch.zeros((batch, 2), dtype=torch.int32, device=dev)
            err = torch.zeros(1, dtype=torch.float64, device=dev)
            id_factor(a[0], k, precision="plain_f32", workspace=ws, out=(Jt[0], Tall[0], small[0], err), sync=False)
            kinfo = small.cpu()
            Tt = Tall[:, : n - k, :].transpose(1, 2)          # (batch, k, n - k), column-major per matrix
        bad = (kinfo[:, 0] != k).nonzero()
        if bad.numel():
            b = int(bad[0, 0])
            raise IDError(f"matrix {b}: rank {int(kinfo[b, 0])} < k = {k} (info {int(kinfo[b, 1])})")
        Ahat = id_reconstruct(a, Jt, Tt, k)
        ctx.save_for_backward(a, Jt, Tt)
        ctx.k = k
        ctx.squeeze = squeeze
        ctx.mark_non_differentiable(Jt)
        if squeeze:
            return Ahat[0], Tt[0], Jt[0]
        return Ahat, Tt, Jt

    @staticmethod
    def backward(ctx, gAhat, gT, gJ):
        a, Jt, Tt = ctx.saved_tensors
        if ctx.squeeze:
            gAhat = None if gAhat is None else gAhat.unsqueeze(0)
            gT = None if gT is None else gT.unsqueeze(0)
        dA = id_backward(a, Jt, Tt, ctx.k, gAhat, gT)
        return (dA[0] if ctx.squeeze else dA), None


# ------------------------------------------------------------------ batched IDs

class BatchPlan:
    """Many IDs of fixed uneven shapes in one launch sequence: mixed precision
    (``precision="mixed_*"``), the FP64 twin (``"plain_f64"``: each matrix's
    sketched FP64 ID as ``id_factor`` computes it, FP64 Omega), or the unsketched
    FP32 pivoted QR of every matrix (``"plain_f32"``, no Omega).

    ``shapes``: list of (m, n); ``ranks``: list of k.  Matrices are column-major
    with leading dimensions ``lda`` (default m; lda * element size must be a
    multiple of 16 bytes).  The plan owns the workspace and the packed outputs.
    ``bind(mats)`` fixes the matrices (CUDA tensors, column-major views such as
    ``buf.t()[:m]``); ``run(omega)`` factors them with the shared Omega (at least
    ell_max x m_max, row-major; low precision bits, or float64 for plain_f64).
    """

    def __init__(self, shapes, ranks, *, dtype=torch.float64, precision="mixed_bf16", oversample=10,
                 refine_steps=1, tol=None, watchdog_ms=0, slab_chunks=0, cpqr_tpc=0, solve_warps=0,
                 solve_cols=0, tune_cache=None, lda=None, device=None):
        lib = load()
        self._lib = lib
        self.batch = len(shapes)
        self.m = [int(s[0]) for s in shapes]
        self.n = [int(s[1]) for s in shapes]
        self.k = [int(r) for r in ranks]
        self.lda = [int(v) for v in (lda if lda is not None else self.m)]
        self.dtype = dtype
        o = lib.id_batch_opts_default()
        o.precision = PRECISIONS[precision]
        o.oversample = oversample
        o.refine_steps = refine_steps
        o.rel_tol = float(tol) if tol else 0.0
        o.watchdog_ms = watchdog_ms
        o.slab_chunks, o.cpqr_tpc, o.solve_warps, o.solve_cols = slab_chunks, cpqr_tpc, solve_warps, solve_cols
        self._cache = tune_cache.encode() if tune_cache else None
        o.tune_cache = self._cache
        i64a = ctypes.c_int64 * self.batch
        m_, n_, l_ = i64a(*self.m), i64a(*self.n), i64a(*self.lda)
        k_ = (ctypes.c_int32 * self.batch)(*self.k)
        h = ctypes.c_void_p(0)
        _check(lib.id_batch_plan_create(self.batch, _DTYPE[dtype], m_, n_, l_, k_, ctypes.byref(o), ctypes.byref(h)),
               "id_batch_plan_create")
        self._h = h
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self._query()
        self.mats = None
        if self.device.type != "cuda":
            return          # planning only (sizes, offsets, describe); nothing to run
        self.k_out = torch.zeros(self.batch, dtype=torch.int32, device=self.device)
        self.info = torch.zeros(self.batch, dtype=torch.int32, device=self.device)
        self.J = torch.empty(max(self.j_off[-1], 1), dtype=torch.int32, device=self.device)
        self.T = torch.empty(max(self.t_off[-1], 1), dtype=torch.float64, device=self.device)
        self.work = torch.empty(max(self.work_bytes, 256), dtype=torch.uint8, device=self.device)

    def _query(self):
        nb = ctypes.c_size_t(0)
        jo = (ctypes.c_int64 * (self.batch + 1))()
        to = (ctypes.c_int64 * (self.batch + 1))()
        em = ctypes.c_int32(0)
        mm = ctypes.c_int64(0)
        _check(self._lib.id_batch_plan_query(self._h, ctypes.byref(nb), jo, to, ctypes.byref(em), ctypes.byref(mm)),
               "id_batch_plan_query")
        self.work_bytes = nb.value
        self.j_off = list(jo)
        self.t_off = list(to)
        self.ell_max = em.value
        self.m_max = mm.value

    def bind(self, mats, stream=None):
        """Fix the matrices (kept referenced by the plan) and write the tables to the workspace."""
        if len(mats) != self.batch:
            raise ValueError("one matrix per plan entry")
        for a, m, n in zip(mats, self.m, self.n):
            if not a.is_cuda or a.dtype != self.dtype or tuple(a.shape) != (m, n) or a.stride(0) != 1:
                raise ValueError("matrices must be column-major CUDA tensors of the planned shapes and dtype")
        self.mats = list(mats)
        arr = (ctypes.c_void_p * self.batch)(*[ctypes.c_void_p(a.data_ptr()) for a in mats])
        _check(self._lib.id_batch_bind(self._h, arr, self.work.data_ptr(), self.work.numel(), _stream_ptr(stream)),
               "id_batch_bind")

    def describe(self) -> dict:
        import json
        need = self._lib.id_batch_plan_describe(self._h, None, 0)
        buf = ctypes.create_string_buffer(int(need))
        self._lib.id_batch_plan_describe(self._h, buf, need)
        return json.loads(buf.value.decode())

    def run(self, omega: torch.Tensor | None = None, stream=None):
        """Enqueue the batch (no synchronisation); outputs land in self.J/T/k_out/info."""
        ld = _omega_ld(omega) if omega is not None else 0
        optr = omega.data_ptr() if omega is not None else None
        _check(self._lib.id_factor_batched(self._h, optr, ld, self.J.data_ptr(), self.T.data_ptr(),
                                           self.k_out.data_ptr(), self.info.data_ptr(), self.work.data_ptr(),
                                           self.work.numel(), _stream_ptr(stream)), "id_factor_batched")

    def autotune(self, omega: torch.Tensor, reps: int = 5, cache_path=None, stream=None):
        best = ctypes.c_double(0.0)
        cp = cache_path.encode() if cache_path else None
        _check(self._lib.id_batch_autotune(self._h, omega.data_ptr(), _omega_ld(omega), self.J.data_ptr(),
                                           self.T.data_ptr(), self.k_out.data_ptr(), self.info.data_ptr(),
                                           self.work.data_ptr(), self.work.numel(), _stream_ptr(stream), reps, cp,
                                           ctypes.byref(best)), "id_batch_autotune")
        return best.value

    def results(self):
        """Per-matrix IDResult list (synchronises)."""
        ks = self.k_out.cpu().tolist()
        infos = self.info.cpu().tolist()
        out = []
        for i in range(self.batch):
            n, kc = self.n[i], self.k[i]
            J = self.J[self.j_off[i]: self.j_off[i + 1]]
            cols = (self.t_off[i + 1] - self.t_off[i]) // kc
            T = self.T[self.t_off[i]: self.t_off[i] + kc * cols].view(cols, kc).t()
            kk = ks[i]
            out.append(IDResult(J, T[:kk, : max(n - kk, 0)], kk, infos[i], None))
        return out

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.id_batch_plan_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def shard_batch(shapes, ranks, world: int, oversample: int = 10):
    """(rank_of, work): the library's longest-processing-time split of a batch over
    ``world`` processes (host only, deterministic) and each rank's modelled flop."""
    lib = load()
    b = len(shapes)
    m_ = (ctypes.c_int64 * b)(*[int(s[0]) for s in shapes])
    n_ = (ctypes.c_int64 * b)(*[int(s[1]) for s in shapes])
    k_ = (ctypes.c_int32 * b)(*[int(r) for r in ranks])
    rank_of = (ctypes.c_int32 * b)()
    work = (ctypes.c_double * world)()
    _check(lib.id_batch_shard(b, m_, n_, k_, oversample, world, rank_of, work), "id_batch_shard")
    return list(rank_of), list(work)
