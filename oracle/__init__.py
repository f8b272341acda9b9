"""FP64 CPU oracle for the column interpolative decomposition.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the GPU library (``paper_2012_00706_gb300``) and the library never calls
it.

The arithmetic of the ID lives in ``id_oracle.c`` (plain C, FP64, compiled
with ``gcc -O2``, no fast-math); this module wraps it with numpy and adds the
pieces that are plain library calls: 2-norms through LAPACK's SVD, the
Lemma 1 bound of Sec. 2, brute-force subset search on tiny inputs, and the
reference gradient of the fixed-pivot adjoint.

Parity pins: every function here is checked in ``tests/test_oracle_*.py``
against something other than itself (exact-rank reconstruction, closed forms,
LAPACK's pivoted QR, brute force, the Table 2 values of the paper, finite
differences).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "id_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

FMT_BF16, FMT_F16 = 0, 1
_FMT = {"bf16": FMT_BF16, "f16": FMT_F16}


def build(force: bool = False) -> str:
    """Compile id_oracle.c into liboracle.so (plain gcc, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            d, i64, i32, p = ctypes.c_double, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
            lib.orc_sketch_f64.argtypes = [p, i64, i64, p, i64, i64, p, i64]
            lib.orc_round_fmt.argtypes = [d, ctypes.c_int]
            lib.orc_round_fmt.restype = d
            lib.orc_block_shift.argtypes = [d, ctypes.c_int, ctypes.c_int]
            lib.orc_block_shift.restype = ctypes.c_int
            lib.orc_quantize.argtypes = [p, i64, i64, i64, ctypes.c_int, ctypes.c_int, i64, ctypes.c_int, p, p]
            lib.orc_quantize.restype = ctypes.c_int
            lib.orc_sketch_lowp.argtypes = [p, i64, i64, p, i64, i64, ctypes.c_int, ctypes.c_int,
                                            i64, ctypes.c_int, p, i64]
            lib.orc_sketch_lowp.restype = ctypes.c_int
            lib.orc_cpqr.argtypes = [p, i64, i64, i64, i32, d, i32, i32, p, p, i64, p, p]
            lib.orc_cpqr.restype = ctypes.c_int
            lib.orc_mgs_cpqr.argtypes = [p, i64, i64, i64, i32, p, p, i64]
            lib.orc_mgs_cpqr.restype = ctypes.c_int
            lib.orc_solve_T.argtypes = [i32, i64, p, p, i64, p, i64]
            lib.orc_residual_fro2.argtypes = [p, i64, i64, i64, i32, p, p, i64]
            lib.orc_residual_fro2.restype = d
            lib.orc_id.argtypes = [p, i64, i64, i64, p, i64, i32, d, i32, i32, p, p, i64, p, p]
            lib.orc_id.restype = ctypes.c_int
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------------- sketch

def sketch_f64(omega: np.ndarray, a: np.ndarray) -> np.ndarray:
    """Y = Omega A in FP64 (plain dot products)."""
    om = np.ascontiguousarray(omega, dtype=np.float64)
    a = _f64(a)
    ell, m = om.shape
    n = a.shape[1]
    y = np.zeros((ell, n), dtype=np.float64, order="F")
    _L().orc_sketch_f64(_ptr(om), ell, m, _ptr(a), a.shape[0], n, _ptr(y), ell)
    return y


def round_fmt(x: float, fmt: str) -> float:
    """Round one value to bfloat16/half, ties to even."""
    return _L().orc_round_fmt(float(x), _FMT[fmt])


def block_shift(mx: float, fmt: str, in_f32: bool = False) -> int:
    """Power-of-two shift of a scaling block from its largest magnitude."""
    return _L().orc_block_shift(float(mx), _FMT[fmt], int(in_f32))


def quantize(a: np.ndarray, fmt: str, block_rows: int, nsplit: int = 1):
    """Scaled low-precision cast of Algorithm 2 with per-(row block, column) power-of-two shifts.

    Each scaled entry is taken at FP32 precision (round to nearest even) and split
    into ``nsplit`` low-format pieces.  ``a`` of dtype float32 is treated as float
    storage.  Returns ``(pieces, shifts, rc)``: pieces (nsplit, m, n) float64 values
    of the low-format pieces, shifts (nblocks, n) int32, rc = -1 on non-finite input.
    """
    in_f32 = int(np.asarray(a).dtype == np.float32)
    a = _f64(a)
    m, n = a.shape
    nb = (m + block_rows - 1) // block_rows
    q = np.zeros(nsplit * m * n, dtype=np.float64)
    s = np.zeros(nb * n, dtype=np.int32)
    rc = _L().orc_quantize(_ptr(a), m, n, m, _FMT[fmt], nsplit, block_rows, in_f32, _ptr(q), _ptr(s))
    pieces = q.reshape(nsplit, n, m).transpose(0, 2, 1)
    return pieces, s.reshape(n, nb).T.copy(), rc


def sketch_lowp(omega: np.ndarray, a: np.ndarray, fmt: str, nsplit: int, block_rows: int):
    """FP64 evaluation of the sketch of the scaled low-precision cast of A."""
    in_f32 = int(np.asarray(a).dtype == np.float32)
    om = np.ascontiguousarray(omega, dtype=np.float64)
    a = _f64(a)
    ell, m = om.shape
    n = a.shape[1]
    y = np.zeros((ell, n), dtype=np.float64, order="F")
    rc = _L().orc_sketch_lowp(_ptr(om), ell, m, _ptr(a), m, n, _FMT[fmt], nsplit, block_rows,
                              in_f32, _ptr(y), ell)
    if rc == -2:
        raise MemoryError("oracle sketch_lowp")
    return y, rc


# --------------------------------------------------------------------- CPQR

def cpqr(w: np.ndarray, k: int | None = None, tol: float | None = None,
         k_max: int | None = None, norm_mode: str = "exact"):
    """Truncated column-pivoted Householder QR (Sec. 1.1), FP64.

    Returns dict(J, R, k, gaps, info); R is (steps x n) with columns by original index.
    """
    w = _f64(w)
    r, n = w.shape
    if tol is None:
        cap = min(int(k), r, n)
        kreq, rt, km = int(k), 0.0, 0
    else:
        km = int(k_max if k_max is not None else min(r, n))
        cap = min(km, r, n)
        kreq, rt = 0, float(tol)
    cap1 = max(cap, 1)
    J = np.zeros(n, dtype=np.int32)
    R = np.zeros((cap1, n), dtype=np.float64, order="F")
    gaps = np.ones(cap1, dtype=np.float64)
    kout = ctypes.c_int32(0)
    mode = {"exact": 0, "downdate": 1}[norm_mode]
    info = _L().orc_cpqr(_ptr(w), r, n, r, kreq, rt, km, mode, _ptr(J), _ptr(R), cap1,
                         ctypes.byref(kout), _ptr(gaps))
    kk = kout.value
    return {"J": J, "R": R[:kk], "k": kk, "gaps": gaps[:kk], "info": info}


def mgs_cpqr(w: np.ndarray, k: int):
    """Greedy selection by reorthogonalised modified Gram-Schmidt (the paper's MGSQR)."""
    w = _f64(w)
    r, n = w.shape
    J = np.zeros(max(k, 1), dtype=np.int32)
    R = np.zeros((max(k, 1), n), dtype=np.float64, order="F")
    info = _L().orc_mgs_cpqr(_ptr(w), r, n, r, k, _ptr(J), _ptr(R), max(k, 1))
    return {"J": J[:k], "R": R[:k], "info": info}


def solve_T(R: np.ndarray, J: np.ndarray, k: int) -> np.ndarray:
    """T = R11^-1 R12 by back-substitution (Algorithm 1, the coefficient solve)."""
    R = _f64(R)
    n = R.shape[1]
    T = np.zeros((max(k, 1), max(n - k, 1)), dtype=np.float64, order="F")
    J = np.ascontiguousarray(J, dtype=np.int32)
    if k > 0 and n > k:
        _L().orc_solve_T(k, n, _ptr(J), _ptr(R), R.shape[0], _ptr(T), T.shape[0])
    return T[:k, :n - k]


def interp_decomp(a: np.ndarray, k: int | None = None, tol: float | None = None,
                  k_max: int | None = None, omega: np.ndarray | None = None,
                  norm_mode: str = "exact"):
    """Oracle ID: optional sketch W = Omega A, truncated CPQR of W, T = R11^-1 R12.

    Returns dict(J, T, k, info, gaps).
    """
    a = _f64(a)
    m, n = a.shape
    om = None if omega is None else np.ascontiguousarray(omega, dtype=np.float64)
    r = m if om is None else om.shape[0]
    if tol is None:
        cap, kreq, rt, km = min(int(k), r, n), int(k), 0.0, 0
    else:
        km = int(k_max if k_max is not None else min(r, n))
        cap, kreq, rt = min(km, r, n), 0, float(tol)
    cap1 = max(cap, 1)
    J = np.zeros(n, dtype=np.int32)
    T = np.zeros((cap1, max(n, 1)), dtype=np.float64, order="F")
    gaps = np.ones(cap1, dtype=np.float64)
    kout = ctypes.c_int32(0)
    mode = {"exact": 0, "downdate": 1}[norm_mode]
    info = _L().orc_id(_ptr(a), m, n, m, None if om is None else _ptr(om),
                       0 if om is None else om.shape[0], kreq, rt, km, mode,
                       _ptr(J), _ptr(T), cap1, ctypes.byref(kout), _ptr(gaps))
    kk = kout.value
    return {"J": J, "T": np.asfortranarray(T[:kk, :n - kk]), "k": kk, "info": info,
            "gaps": gaps[:kk]}


# ------------------------------------------------- rank-adaptive sketched ID

def adaptive_id(a: np.ndarray, omega: np.ndarray, tol: float, block: int, k_max: int,
                oversample: int = 10):
    """Rank-adaptive randomized ID (the sketching the paper names as future work in Sec. 5,
    grown by blocks): for ell = block, 2 block, ... (at most omega's rows), Y = Omega(0:ell) A,
    the truncated CPQR of Y with k = min(k_max, ell - oversample) steps (fewer if a
    residual norm reaches zero), T = R11^-1 R12, and the exact relative Frobenius residual
    e = ||A - A(:,J) P||_F / ||A||_F; stop at the first ell whose e <= tol, or at the last
    block.  The rank grows with the sketch, so it is the smallest multiple-of-block step
    that meets the tolerance.  Returns the ID of the final round with "ell" and "err"."""
    a = _f64(a)
    om = np.ascontiguousarray(omega, dtype=np.float64)
    ell_max = om.shape[0]
    na2 = float(np.sum(a * a))
    out = None
    ell = 0
    while ell < ell_max:
        ell = min(ell + block, ell_max)
        k = max(1, min(k_max, ell - oversample, a.shape[1]))
        out = interp_decomp(a, k=k, omega=om[:ell])
        err = np.sqrt(residual_fro2(a, out["J"], out["T"], out["k"]) / na2) if na2 > 0 else 0.0
        out["ell"], out["err"] = ell, float(err)
        if err <= tol:
            break
    return out


# ------------------------------------------------------- row and two-sided IDs

def row_id(a: np.ndarray, k: int, omega: np.ndarray | None = None):
    """Row ID A ~= X A(I[0:k], :): the column ID of A^T (Omega, if given, is ell x n).
    Returns interp_decomp's dict for A^T: J are the row indices I, T gives X(I[k:], :) = T^T."""
    return interp_decomp(np.asarray(a, dtype=np.float64).T, k=k, omega=omega)


def two_sided_id(a: np.ndarray, k: int, omega: np.ndarray | None = None):
    """Two-sided ID A ~= X A(I[0:k], J[0:k]) P: the column ID (J, T) of A, then the rank-k
    row ID (I, Tr) of the skeleton A(:, J[0:k]).  Returns (col, row) dicts."""
    a = np.asarray(a, dtype=np.float64)
    col = interp_decomp(a, k=k, omega=omega)
    row = row_id(a[:, col["J"][:k]], k)
    return col, row


def two_sided_reconstruct(a: np.ndarray, col, row, k: int) -> np.ndarray:
    """X A(I[0:k], J[0:k]) P with X(I[0:k], :) = I_k, X(I[k:], :) = Tr^T."""
    a = np.asarray(a, dtype=np.float64)
    m, n = a.shape
    X = coefficient_matrix(row["J"], row["T"], k, m).T
    P = coefficient_matrix(col["J"], col["T"], k, n)
    return X @ a[np.ix_(row["J"][:k], col["J"][:k])] @ P


# ------------------------------------------------------ Algorithm 2 (low ID)

def low_cast(a: np.ndarray, fmt: str, block_rows: int = 64) -> np.ndarray:
    """A_L = fl(A) of Algorithm 2 with power-of-two scaling per (row block, column):
    the first piece of ``quantize`` times 2^shift (FP64 values)."""
    pieces, shifts, _ = quantize(a, fmt, block_rows, 1)
    m = pieces.shape[1]
    scale = np.repeat(2.0 ** shifts.astype(np.float64), block_rows, axis=0)[:m]
    return np.asfortranarray(pieces[0] * scale)


def low_id(a: np.ndarray, fmt: str, k: int, block_rows: int = 64):
    """Algorithm 2 without a sketch: the ID of A_L = low_cast(A).  Returns the ID of A_L
    (dict as interp_decomp) with A_L added under "AL"; the mixed approximation is
    reconstruct(A, J, T, k), the low one reconstruct(AL, J, T, k) (Sec. 2)."""
    al = low_cast(a, fmt, block_rows)
    out = interp_decomp(al, k=k)
    out["AL"] = al
    return out


# ------------------------------------------------------------ reconstruction

def coefficient_matrix(J: np.ndarray, T: np.ndarray, k: int, n: int) -> np.ndarray:
    """P with P(:, J[0:k]) = I_k and P(:, J[k:n]) = T (Algorithm 1)."""
    P = np.zeros((k, n), dtype=np.float64)
    P[:, J[:k]] = np.eye(k)
    P[:, J[k:]] = T
    return P


def reconstruct(a: np.ndarray, J: np.ndarray, T: np.ndarray, k: int) -> np.ndarray:
    """A_hat = A(:, J[0:k]) P, evaluated in FP64 (Remark after Lemma 1)."""
    a = np.asarray(a, dtype=np.float64)
    return a[:, J[:k]] @ coefficient_matrix(J, T, k, a.shape[1])


def residual_fro2(a: np.ndarray, J: np.ndarray, T: np.ndarray, k: int) -> float:
    a = _f64(a)
    T = _f64(T) if T.size else np.zeros((1, 1))
    J = np.ascontiguousarray(J, dtype=np.int32)
    return _L().orc_residual_fro2(_ptr(a), a.shape[0], a.shape[1], a.shape[0], k, _ptr(J),
                                  _ptr(T), max(T.shape[0], 1))


def two_norm(x: np.ndarray) -> float:
    """Spectral norm ||x||_2 (the error metric of Sec. 3).

    Moderate sizes: LAPACK's SVD (numpy).  Larger ones: the square root of the
    largest eigenvalue of the smaller Gram matrix x^T x or x x^T (LAPACK's
    symmetric eigensolver), the plain identity ||x||_2^2 = lambda_max(x^T x); the
    largest eigenvalue of a Gram matrix is computed to a relative accuracy of a
    modest multiple of the FP64 unit round-off, far below every tolerance the
    tests apply to norms.
    """
    x = np.asarray(x, dtype=np.float64)
    if x.size == 0:
        return 0.0
    if min(x.shape) <= 2000 and x.size <= 4_000_000:
        return float(np.linalg.norm(x, 2))
    g = x.T @ x if x.shape[1] <= x.shape[0] else x @ x.T
    lam = float(np.linalg.eigvalsh(g)[-1])
    return float(np.sqrt(max(lam, 0.0)))


def rel_err(a: np.ndarray, J: np.ndarray, T: np.ndarray, k: int, norm: str = "2") -> float:
    """||A - A(:,J) P|| / ||A|| in the 2-norm (the paper's metric, Sec. 3) or Frobenius."""
    a = np.asarray(a, dtype=np.float64)
    res = a[:, J[k:]] - a[:, J[:k]] @ T if k < a.shape[1] else np.zeros((a.shape[0], 0))
    if norm == "fro":
        return float(np.linalg.norm(res) / np.linalg.norm(a))
    return two_norm(res) / two_norm(a)


def id_distance(a: np.ndarray, J1, T1, k1, J2, T2, k2) -> float:
    """||A_hat_1 - A_hat_2||_2 / ||A||_2 (the Sec. 3.1 comparison between two IDs)."""
    return two_norm(reconstruct(a, J1, T1, k1) - reconstruct(a, J2, T2, k2)) / two_norm(a)


def lemma1_bound(k: int, n: int, sigma_next: float) -> float:
    """sqrt(1 + k(n-k)) sigma_{k+1}: Lemma 1 (Sec. 2) bound on the best rank-k ID."""
    return float(np.sqrt(1.0 + k * (n - k)) * sigma_next)


def cpqr_bound(k: int, n: int, sigma_next: float) -> float:
    """sqrt(1 + k(n-k)) 2^k sigma_{k+1}: bound for the greedy (CPQR) ID."""
    return float(np.sqrt(1.0 + k * (n - k)) * 2.0 ** k * sigma_next)


# ------------------------------------------------------------- brute force

def brute_force(a: np.ndarray, k: int):
    """Every k-subset of columns on a tiny input.

    For each subset S: err_S = ||A - A_S A_S^+ A||_2 (best coefficients for S,
    via LAPACK lstsq) and vol_S = |det| of the k x k Gram root.  Returns
    (best_err, best_subset, maxvol_subset, maxvol_P) where maxvol_P is the
    coefficient matrix of the max-volume subset (P = A_S^+ A).
    """
    import itertools
    a = np.asarray(a, dtype=np.float64)
    n = a.shape[1]
    best, best_s, vol_best, vol_s = np.inf, None, -1.0, None
    for s in itertools.combinations(range(n), k):
        x = a[:, s]
        coef, *_ = np.linalg.lstsq(x, a, rcond=None)
        e = np.linalg.norm(a - x @ coef, 2)
        if e < best:
            best, best_s = e, s
        sv = np.linalg.svd(x, compute_uv=False)
        vol = float(np.prod(sv))
        if vol > vol_best:
            vol_best, vol_s = vol, s
    coef, *_ = np.linalg.lstsq(a[:, vol_s], a, rcond=None)
    return best, best_s, vol_s, coef


# -------------------------------------------------------------- the adjoint

def adjoint_ref(a: np.ndarray, J: np.ndarray, k: int, gbar: np.ndarray | None,
                tbar: np.ndarray | None) -> np.ndarray:
    """Gradient of L(A_hat, T) w.r.t. A with the pivots J held fixed, FP64.

    With X = A(:,J[0:k]), C = A(:,J[k:n]), T = X^+ C and
    A_hat = [X, X T] (in the column order of J):
      C_bar = Pi G_c + X^+T T_bar,
      X_bar = G_s + (I - Pi) G_c T^T + (I - Pi) C G_c^T X^+T
              - X^+T T_bar T^T + (I - Pi) C T_bar^T (X^T X)^-1,
    Pi = X X^+, G_s / G_c the skeleton / complement columns of dL/dA_hat.
    (Least-squares derivatives of Golub and Pereyra, derived for this
    fixed-pivot map; X^+ by LAPACK SVD.)
    """
    a = np.asarray(a, dtype=np.float64)
    m, n = a.shape
    Js, Jc = J[:k], J[k:]
    X, C = a[:, Js], a[:, Jc]
    Xp = np.linalg.pinv(X)
    T = Xp @ C
    Pi = X @ Xp
    I = np.eye(m)
    Gs = np.zeros((m, k)) if gbar is None else np.asarray(gbar, np.float64)[:, Js]
    Gc = np.zeros((m, n - k)) if gbar is None else np.asarray(gbar, np.float64)[:, Jc]
    Tb = np.zeros((k, n - k)) if tbar is None else np.asarray(tbar, np.float64)
    XtXi = np.linalg.inv(X.T @ X)
    Cbar = Pi @ Gc + Xp.T @ Tb
    Xbar = (Gs + (I - Pi) @ Gc @ T.T + (I - Pi) @ C @ Gc.T @ Xp.T
            - Xp.T @ Tb @ T.T + (I - Pi) @ C @ Tb.T @ XtXi)
    out = np.zeros_like(a)
    out[:, Js] = Xbar
    out[:, Jc] = Cbar
    return out


def fixed_pivot_forward(a: np.ndarray, J: np.ndarray, k: int):
    """(A_hat, T) of the fixed-pivot map used by the adjoint: T = X^+ C, A_hat = A(:,J) P."""
    a = np.asarray(a, dtype=np.float64)
    X, C = a[:, J[:k]], a[:, J[k:]]
    T = np.linalg.lstsq(X, C, rcond=None)[0]
    return reconstruct(a, J, T, k), T
