"""Seeded synthetic inputs for the column interpolative decomposition (ID).

This module only *draws* inputs: random orthonormal factors, singular-value
profiles, snapshot matrices and Gaussian test matrices.  It holds none of the
ID's own arithmetic (no pivoting, no QR of the data, no coefficient solve), so
both the FP64 CPU oracle and the GPU path can consume the same arrays.

Shapes and value distributions follow the workloads of the paper:

* ``paper_dataset`` -- the Slow/Medium/Fast matrices of Sec. 3 (singular
  values i^-1, i^-2, i^-4, 1000x1000, inputs of width n are the first n
  columns; Table 2).
* ``config_*`` -- the five benchmark workloads built around the ID hot path
  (plain FP64 ID, sketched mixed-precision ID, snapshot matrix, uneven batch,
  differentiable batch).

Orthonormal factors are Gaussian matrices orthonormalised by numpy's QR with
the signs fixed by diag(R), so a seed gives the same factors on any machine up
to LAPACK rounding.  Every function takes an explicit seed.
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = [
    "orthonormal", "lowrank", "paper_sigma", "paper_dataset", "gaussian_omega",
    "config1", "config2", "config3", "config4", "config5", "BatchItem",
    "separated_matrix", "exact_triangular_id_matrix", "to_bf16_bits", "to_f16_bits", "lowrank_device",
    "config4_device",
]


def orthonormal(rng: np.random.Generator, m: int, n: int) -> np.ndarray:
    """m x n matrix with orthonormal columns: QR of a Gaussian draw, signs fixed."""
    g = rng.standard_normal((m, n))
    q, r = np.linalg.qr(g, mode="reduced")
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s[None, :]


def lowrank(m: int, n: int, sigma: np.ndarray, seed: int, dtype=np.float64) -> np.ndarray:
    """A = U diag(sigma) V^T with seeded orthonormal U (m x r), V (n x r), r = len(sigma).

    Returned in Fortran (column-major) order, the layout the ID works on.
    """
    rng = np.random.default_rng(seed)
    r = len(sigma)
    u = orthonormal(rng, m, r)
    v = orthonormal(rng, n, r)
    a = (u * np.asarray(sigma, dtype=np.float64)[None, :]) @ v.T
    return np.asfortranarray(a.astype(dtype))


def paper_sigma(kind: str, n: int = 1000) -> np.ndarray:
    """Singular values of the Slow/Medium/Fast datasets (Sec. 3, Table 2)."""
    p = {"slow": 1.0, "medium": 2.0, "fast": 4.0}[kind]
    i = np.arange(1, n + 1, dtype=np.float64)
    return i ** (-p)


def paper_dataset(kind: str, ncols: int | None = None, m: int = 1000, n: int = 1000,
                  seed: int = 0) -> np.ndarray:
    """Slow/Medium/Fast test matrix of Sec. 3; ``ncols`` keeps the first columns."""
    a = lowrank(m, n, paper_sigma(kind, min(m, n)), seed)
    if ncols is not None:
        a = np.asfortranarray(a[:, :ncols])
    return a


def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float values to bfloat16 (round-to-nearest-even, via torch) and return uint16 bits."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.bfloat16)
    return t.view(torch.int16).numpy().view(np.uint16)


def to_f16_bits(x: np.ndarray) -> np.ndarray:
    """Round float values to IEEE half (numpy's round-to-nearest-even) and return uint16 bits."""
    return np.ascontiguousarray(x, dtype=np.float16).view(np.uint16)


def _bits_to_f64(bits: np.ndarray, fmt: str) -> np.ndarray:
    if fmt == "f16":
        return bits.view(np.float16).astype(np.float64)
    b32 = bits.astype(np.uint32) << 16
    return b32.view(np.float32).astype(np.float64)


def gaussian_omega(ell: int, m: int, seed: int, fmt: str = "bf16"):
    """Gaussian test matrix Omega (ell x m, row-major: row i contiguous).

    The N(0,1) draws are rounded once to ``fmt`` so that Omega is exactly
    representable in the low format and adds no rounding of its own.  Returns
    ``(omega_f64, omega_bits)``: the values as float64 and the uint16 bit
    patterns the GPU reads.
    """
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((ell, m)).astype(np.float32)
    bits = to_bf16_bits(g) if fmt == "bf16" else to_f16_bits(g)
    return _bits_to_f64(bits, fmt).reshape(ell, m), bits.reshape(ell, m)


def separated_matrix(m: int, n: int, seed: int, decay: float = 0.93) -> np.ndarray:
    """Full-rank matrix whose greedy column norms stay well separated.

    Columns are Gaussian scaled by decay^j (in a shuffled order), which keeps
    the largest residual norm clearly ahead of the runner-up at every step of
    a pivoted QR, so that pivot choices do not depend on rounding.
    """
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((m, n))
    scale = decay ** rng.permutation(n).astype(np.float64)
    return np.asfortranarray(g * scale[None, :])


# ---------------------------------------------------------------- workloads

def config1(seed: int = 1):
    """Plain FP64 ID: 1000x500, sigma_i = 10^(-i/25), k = 50, no sketch."""
    m, n, k = 1000, 500, 50
    sigma = 10.0 ** (-np.arange(1, n + 1) / 25.0)
    return {"A": lowrank(m, n, sigma, seed), "m": m, "n": n, "k": k}


def config2(seed: int = 2, m: int = 20000, n: int = 2000, k: int = 100, p: int = 10,
            omega_fmt: str = "bf16"):
    """Sketched ID: m x n FP64, sigma_i = i^-2, k = 100, ell = k + 10, Gaussian Omega."""
    sigma = np.arange(1, min(m, n) + 1, dtype=np.float64) ** -2.0
    a = lowrank(m, n, sigma, seed)
    om, bits = gaussian_omega(k + p, m, seed + 1000, omega_fmt)
    return {"A": a, "m": m, "n": n, "k": k, "ell": k + p, "omega": om, "omega_bits": bits}


def config3(seed: int = 3, m: int = 65536, n: int = 1000, modes: int = 40,
            noise: float = 1e-6, dt: float = 0.01):
    """Snapshot matrix, FP32: each column a sum of travelling sinusoids plus noise.

    A[i, s] = sum_j 0.8^j sin(kappa_j (x_i - c_j t_s) + phi_j) + noise * N(0,1),
    x_i = 2 pi i / m, kappa_j = j + 1, c_j ~ U[0.5, 2], phi_j ~ U[0, 2 pi),
    t_s = dt * s.  Built as Phi Psi^T through the angle-addition identity.
    """
    rng = np.random.default_rng(seed)
    x = 2.0 * np.pi * np.arange(m) / m
    t = dt * np.arange(n)
    kap = np.arange(1, modes + 1, dtype=np.float64)
    c = rng.uniform(0.5, 2.0, modes)
    phi = rng.uniform(0.0, 2.0 * np.pi, modes)
    amp = 0.8 ** np.arange(modes)
    theta = phi[None, :] - (kap * c)[None, :] * t[:, None]          # n x modes
    phi_mat = np.concatenate([np.sin(np.outer(x, kap)), np.cos(np.outer(x, kap))], axis=1)
    psi_mat = np.concatenate([np.cos(theta) * amp, np.sin(theta) * amp], axis=1)
    a = phi_mat @ psi_mat.T
    a += noise * rng.standard_normal((m, n))
    return {"A": np.asfortranarray(a.astype(np.float32)), "m": m, "n": n, "tol": 1e-6}


@dataclasses.dataclass
class BatchItem:
    m: int
    n: int
    r: int
    A: np.ndarray


def config4_shapes(count: int = 512, seed: int = 4, m_range=(256, 4096), n_range=(64, 1024),
                   r_range=(8, 128)):
    """(m, n, r) triples of the uneven batch: m, n uniform, n redrawn until n <= m, r clipped to n."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        while True:
            n = int(rng.integers(n_range[0], n_range[1] + 1))
            if n <= m:
                break
        r = min(int(rng.integers(r_range[0], r_range[1] + 1)), n)
        out.append((m, n, r))
    return out


def config4(count: int = 512, seed: int = 4, **kw):
    """Uneven batch of FP64 matrices with exact rank r and sigma_i = 10^(-i/r), i <= r."""
    items = []
    for idx, (m, n, r) in enumerate(config4_shapes(count, seed, **kw)):
        sigma = 10.0 ** (-np.arange(1, r + 1) / r)
        items.append(BatchItem(m, n, r, lowrank(m, n, sigma, seed * 100003 + idx)))
    return items


def lowrank_device(m: int, n: int, sigma, seed: int, device, lda: int | None = None):
    """``lowrank`` with the product formed in GPU memory (for the full-size batch, whose
    4.7 GB the host would take minutes to multiply out).  The orthonormal factors are
    the same numpy draws as ``lowrank``'s; only the product U diag(sigma) V^T runs on
    the device.  Returns (buffer, view): the buffer is n x lda row-major, i.e. the
    m x n view is column-major with leading dimension lda."""
    import torch
    rng = np.random.default_rng(seed)
    r = len(sigma)
    u = orthonormal(rng, m, r)
    v = orthonormal(rng, n, r)
    su = torch.from_numpy(np.ascontiguousarray(u * np.asarray(sigma, dtype=np.float64)[None, :])).to(device)
    tv = torch.from_numpy(np.ascontiguousarray(v)).to(device)
    lda = lda or m
    buf = torch.zeros((n, lda), dtype=torch.float64, device=device)
    buf[:, :m] = tv @ su.T
    return buf, buf.t()[:m]


def config4_device(device, count: int = 512, seed: int = 4, lda_multiple: int = 2, indices=None, **kw):
    """The uneven batch of ``config4`` drawn on the GPU, leading dimensions rounded up to
    a multiple of ``lda_multiple`` (2 doubles = 16 bytes, what TMA needs).  ``indices``
    keeps a subset (one process's share); matrix i is the same whichever subset holds it."""
    all_shapes = config4_shapes(count, seed, **kw)
    keep = list(range(count)) if indices is None else list(indices)
    shapes = [all_shapes[i] for i in keep]
    bufs = []
    for idx, (m, n, r) in zip(keep, shapes):
        sigma = 10.0 ** (-np.arange(1, r + 1) / r)
        lda = (m + lda_multiple - 1) // lda_multiple * lda_multiple
        bufs.append(lowrank_device(m, n, sigma, seed * 100003 + idx, device, lda))
    return shapes, bufs


def config5(count: int = 64, m: int = 2048, n: int = 512, rank: int = 32, seed: int = 5):
    """Differentiable batch: FP32 matrices of exact rank 32, sigma_i = 10^(-i/16); Gaussian B."""
    sigma = 10.0 ** (-np.arange(1, rank + 1) / 16.0)
    a = np.stack([lowrank(m, n, sigma, seed * 7919 + i) for i in range(count)]).astype(np.float32)
    rng = np.random.default_rng(seed + 17)
    b = rng.standard_normal((count, m, n)).astype(np.float32)
    return {"A": a, "B": b, "k": rank, "m": m, "n": n}


def probe_vectors(n: int, s: int, seed: int) -> np.ndarray:
    """Gaussian probe vectors (n x s, column-major) for randomized norm estimates."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((n, s)))


def sinusoid_rank(modes: int) -> int:
    """Exact rank of the noiseless snapshot matrix: two per travelling mode."""
    return 2 * modes


def exact_triangular_id_matrix(k: int = 24, n: int = 224, rows: int = 40, c: float = 0.5, seed: int = 0):
    """FP32 matrix whose column-pivoted Householder QR is exact in FP32 and FP64.

    Columns perm[0..k-1] hold an upper-triangular W11 (rows 0..k-1) with diagonal
    2^0, 2^-1, ..., 2^-(k-1) and off-diagonal entries c 2^-i u in column i (u uniform
    in [-1, 1], rounded to FP32); the other n - k columns hold c 2^-r u in row r < k;
    rows k..rows-1 are zero.  Greedy pivoting then takes the triangular columns in
    order (each step's leading residual norm is at least twice the runner-up's), every
    reflector maps a multiple of a unit vector (v = e_j, tau = 2), and R equals -W
    exactly.  The condition number of W11 is at least 2^(k-1).  Returns (W, perm)."""
    rng = np.random.default_rng(seed)
    w = np.zeros((rows, n), dtype=np.float64)
    d = 2.0 ** -np.arange(k)
    tri = np.triu(c * rng.uniform(-1.0, 1.0, (k, k)) * d[None, :], 1) + np.diag(d)
    rest = c * rng.uniform(-1.0, 1.0, (k, n - k)) * d[:, None]
    perm = rng.permutation(n)
    w[:k, perm[:k]] = tri
    w[:k, perm[k:]] = rest
    return np.asfortranarray(w.astype(np.float32)), perm
