"""Adjoint of the fixed-pivot ID (a8) and the reconstruction, GPU vs the FP64 oracle.

Tolerances: the GPU runs in FP32.  The adjoint applies R^-1 and R^-T of the skeleton's
thin QR, which amplify FP32 rounding by kappa(X); its relative Frobenius difference from
the FP64 reference gradient is bounded by 10 kappa(X) u32 (u32 = 2^-24), floored at 1e-5
(the gate for well-conditioned skeletons).  End to end (GPU pivots and T from the FP32
pivoted QR) the same bound plus the FP32 error of T; central differences (step 1e-4,
FP64) agree to 1e-3.
"""
import numpy as np
import pytest
import torch

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gid():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2012_00706_gb300 as g
    g.load()
    return g


def _case(batch, m, n, k, seed, decay=0.85):
    rng = np.random.default_rng(seed)
    sig = decay ** np.arange(n)
    A = np.stack([wl.lowrank(m, n, sig, seed * 31 + b) for b in range(batch)]).astype(np.float32)
    G = rng.standard_normal((batch, m, n)).astype(np.float32)
    Tb = rng.standard_normal((batch, k, n - k))
    return A, G, Tb


def _dev_cm(x, dev):
    """(batch, m, n) numpy -> CUDA tensor with column-major matrices."""
    return torch.from_numpy(np.ascontiguousarray(np.swapaxes(x, 1, 2))).to(dev).transpose(1, 2)


@pytest.mark.parametrize("batch,m,n,k", [(3, 300, 80, 12), (2, 700, 150, 33), (1, 129, 40, 40), (2, 2048, 512, 32),
                                         (2, 2048, 512, -32)])
def test_backward_matches_fp64_reference(gid, orc, batch, m, n, k):
    """k < 0 marks the differentiable workload's spectrum: exact rank 32, sigma_i = 10^(-i/16)."""
    dev = torch.device("cuda:0")
    if k < 0:
        k = -k
        A = wl.config5(count=batch, m=m, n=n, rank=k, seed=15)["A"]
        rng = np.random.default_rng(16)
        G = rng.standard_normal((batch, m, n)).astype(np.float32)
        Tb = rng.standard_normal((batch, k, n - k))
    else:
        A, G, Tb = _case(batch, m, n, k, seed=m + n + k)
    Js, Ts, refs = [], [], []
    for b in range(batch):
        a64 = A[b].astype(np.float64)
        J = orc.interp_decomp(a64, k=k)["J"]
        T = np.linalg.lstsq(a64[:, J[:k]], a64[:, J[k:]], rcond=None)[0]
        Js.append(J)
        Ts.append(T)
        refs.append(orc.adjoint_ref(a64, J, k, G[b].astype(np.float64), Tb[b]))
    Jt = torch.from_numpy(np.stack(Js).astype(np.int32)).to(dev)
    Tt = _dev_cm(np.stack(Ts), dev) if n > k else torch.zeros((batch, k, 0), dtype=torch.float64, device=dev)
    dA = gid.id_backward(_dev_cm(A, dev), Jt, Tt, k, _dev_cm(G, dev),
                         _dev_cm(Tb, dev) if n > k else None).cpu().numpy()
    for b in range(batch):
        kappa = np.linalg.cond(A[b].astype(np.float64)[:, Js[b][:k]])
        rel = np.linalg.norm(dA[b] - refs[b]) / np.linalg.norm(refs[b])
        assert rel <= max(1e-5, 10.0 * kappa * 2.0 ** -24), (b, rel, kappa)


def test_backward_only_one_cotangent(gid, orc):
    """dL/dA_hat alone and dL/dT alone (the other argument null)."""
    dev = torch.device("cuda:0")
    A, G, Tb = _case(2, 200, 60, 10, seed=3)
    for use_g in (True, False):
        Js, Ts, refs = [], [], []
        for b in range(2):
            a64 = A[b].astype(np.float64)
            J = orc.interp_decomp(a64, k=10)["J"]
            T = np.linalg.lstsq(a64[:, J[:10]], a64[:, J[10:]], rcond=None)[0]
            Js.append(J)
            Ts.append(T)
            refs.append(orc.adjoint_ref(a64, J, 10, G[b].astype(np.float64) if use_g else None,
                                        None if use_g else Tb[b]))
        dA = gid.id_backward(_dev_cm(A, dev), torch.from_numpy(np.stack(Js).astype(np.int32)).to(dev),
                             _dev_cm(np.stack(Ts), dev), 10, _dev_cm(G, dev) if use_g else None,
                             None if use_g else _dev_cm(Tb, dev)).cpu().numpy()
        for b in range(2):
            kappa = np.linalg.cond(A[b].astype(np.float64)[:, Js[b][:10]])
            assert np.linalg.norm(dA[b] - refs[b]) / np.linalg.norm(refs[b]) <= max(1e-5, 10.0 * kappa * 2.0 ** -24)


def test_reconstruct_matches_oracle(gid, orc):
    dev = torch.device("cuda:0")
    A, _, _ = _case(2, 250, 70, 15, seed=9)
    for b in range(2):
        a64 = A[b].astype(np.float64)
        out = orc.interp_decomp(a64, k=15)
        res_J = torch.from_numpy(out["J"].astype(np.int32)).to(dev)
        T = torch.from_numpy(np.asfortranarray(out["T"])).to(dev)
        Ah = gid.id_reconstruct(torch.from_numpy(np.asfortranarray(A[b])).to(dev), res_J, T, 15).cpu().numpy()
        ref = orc.reconstruct(a64, out["J"], out["T"], 15)
        assert np.max(np.abs(Ah - ref)) <= 1e-5 * np.max(np.abs(ref))
        assert np.array_equal(Ah[:, out["J"][:15]], A[b][:, out["J"][:15]])


def test_autograd_end_to_end_and_finite_differences(gid, orc):
    """Loss ||A_hat(:, Jc) - B||_F^2 (the differentiable workload) through IDFunction:
    gradient vs the FP64 reference gradient (1e-4) and vs central differences (1e-3)."""
    dev = torch.device("cuda:0")
    m, n, k = 256, 64, 8
    sigma = 10.0 ** (-np.arange(1, k + 1) / 16.0)
    A = wl.lowrank(m, n, sigma, 5).astype(np.float32)
    B = np.random.default_rng(6).standard_normal((m, n - k)).astype(np.float32)
    At = torch.from_numpy(np.asfortranarray(A)).to(dev).requires_grad_(True)
    Ahat, T, J = gid.IDFunction.apply(At, k)
    Jn = J.cpu().numpy()
    Bt = torch.from_numpy(B).to(dev)
    loss = ((Ahat[:, J[k:].long()] - Bt) ** 2).sum()
    loss.backward()
    g_gpu = At.grad.cpu().numpy().astype(np.float64)
    a64 = A.astype(np.float64)
    ah, _ = orc.fixed_pivot_forward(a64, Jn, k)
    Gfull = np.zeros((m, n))
    Gfull[:, Jn[k:]] = 2.0 * (ah[:, Jn[k:]] - B)
    ref = orc.adjoint_ref(a64, Jn, k, Gfull, None)
    kappa = np.linalg.cond(a64[:, Jn[:k]])
    assert np.linalg.norm(g_gpu - ref) / np.linalg.norm(ref) <= max(1e-4, 20.0 * kappa * 2.0 ** -24)

    def loss64(x):
        ahx, _ = orc.fixed_pivot_forward(x, Jn, k)
        return float(np.sum((ahx[:, Jn[k:]] - B) ** 2))

    rng = np.random.default_rng(7)
    h = 1e-4
    for _ in range(25):
        i, j = int(rng.integers(m)), int(rng.integers(n))
        e = np.zeros_like(a64)
        e[i, j] = h
        fd = (loss64(a64 + e) - loss64(a64 - e)) / (2 * h)
        assert abs(fd - g_gpu[i, j]) <= 1e-3 * max(1.0, np.max(np.abs(ref)))
