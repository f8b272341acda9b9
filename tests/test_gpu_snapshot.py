"""Rank by tolerance and the FP64 error estimate on snapshot-style FP32 data (the
travelling-sinusoid matrices standing in for the paper's particle-laden-flow
snapshots), through the C ABI, against the FP64 oracle.

* rank: the sketched mixed path stops on the sketch's remaining norm; with an
  FP32-accurate sketch (BF16x3) the rank equals the oracle's on the same Omega
  within one step either way (the stopping norm is an FP32 downdate);
* error estimate: the FP64 Frobenius residual the library returns equals the
  oracle's ||A - A(:,J) P||_F / ||A||_F at the GPU's own J, T to 1e-10 relative;
* FP16 sketch: E1 (e_M <= 1.1 e_D + 10 u_16) at a fixed rank, and the rank the
  FP16 sketch picks at tolerance 1e-6 is reported against its rounding floor.
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


@pytest.fixture(scope="module")
def dev():
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def snap():
    c = wl.config3(m=16384, n=500)
    return c["A"]                      # FP32, column-major


def omega_dev(bits, dev, fmt):
    t = torch.from_numpy(np.ascontiguousarray(bits).view(np.int16)).to(dev)
    return t.view(torch.bfloat16 if fmt == "bf16" else torch.float16)


def fro_err(a64, J, T, k):
    res = a64[:, J[k:]] - a64[:, J[:k]] @ T if k < a64.shape[1] else np.zeros((a64.shape[0], 0))
    return float(np.linalg.norm(res) / np.linalg.norm(a64))


def test_snapshot_rank_by_tolerance_bf16x3(gid, dev, orc, snap):
    a = snap
    a64 = a.astype(np.float64)
    kmax, tol = 120, 1e-6
    om, bits = wl.gaussian_omega(kmax + 10, a.shape[0], 301, "bf16")
    ref = orc.interp_decomp(a64, tol=tol, k_max=kmax, omega=om)
    res = gid.id_factor(torch.from_numpy(a).to(dev), tol=tol, k_max=kmax, precision="mixed_bf16x3",
                        omega=omega_dev(bits, dev, "bf16"), estimate_error=True)
    assert res.info == 0
    assert abs(res.k - ref["k"]) <= 1, (res.k, ref["k"])
    J, T = res.J.cpu().numpy(), res.T.cpu().numpy()
    e = fro_err(a64, J, T, res.k)
    assert abs(res.err - e) <= 1e-10 * max(e, 1e-300)
    # the rank the sketch picked leaves a residual at the tolerance's scale
    assert e <= 10 * tol


def test_snapshot_error_estimate_full_size(gid, dev, orc):
    """The 65536 x 1000 snapshot matrix: the FP64 estimate equals the exact relative
    Frobenius residual of the returned ID (numpy FP64 on the host)."""
    c = wl.config3()
    a = c["A"]
    kmax = 100
    om, bits = wl.gaussian_omega(kmax + 10, a.shape[0], 302, "bf16")
    res = gid.id_factor(torch.from_numpy(a).to(dev), tol=1e-6, k_max=kmax, precision="mixed_bf16x3",
                        omega=omega_dev(bits, dev, "bf16"), estimate_error=True)
    assert res.info == 0 and 0 < res.k <= kmax
    e = fro_err(a.astype(np.float64), res.J.cpu().numpy(), res.T.cpu().numpy(), res.k)
    assert abs(res.err - e) <= 1e-10 * e


def test_snapshot_f16_sketch(gid, dev, orc, snap):
    """FP16 sketch of the FP32 snapshots: E1 at a fixed rank.  At tolerance 1e-6 the
    half-precision cast's rounding noise (about 1.8e-5 of ||A||, well above the
    tolerance) stays in the sketch's remaining norm, so the stopping test never fires
    and the rank runs to k_max, while the FP32-accurate three-piece sketch stops
    below it."""
    a = snap
    a64 = a.astype(np.float64)
    k = 60
    om, bits = wl.gaussian_omega(k + 10, a.shape[0], 303, "f16")
    ref = orc.interp_decomp(a64, k=k, omega=om)
    res = gid.id_factor(torch.from_numpy(a).to(dev), k, precision="mixed_f16", omega=omega_dev(bits, dev, "f16"))
    assert res.info == 0 and res.k == k
    e_m = orc.rel_err(a64, res.J.cpu().numpy(), res.T.cpu().numpy(), k)
    e_d = orc.rel_err(a64, ref["J"], ref["T"], k)
    assert e_m <= 1.1 * e_d + 10 * 2.0 ** -11
    kmax = 120
    om2, bits2 = wl.gaussian_omega(kmax + 10, a.shape[0], 304, "f16")
    r16 = gid.id_factor(torch.from_numpy(a).to(dev), tol=1e-6, k_max=kmax, precision="mixed_f16",
                        omega=omega_dev(bits2, dev, "f16"))
    om3, bits3 = wl.gaussian_omega(kmax + 10, a.shape[0], 304, "bf16")
    r3 = gid.id_factor(torch.from_numpy(a).to(dev), tol=1e-6, k_max=kmax, precision="mixed_bf16x3",
                       omega=omega_dev(bits3, dev, "bf16"))
    assert r16.info == 0 and r3.info == 0
    assert r16.k == kmax, r16.k
    assert 0 < r3.k < kmax, r3.k


def test_snapshot_plain_f64_tolerance(gid, dev, orc, snap):
    """The plain FP64 path on the same FP32 data (no sketch): rank and pivots of the
    oracle's exact-norm CPQR at tolerance 1e-6."""
    a = snap[:4096, :300].copy(order="F")
    a64 = a.astype(np.float64)
    ref = orc.interp_decomp(a64, tol=1e-6, k_max=150)
    res = gid.id_factor(torch.from_numpy(a64.copy(order="F")).to(dev), tol=1e-6, k_max=150, precision="plain_f64")
    assert res.info == 0
    assert abs(res.k - ref["k"]) <= 1
    sep = ref["gaps"] >= 1e-8
    first = int(np.argmax(~sep)) if np.any(~sep) else min(res.k, ref["k"])
    first = min(first, res.k, ref["k"])
    assert np.array_equal(res.J.cpu().numpy()[:first], ref["J"][:first])
