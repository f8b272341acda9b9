"""Algorithm 2 on the whole matrix (the low_* precisions) and the two approximations of
Sec. 2, through the C ABI, against the FP64 oracle.

* A_L (id_low_cast): bit-exact against the oracle's scaled cast, both formats, FP64 and
  FP32 input, on data spanning many binades with ragged blocks;
* the ID of A_L on the paper's Slow / Medium / Fast matrices (1000 x 1000, sigma_i =
  i^-1, i^-2, i^-4): pivots equal the oracle's ID of the same A_L up to its first step
  whose two leading norms are within 1e-3 (the GPU pivots in FP32), and both
  approximations meet the matched-accuracy criterion against the oracle's:
  e_X <= 1.1 e_X,oracle + 10 u32 for X = M (A_hat_M = A_D(:,J) P) and X = L
  (A_hat_L = A_L(:,J) P), e the relative 2-norm error against A_D;
* id_reconstruct_one against the FP64 product A(:,J[:k]) P, FP64 and FP32.
"""
import numpy as np
import pytest
import torch

import workloads as wl

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
FMT = {"low_bf16": "bf16", "low_f16": "f16"}


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


def rel2(orc, x, a):
    return orc.two_norm(x) / orc.two_norm(a)


@pytest.mark.parametrize("precision", ["low_bf16", "low_f16"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_low_cast_bit_exact(gid, dev, orc, precision, dtype):
    rng = np.random.default_rng(11)
    m, n = 333, 29
    a = rng.standard_normal((m, n)) * 10.0 ** rng.uniform(-8, 8, (m, n))
    a[:, 4] = 0.0
    a[70:140, 6] *= 1e-20
    a = np.asfortranarray(a.astype(dtype))
    al = gid.low_cast(torch.from_numpy(a).to(dev), precision).cpu().numpy().astype(np.float64)
    ref = orc.low_cast(a, FMT[precision])
    assert np.array_equal(al, ref)


@pytest.mark.parametrize("precision", ["low_bf16", "low_f16"])
@pytest.mark.parametrize("kind,k", [("slow", 20), ("medium", 20), ("fast", 20), ("fast", 51)])
def test_low_id_paper_datasets(gid, dev, orc, precision, kind, k):
    a = wl.paper_dataset(kind, seed=21)
    fmt = FMT[precision]
    ref = orc.low_id(a, fmt, k)
    at = torch.from_numpy(a).to(dev)
    res = gid.id_factor(at, k, precision=precision)
    assert res.info == 0 and res.k == k
    J = res.J.cpu().numpy()
    assert sorted(J.tolist()) == list(range(a.shape[1]))
    close = ref["gaps"] < 1e-3
    first = int(np.argmax(close)) if np.any(close) else k
    assert np.array_equal(J[:first], ref["J"][:first])
    al_dev = gid.low_cast(at, precision)
    hm = gid.reconstruct(at, res.J, res.T, k).cpu().numpy()
    hl = gid.reconstruct(al_dev, res.J, res.T, k).cpu().numpy().astype(np.float64)
    e_m, e_l = rel2(orc, a - hm, a), rel2(orc, a - hl, a)
    ref_m = orc.reconstruct(a, ref["J"], ref["T"], k)
    ref_l = orc.reconstruct(ref["AL"], ref["J"], ref["T"], k)
    r_m, r_l = rel2(orc, a - ref_m, a), rel2(orc, a - ref_l, a)
    assert e_m <= 1.1 * r_m + 10 * U32, (e_m, r_m)
    assert e_l <= 1.1 * r_l + 10 * U32, (e_l, r_l)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_reconstruct_one(gid, dev, orc, dtype):
    rng = np.random.default_rng(12)
    m, n, k = 517, 203, 37
    a = np.asfortranarray(rng.standard_normal((m, n)))
    J = rng.permutation(n).astype(np.int32)
    T = rng.standard_normal((k, n - k))
    ref = orc.reconstruct(a.astype(dtype).astype(np.float64), J, T, k)
    Td = torch.from_numpy(np.asfortranarray(T)).to(dev)
    got = gid.reconstruct(torch.from_numpy(a.astype(dtype)).to(dev), torch.from_numpy(J).to(dev), Td, k)
    got = got.cpu().numpy().astype(np.float64)
    tol = 1e-13 if dtype == np.float64 else 2e-6
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))
    assert np.array_equal(got[:, J[:k]], a.astype(dtype)[:, J[:k]].astype(np.float64))
