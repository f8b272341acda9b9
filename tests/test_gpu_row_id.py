"""Row and two-sided IDs (id_factor_rows, id_factor_two_sided) against the FP64 oracle,
through the C ABI.

* plain FP64 row ID on separated rows: the oracle's row indices and T (the column ID of
  A^T), including a ragged shape whose transpose crosses the 32 x 32 tiles unevenly;
* sketched BF16x3 row ID: e_M <= 1.1 e_D + 10 u32 against the oracle's sketched row ID
  with the same Omega (ell x n);
* two-sided FP64: the oracle's column and row indices, and a reconstruction error equal
  to the column ID's (the rank-k row ID of the skeleton is exact).
"""
import numpy as np
import pytest
import torch

import workloads as wl

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


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


@pytest.mark.parametrize("m,n,k", [(300, 700, 25), (333, 97, 30)])
def test_row_id_plain_f64(gid, dev, orc, m, n, k):
    a = np.asfortranarray(wl.separated_matrix(n, m, seed=m + n, decay=0.9).T)   # separated rows
    ref = orc.row_id(a, k)
    assert np.min(ref["gaps"]) >= 1e-8
    res = gid.id_factor_rows(torch.from_numpy(a).to(dev), k, estimate_error=True)
    assert res.info == 0 and res.k == k
    assert np.array_equal(res.J.cpu().numpy(), ref["J"])
    T = res.T.cpu().numpy()
    assert np.max(np.abs(T - ref["T"])) <= 1e-9 * max(1.0, np.max(np.abs(ref["T"])))
    e = orc.rel_err(a.T, ref["J"], ref["T"], k, "fro")
    assert abs(res.err - e) <= 1e-10


def test_row_id_sketched_bf16x3(gid, dev, orc):
    m, n, k, ell = 2000, 1500, 40, 50
    a = wl.lowrank(m, n, np.arange(1, min(m, n) + 1, dtype=np.float64) ** -2.0, 51)
    om, bits = wl.gaussian_omega(ell, n, 52, "bf16")
    ldo = (n + 7) // 8 * 8                    # the tensor-core sketch reads Omega rows by TMA
    padded = np.zeros((ell, ldo), dtype=np.uint16)
    padded[:, :n] = bits
    omega = torch.from_numpy(padded.view(np.int16)).to(dev).view(torch.bfloat16)[:, :n]
    res = gid.id_factor_rows(torch.from_numpy(a).to(dev), k, precision="mixed_bf16x3", omega=omega)
    assert res.info == 0 and res.k == k
    ref = orc.row_id(a, k, omega=om)
    e_m = orc.rel_err(a.T, res.J.cpu().numpy(), res.T.cpu().numpy(), k)
    e_d = orc.rel_err(a.T, ref["J"], ref["T"], k)
    assert e_m <= 1.1 * e_d + 10 * U32, (e_m, e_d)


def test_two_sided_plain_f64(gid, dev, orc):
    a = wl.separated_matrix(500, 300, seed=53, decay=0.9)
    k = 20
    col_ref, row_ref = orc.two_sided_id(a, k)
    col, row = gid.id_factor_two_sided(torch.from_numpy(a).to(dev), k)
    assert col.info == 0 and row.info == 0 and col.k == k and row.k == k
    assert np.array_equal(col.J.cpu().numpy(), col_ref["J"])
    assert np.array_equal(row.J.cpu().numpy(), row_ref["J"])
    got = {"J": row.J.cpu().numpy(), "T": row.T.cpu().numpy()}
    cg = {"J": col.J.cpu().numpy(), "T": col.T.cpu().numpy()}
    h = orc.two_sided_reconstruct(a, cg, got, k)
    e2 = np.linalg.norm(a - h) / np.linalg.norm(a)
    e1 = orc.rel_err(a, col_ref["J"], col_ref["T"], k, "fro")
    assert abs(e2 - e1) <= 1e-10
