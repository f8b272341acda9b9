"""Rank-adaptive randomized ID (id_factor_adaptive) against the FP64 oracle's adaptive ID
with the same Omega, through the C ABI.

* plain FP64 (FP64 sketch, FP64 pivoted QR): the same number of sketch rows and the same
  rank as the oracle, the same pivots up to the oracle's first step whose two leading norms
  are within 1e-8, the same residual to 1e-10;
* three-piece bfloat16 sketch: the residual meets the tolerance and the rows used are
  within one block of the oracle's (the sketch is FP32-accurate, not exact);
* an exact-rank matrix stops at the first block whose rank covers it.
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
def problem():
    m, n = 3000, 400
    sig = 10.0 ** (-np.arange(1, n + 1) / 20.0)
    a = wl.lowrank(m, n, sig, 41)
    om, bits = wl.gaussian_omega(160, m, 42, "bf16")
    return a, om, bits


def test_adaptive_plain_f64_matches_oracle(gid, dev, orc, problem):
    a, om, _ = problem
    tol, block, kmax = 1e-5, 16, 150
    ref = orc.adaptive_id(a, om, tol, block, kmax)
    res, ell = gid.id_factor_adaptive(torch.from_numpy(a).to(dev), tol, kmax, torch.from_numpy(om).to(dev),
                                      block=block, precision="plain_f64")
    assert res.info == 0
    assert ell == ref["ell"] and res.k == ref["k"], (ell, ref["ell"], res.k, ref["k"])
    J = res.J.cpu().numpy()
    close = ref["gaps"] < 1e-8
    first = int(np.argmax(close)) if np.any(close) else ref["k"]
    assert first > 10
    assert np.array_equal(J[:first], ref["J"][:first])
    assert abs(res.err - ref["err"]) <= 1e-10
    assert res.err <= tol


def test_adaptive_mixed_meets_tolerance(gid, dev, orc, problem):
    a, om, bits = problem
    tol, block, kmax = 1e-5, 16, 150
    ref = orc.adaptive_id(a, om, tol, block, kmax)
    omega = torch.from_numpy(bits.view(np.int16)).to(dev).view(torch.bfloat16)
    res, ell = gid.id_factor_adaptive(torch.from_numpy(a).to(dev), tol, kmax, omega, block=block,
                                      precision="mixed_bf16x3")
    assert res.info == 0
    assert abs(ell - ref["ell"]) <= block
    e = orc.rel_err(a, res.J.cpu().numpy(), res.T.cpu().numpy(), res.k, "fro")
    assert abs(res.err - e) <= 1e-10 * max(e, 1e-300)
    assert e <= tol


def test_adaptive_exact_rank(gid, dev, orc):
    m, n, r = 2000, 300, 23
    a = wl.lowrank(m, n, 0.8 ** np.arange(r), 43)
    _, bits = wl.gaussian_omega(128, m, 44, "bf16")
    omega = torch.from_numpy(bits.view(np.int16)).to(dev).view(torch.bfloat16)
    res, ell = gid.id_factor_adaptive(torch.from_numpy(a).to(dev), 1e-5, 100, omega, block=16,
                                      precision="mixed_bf16x3")
    assert ell == 48
    assert res.err <= 1e-5
