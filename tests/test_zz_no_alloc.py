"""id_sketch_noalloc: the sketch entry point for callers that cannot allocate device
memory (its scratch is a static device array inside the library).  Checked through
the C ABI against id_sketch, the entry point that takes a caller workspace, on two
calls in a row.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import workloads as wl

pytestmark = pytest.mark.gpu

ID_OK, ID_ERR_WORKSPACE = 0, 2


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2012_00706_gb300 as gid
    L = gid.load()
    p, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    L.id_sketch_noalloc.argtypes = [p, ctypes.c_int, i64, i64, i64, p, i64, i32, i32, p, i64, p, p]
    L.id_sketch_noalloc.restype = ctypes.c_int
    return L


def _noalloc(L, a, omega, precision, ydtype):
    import paper_2012_00706_gb300 as gid
    m, n = a.shape
    ell = omega.shape[0]
    y = torch.empty((n, ell), dtype=ydtype, device=a.device).t()
    info = torch.zeros(1, dtype=torch.int32, device=a.device)
    code = L.id_sketch_noalloc(a.data_ptr(), 0 if a.dtype == torch.float64 else 1, m, n, a.stride(1),
                               omega.data_ptr(), omega.stride(0), ell, gid.PRECISIONS[precision], y.data_ptr(),
                               ell, info.data_ptr(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return code, y, info


@pytest.mark.parametrize("precision", ["mixed_bf16", "plain_f64"])
def test_noalloc_sketch_matches_workspace_sketch(lib, precision):
    import paper_2012_00706_gb300 as gid
    dev = torch.device("cuda:0")
    m, n, ell = 3000, 300, 40
    rng = np.random.default_rng(5)
    a = torch.from_numpy(np.asfortranarray(rng.standard_normal((m, n)))).to(dev)
    if precision == "plain_f64":
        omega = torch.from_numpy(rng.standard_normal((ell, m))).to(dev)
        ydt = torch.float64
        tol = 1e-12
    else:
        _, bits = wl.gaussian_omega(ell, m, 6, "bf16")
        omega = torch.from_numpy(bits.view(np.int16)).to(dev).view(torch.bfloat16)
        ydt = torch.float32
        tol = 2.0 * (64 + 50 + 16) * 2.0 ** -24        # the FP32-accumulation bound of the sketch tests
    ref = gid.id_sketch(a, omega, precision)
    scale = float(ref.abs().max())
    for _ in range(2):
        code, y, info = _noalloc(lib, a, omega, precision, ydt)
        torch.cuda.synchronize()
        assert code == ID_OK
        assert int(info.item()) == 0
        assert float((y - ref).abs().max()) <= tol * scale


def test_noalloc_rejects_problems_beyond_its_scratch(lib):
    dev = torch.device("cuda:0")
    m, n, ell = 256, 100000, 128              # split-K partials far beyond the static scratch
    a = torch.zeros((n, m), dtype=torch.float32, device=dev).t()
    omega = torch.zeros((ell, m), dtype=torch.bfloat16, device=dev)
    code, _, _ = _noalloc(lib, a, omega, "mixed_bf16", torch.float32)
    assert code == ID_ERR_WORKSPACE


def test_noalloc_limit_is_the_workspace_size_less_its_slack(lib):
    """The static array holds exactly ID_NOALLOC_SCRATCH_BYTES of split-K partial sums: a
    64-row FP32 matrix with ell = 16 has one row slab, so n columns need 64 n bytes.
    n = 2^18 fills the array to the byte and runs (and matches id_sketch); one more column
    is refused.  id_sketch_workspace_size reports the same figure plus 512 bytes of slack."""
    import paper_2012_00706_gb300 as gid
    dev = torch.device("cuda:0")
    m, ell, limit = 64, 16, 16 * 1024 * 1024
    n = limit // (ell * 4)
    nb = ctypes.c_size_t(0)
    assert lib.id_sketch_workspace_size(1, m, n, ell, gid.PRECISIONS["mixed_bf16"], ctypes.byref(nb)) == ID_OK
    assert nb.value - 512 == limit
    rng = np.random.default_rng(8)
    big = torch.from_numpy(rng.standard_normal((n + 1, m)).astype(np.float32)).to(dev)
    _, bits = wl.gaussian_omega(ell, m, 9, "bf16")
    omega = torch.from_numpy(bits.view(np.int16)).to(dev).view(torch.bfloat16)
    a = big[:n].t()
    code, y, info = _noalloc(lib, a, omega, "mixed_bf16", torch.float32)
    torch.cuda.synchronize()
    assert code == ID_OK and int(info.item()) == 0
    ref = gid.id_sketch(a, omega, "mixed_bf16")
    assert float((y - ref).abs().max()) <= 2.0 * (64 + 1 + 16) * 2.0 ** -24 * float(ref.abs().max())
    code, _, _ = _noalloc(lib, big.t(), omega, "mixed_bf16", torch.float32)
    assert code == ID_ERR_WORKSPACE
