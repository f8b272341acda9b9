"""The C-ABI library builds, loads and exports every entry point its headers declare;
host-side argument checks answer without a GPU."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for mt in re.finditer(r"^[A-Za-z_][\w \*]*?\b(id_\w+)\s*\(", text, flags=re.M):
            names.add(mt.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import paper_2012_00706_gb300 as gid
    return gid.load()


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("id_factor", "id_workspace_size", "id_status_string", "id_sketch", "id_scale_cast"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    import paper_2012_00706_gb300 as gid
    for code in range(6):
        assert gid.status_string(code).startswith("ID_")
    assert lib.id_version().decode().startswith("gb300-id")


def _ws(lib, dtype, m, n, **kw):
    import paper_2012_00706_gb300 as gid
    o = gid.IDOpts()
    lib.id_opts_default(ctypes.byref(o))
    for key, v in kw.items():
        setattr(o, key, v)
    nb = ctypes.c_size_t(0)
    code = lib.id_workspace_size(dtype, m, n, ctypes.byref(o), ctypes.byref(nb))
    return code, nb.value


def test_workspace_size_and_argument_checks(lib):
    ok, nbytes = _ws(lib, 0, 1000, 500, k=50)
    assert ok == 0 and nbytes >= 1000 * 500 * 8
    assert _ws(lib, 0, 1000, 500, k=0)[0] == 1            # k < 1
    assert _ws(lib, 0, 1000, 500, k=501)[0] == 1          # k > min(m, n)
    assert _ws(lib, 0, 0, 5, k=1)[0] == 1                 # empty
    assert _ws(lib, 0, 1000, 500, k=50, precision=2)[0] == 1   # mixed without sketch
    assert _ws(lib, 0, 1000, 500, k=50, precision=9)[0] == 1   # unknown precision
    fake_omega = 0x1000
    ok, nb = _ws(lib, 0, 20000, 2000, k=100, sketch=1, ell=110, precision=2, omega=fake_omega)
    assert ok == 0 and nb > 110 * 2000 * 4
    assert _ws(lib, 0, 20000, 2000, k=100, sketch=1, ell=99, precision=2, omega=fake_omega)[0] == 1  # ell < k
    assert _ws(lib, 0, 20000, 2000, k=100, sketch=1, ell=300, precision=2, omega=fake_omega)[0] == 1  # ell > max
    assert _ws(lib, 0, 20000, 2000, k=100, sketch=1, ell=110, precision=2, omega=fake_omega + 8)[0] == 1
    assert _ws(lib, 0, 20000, 2000, k=100, sketch=1, ell=110, precision=2, omega=fake_omega,
               omega_ld=20004)[0] == 1   # TMA needs a row stride that is a multiple of 8
    assert _ws(lib, 0, 1000, 500, rel_tol=1e-6, k_max=50)[0] == 0
    assert _ws(lib, 0, 1000, 500, rel_tol=1e-6, k_max=0)[0] == 1
    # PLAIN_F32 pivots A itself: FP32 or FP64 storage (rounded to FP32 on load), no sketch
    assert _ws(lib, 1, 1000, 500, k=50, precision=1)[0] == 0
    assert _ws(lib, 0, 1000, 500, k=50, precision=1)[0] == 0
    assert _ws(lib, 1, 20000, 2000, k=100, sketch=1, ell=110, precision=1, omega=fake_omega)[0] == 1
    # Algorithm 2 on the whole matrix: no sketch
    assert _ws(lib, 0, 1000, 500, k=50, precision=6)[0] == 0
    assert _ws(lib, 1, 1000, 500, k=50, precision=7)[0] == 0
    assert _ws(lib, 0, 20000, 2000, k=100, sketch=1, ell=110, precision=7, omega=fake_omega)[0] == 1
    assert _ws(lib, 0, 1000, 500, k=50, precision=8)[0] == 1
    # the plain FP64 sketch takes FP64 data only
    assert _ws(lib, 1, 20000, 2000, k=100, sketch=1, ell=110, precision=0, omega=fake_omega)[0] == 1


def test_factor_rejects_null_outputs(lib):
    import paper_2012_00706_gb300 as gid
    o = gid.IDOpts()
    lib.id_opts_default(ctypes.byref(o))
    o.k = 3
    code = lib.id_factor(None, 0, 10, 5, 10, ctypes.byref(o), None, None, 3, None, None, None, None, 0, None)
    assert code == 1


def test_check_widen_rejects_null_output(lib):
    assert lib.id_check_widen(None, None) == 1
