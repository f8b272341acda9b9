"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test pins the oracle against mathematics, a library routine, brute force
or a value printed in the paper, chosen so that a dropped term, a wrong sign,
a wrong index or a transposed operand in the oracle fails at least one test.
"""
import itertools
import os

import numpy as np
import pytest

import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def golden():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, val, tol, *_ = line.split()
        out[name] = (float(val), float(tol))
    return out


def rand_lowrank(m, n, k, seed, decay=0.7):
    sigma = decay ** np.arange(k)
    return wl.lowrank(m, n, sigma, seed)


# ----------------------------------------------------------- paper values

def test_table1_unit_roundoff():
    """Table 1: u = 2^-11, 2^-24, 2^-53 for half/single/double."""
    g = golden()
    for name, u in [("table1_u_half", 2.0 ** -11), ("table1_u_single", 2.0 ** -24),
                    ("table1_u_double", 2.0 ** -53)]:
        val, tol = g[name]
        assert abs(u - val) <= tol * val


@pytest.mark.parametrize("kind", ["slow", "medium", "fast"])
def test_table2_dataset_spectrum(kind):
    """Table 2: sigma_50/sigma_1 and sigma_n/sigma_1 of the generated Slow/Medium/Fast matrices.

    The singular values are measured with LAPACK on the generated matrix, so this
    pins the generator, not just the profile formula.
    """
    g = golden()
    a = wl.paper_dataset(kind, seed=11)
    s = np.linalg.svd(a, compute_uv=False)
    v50, t50 = g[f"table2_{kind}_s50"]
    assert abs(s[49] / s[0] - v50) <= t50 * v50
    vn, tn = g[f"table2_{kind}_sn"]
    if kind != "fast":  # sigma_n/sigma_1 = 1e-12 is below LAPACK's resolution of ||A|| 1e-16 * cond
        assert abs(s[-1] / s[0] - vn) <= tn * vn
    else:
        assert abs(wl.paper_sigma("fast")[-1] / wl.paper_sigma("fast")[0] - vn) <= tn * vn


@pytest.mark.parametrize("kind", ["slow", "medium", "fast"])
def test_sec3_eckart_young_rank20(kind, orc):
    """Sec. 3.1: the optimal rank-20 2-norm error is sigma_21 (1/21, 1/441, ~5e-6).

    Checked through oracle.two_norm of A minus its truncated SVD.
    """
    g = golden()
    a = wl.paper_dataset(kind, seed=12)
    u, s, vt = np.linalg.svd(a)
    best20 = (u[:, :20] * s[:20]) @ vt[:20]
    err = orc.two_norm(a - best20) / orc.two_norm(a)
    val, tol = g[f"sec3_{kind}_opt20"]
    assert abs(err - val) <= tol * val


def test_sec3_lemma1_bound_fast_k51(orc):
    """Sec. 3.1 prints 3.3e-5 for the Lemma 1 bound at Fast, k=51, n=1000.

    sqrt(1 + 51*949) = 220 exactly; the printed number uses sigma_51 = 51^-4
    (the paper's index reading; sigma_52 would give 3.0e-5)."""
    g = golden()
    val, tol = g["sec3_fast_k51_bound"]
    sig = wl.paper_sigma("fast")
    b = orc.lemma1_bound(51, 1000, sig[50])
    assert abs(b - val) <= tol * val
    assert abs(orc.lemma1_bound(51, 1000, sig[51]) - val) > tol * val


# ------------------------------------------------------------- 2-norm

@pytest.mark.parametrize("m,n", [(4001, 1000), (1000, 4001), (2001, 2001)])
def test_two_norm_large_branch_matches_lapack(orc, m, n):
    """Just past the size where oracle.two_norm leaves LAPACK's SVD for the Gram
    matrix's largest eigenvalue: both branches agree with numpy's SVD-based 2-norm,
    for tall, wide and square inputs (a transposed Gram product or a wrong
    eigenvalue index would fail)."""
    rng = np.random.default_rng(m + 7 * n)
    x = rng.standard_normal((m, n)) * np.linspace(1.0, 3.0, n)[None, :]
    assert min(x.shape) > 2000 or x.size > 4_000_000
    ref = float(np.linalg.norm(x, 2))
    assert abs(orc.two_norm(x) - ref) <= 1e-12 * ref


def test_two_norm_known_singular_values(orc):
    """A = U diag(sigma) V^T with sigma_1 = 3, sigma_2 = 2.9999 (a close runner-up,
    which slows a power iteration): the 2-norm is sigma_1 in both branches."""
    sig = np.array([3.0, 2.9999] + [1.0 / i for i in range(3, 60)])
    for m, n in [(300, 200), (5000, 900)]:
        a = wl.lowrank(m, n, sig, 17)
        assert abs(orc.two_norm(a) - 3.0) <= 1e-12 * 3.0
        assert abs(orc.two_norm(np.asfortranarray(a.T)) - 3.0) <= 1e-12 * 3.0


# ------------------------------------------------------------ sketch, cast

def test_sketch_f64_matches_blas(orc):
    rng = np.random.default_rng(0)
    om = rng.standard_normal((13, 300))
    a = np.asfortranarray(rng.standard_normal((300, 17)))
    y = orc.sketch_f64(om, a)
    ref = om @ a
    assert np.max(np.abs(y - ref)) <= 1e-12 * np.max(np.abs(ref))
    # operand order matters: (Omega A) != (A^T Omega^T)^T only through layout; a transposed
    # read of Omega would change the values
    assert y.shape == (13, 17)


def test_round_half_matches_numpy(orc):
    """RNE to IEEE half agrees bit-for-bit with numpy's float16 cast, incl. ties,
    subnormals and overflow."""
    rng = np.random.default_rng(1)
    vals = list(rng.standard_normal(3000) * 10.0 ** rng.uniform(-9, 5, 3000))
    # exact ties: midpoints between neighbouring half values
    h = np.array([1.0, 1.5, 3.0, 2.0 ** -14, 2.0 ** -20, 1000.0], dtype=np.float16)
    nxt = np.nextafter(h, np.float16(np.inf))
    vals += list((h.astype(np.float64) + nxt.astype(np.float64)) / 2)
    vals += [65504.0, 65519.9, 65520.0, 1e6, -3e-8, 2.0 ** -25, 3 * 2.0 ** -26, 0.0, -0.0]
    for x in vals:
        got = orc.round_fmt(x, "f16")
        ref = float(np.float16(x))
        assert (got == ref) or (np.isinf(got) and np.isinf(ref) and np.sign(got) == np.sign(ref)), x


def test_round_bf16_matches_torch(orc):
    """RNE to bfloat16 agrees with torch's float32->bfloat16 cast on float32-exact inputs."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    x32 = (rng.standard_normal(4000) * 10.0 ** rng.uniform(-30, 30, 4000)).astype(np.float32)
    # ties: low 16 bits exactly 0x8000
    ties = (np.arange(1, 200, dtype=np.uint32) * 977 << 16 | 0x8000).view(np.float32)
    x32 = np.concatenate([x32, ties[np.isfinite(ties)]])
    ref = torch.from_numpy(x32).to(torch.bfloat16).float().numpy().astype(np.float64)
    got = np.array([orc.round_fmt(float(v), "bf16") for v in x32])
    assert np.array_equal(got, ref)


def test_round_bf16_from_double_is_single_rounding(orc):
    """FP64 -> bf16 rounds once: a double just above a bf16 midpoint must round up
    even where rounding through float32 first would land on the midpoint and tie
    to even (double rounding)."""
    base = 1.0 + 2.0 ** -7          # bf16 value with odd last bit ... 1.0078125
    mid = 1.0 + 2.0 ** -8           # midpoint between 1.0 and 1.0078125
    x = mid + 2.0 ** -40            # rounds to float32 as the midpoint exactly
    assert float(np.float32(x)) == mid
    assert orc.round_fmt(x, "bf16") == base
    assert orc.round_fmt(mid, "bf16") == 1.0   # tie to even


@pytest.mark.parametrize("fmt,lo,hi", [("bf16", 0.5, 1.0), ("f16", 2.0 ** 13, 2.0 ** 14)])
def test_block_shift_range(orc, fmt, lo, hi):
    rng = np.random.default_rng(3)
    for mx in np.abs(rng.standard_normal(500)) * 10.0 ** rng.uniform(-20, 20, 500):
        s = orc.block_shift(mx, fmt)
        assert lo <= mx * 2.0 ** -s < hi
    assert orc.block_shift(0.0, fmt) == 0


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_quantize_error_bounds(orc, fmt):
    """Pieces reconstruct x 2^-s within the format's unit round-off (1 piece) and to
    FP32 accuracy (3 pieces); shifts follow the block maxima."""
    rng = np.random.default_rng(4)
    a = np.asfortranarray(rng.standard_normal((70, 5)) * 10.0 ** rng.uniform(-3, 3, (70, 5)))
    u = 2.0 ** -8 if fmt == "bf16" else 2.0 ** -11
    for nsplit in (1, 2, 3):
        pieces, shifts, rc = orc.quantize(a, fmt, 32, nsplit)
        assert rc == 0
        assert shifts.shape == (3, 5)
        scale = np.repeat(2.0 ** shifts, 32, axis=0)[:70]
        back = pieces.sum(axis=0) * scale
        err = np.abs(back - a)
        # each piece adds a relative factor u; the FP32 step adds 2^-24; subnormal
        # half pieces add an absolute 2^-25 (half of the smallest subnormal)
        bound = (u ** nsplit + 2.0 ** -24) * np.abs(a) * 1.0001 + 2.0 ** -25 * scale * (fmt == "f16")
        assert np.all(err <= bound)
        for b in range(3):
            mx = np.max(np.abs(a[b * 32:(b + 1) * 32]), axis=0)
            for j in range(5):
                assert shifts[b, j] == orc.block_shift(mx[j], fmt)


def test_quantize_three_bf16_pieces_are_fp32_value(orc):
    """Reading of the cast: the scaled value is taken at FP32 first; three bfloat16
    pieces then sum to fl32(x 2^-s) exactly, for double and float storage."""
    rng = np.random.default_rng(14)
    a = rng.standard_normal((128, 6)) * 10.0 ** rng.uniform(-5, 5, (128, 6))
    for arr in (np.asfortranarray(a), np.asfortranarray(a.astype(np.float32))):
        pieces, shifts, rc = orc.quantize(arr, "bf16", 64, 3)
        scale = np.repeat(2.0 ** shifts, 64, axis=0)
        x32 = (arr.astype(np.float64) / scale).astype(np.float32).astype(np.float64)
        assert np.array_equal(pieces.sum(axis=0), x32)
        # piece 0 is a bfloat16 value: its low 16 float bits are zero
        p0 = pieces[0].astype(np.float32).view(np.uint32)
        assert np.all(p0 & 0xFFFF == 0)


def test_block_shift_zero_and_subnormal(orc):
    """Zero or input-subnormal block maxima get shift 0."""
    assert orc.block_shift(0.0, "bf16") == 0
    assert orc.block_shift(2.0 ** -1070, "bf16") == 0
    assert orc.block_shift(2.0 ** -130, "f16", in_f32=True) == 0
    assert orc.block_shift(2.0 ** -130, "bf16") == -129


def test_sketch_lowp_limits(orc):
    """3-piece bf16 sketch equals the FP64 sketch to ~1e-6 relative; 1 piece does not."""
    rng = np.random.default_rng(5)
    om, _ = wl.gaussian_omega(12, 256, 7, "bf16")
    a = np.asfortranarray(rng.standard_normal((256, 9)))
    ref = om @ a
    y3, rc = orc.sketch_lowp(om, a, "bf16", 3, 64)
    y1, _ = orc.sketch_lowp(om, a, "bf16", 1, 64)
    scale = np.abs(om) @ np.abs(a)
    assert rc == 0
    assert np.max(np.abs(y3 - ref) / scale) <= 2.0 ** -20
    assert np.max(np.abs(y1 - ref) / scale) > 2.0 ** -16
    assert np.max(np.abs(y1 - ref) / scale) <= 2.0 ** -8


def test_sketch_lowp_nonfinite_flag(orc):
    om, _ = wl.gaussian_omega(4, 40, 1, "bf16")
    a = np.ones((40, 3))
    a[5, 1] = np.nan
    _, rc = orc.sketch_lowp(om, a, "bf16", 1, 16)
    assert rc == -1


# -------------------------------------------------------------------- CPQR

@pytest.mark.parametrize("m,n,k", [(60, 40, 7), (33, 33, 11), (200, 50, 1)])
def test_exact_rank_reconstruction(orc, m, n, k):
    """Exact rank k => relative reconstruction error <= 1e-12 (2-norm and Frobenius)."""
    a = rand_lowrank(m, n, k, seed=m + n + k)
    out = orc.interp_decomp(a, k=k)
    assert out["k"] == k and out["info"] == 0
    assert orc.rel_err(a, out["J"], out["T"], k) <= 1e-12
    assert orc.rel_err(a, out["J"], out["T"], k, "fro") <= 1e-12
    assert sorted(out["J"].tolist()) == list(range(n))


def test_k1_closed_form(orc):
    """k=1: J[0] = argmax column norm; T = a_J^T A_Jc / ||a_J||^2."""
    a = wl.separated_matrix(40, 12, seed=9)
    out = orc.interp_decomp(a, k=1)
    p = int(np.argmax(np.sum(a * a, axis=0)))
    assert out["J"][0] == p
    jc = [i for i in range(12) if i != p]
    assert out["J"][1:].tolist() == jc
    t = a[:, p] @ a[:, jc] / (a[:, p] @ a[:, p])
    assert np.allclose(out["T"][0], t, rtol=1e-12, atol=1e-14)


def test_T_is_lstsq_at_oracle_pivots(orc):
    """T = R11^-1 R12 equals the least-squares solution lstsq(A_J, A_Jc) (LAPACK)."""
    a = wl.separated_matrix(80, 30, seed=10)
    k = 9
    out = orc.interp_decomp(a, k=k)
    J = out["J"]
    ref = np.linalg.lstsq(a[:, J[:k]], a[:, J[k:]], rcond=None)[0]
    assert np.max(np.abs(out["T"] - ref)) <= 1e-10 * max(1.0, np.max(np.abs(ref)))


def test_residual_equals_R22(orc):
    """||A - A(:,J)T||_F^2 = ||A||_F^2 - ||R(0:k,:)||_F^2 (= ||R22||_F^2, Q orthogonal)."""
    a = wl.separated_matrix(50, 35, seed=11)
    k = 12
    c = orc.cpqr(a, k=k)
    T = orc.solve_T(c["R"], c["J"], k)
    res = orc.residual_fro2(a, c["J"], T, k)
    r22 = np.sum(a * a) - np.sum(c["R"] ** 2)
    assert abs(res - r22) <= 1e-12 * np.sum(a * a)
    # R is upper triangular in the pivot order, with |R(j,j)| = residual norm of the pivot
    Rp = c["R"][:, c["J"]]
    assert np.allclose(np.tril(Rp[:, :k], -1), 0.0)


def test_pivots_and_diag_match_lapack(orc):
    """LAPACK dgeqp3 (scipy) picks the same first k pivots on separated columns and
    |diag R| agrees."""
    sla = pytest.importorskip("scipy.linalg")
    for seed in range(4):
        a = wl.separated_matrix(90, 40, seed=100 + seed)
        k = 15
        c = orc.cpqr(a, k=k)
        assert np.min(c["gaps"]) > 1e-6
        _, r, piv = sla.qr(a, pivoting=True, mode="economic")
        assert c["J"][:k].tolist() == piv[:k].tolist()
        d = np.abs(c["R"][np.arange(k), c["J"][:k]])
        assert np.allclose(d, np.abs(np.diag(r))[:k], rtol=1e-12)
        # the whole R row block agrees up to row signs
        rp = c["R"][:, piv]
        assert np.allclose(np.abs(rp), np.abs(r[:k]), rtol=1e-9, atol=1e-12 * np.abs(r).max())


def test_householder_exact_on_power_of_two_triangle(orc):
    """Greedy Householder CPQR of a triangular matrix with power-of-two diagonal and
    separated norms: pivots in triangular order, R = -W exactly (beta = -sign(alpha)
    ||x|| flips each row), and T = W11^-1 W12 to FP64 accuracy (numpy's solve)."""
    w, perm = wl.exact_triangular_id_matrix(k=12, n=60, rows=20)
    w64 = w.astype(np.float64)
    out = orc.cpqr(w64, k=12)
    assert np.array_equal(out["J"][:12], perm[:12])
    assert np.array_equal(out["R"], -w64[:12])
    T = orc.solve_T(out["R"], out["J"], 12)
    ref = np.linalg.solve(w64[:12, out["J"][:12]], w64[:12, out["J"][12:]])
    assert np.max(np.abs(T - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_low_cast_unit_blocks_is_the_library_cast(orc):
    """Blocks whose largest magnitude already sits in the format's target binade get shift 0,
    so A_L is the plain round-to-nearest cast: torch's bfloat16 and numpy's float16."""
    import torch
    rng = np.random.default_rng(3)
    a = rng.uniform(-0.999, 0.999, (200, 7)).astype(np.float32)
    a[0::64, :] = 0.999                                  # each 64-row block's maximum in [0.5, 1)
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(orc.low_cast(a, "bf16"), ref)
    h = (a * 2.0 ** 14 * 0.999).astype(np.float32)        # maxima in [2^13, 2^14)
    h[0::64, :] = 2.0 ** 14 * 0.999
    assert np.array_equal(orc.low_cast(h, "f16"), h.astype(np.float16).astype(np.float64))


def test_low_id_of_representable_data_is_the_plain_id(orc):
    """Integers of at most 8 significant bits are bfloat16 values at any power-of-two
    scale: A_L = A, and Algorithm 2's low ID equals Algorithm 1's ID."""
    rng = np.random.default_rng(4)
    a = np.asfortranarray(rng.integers(-120, 121, (90, 40)).astype(np.float64) * 2.0 ** rng.integers(-5, 6, (1, 40)))
    out = orc.low_id(a, "bf16", 10)
    assert np.array_equal(out["AL"], a)
    ref = orc.interp_decomp(a, k=10)
    assert np.array_equal(out["J"], ref["J"]) and np.array_equal(out["T"], ref["T"])


def test_adaptive_id_exact_rank_and_invariants(orc):
    """Exact rank r: the adaptive ID stops at the first block with ell - oversample >= r
    (ell = 48 for r = 23, blocks of 16), where its rank ell - oversample covers r and the
    reconstruction is exact (the later pivots pick up rounding only); on a decaying
    spectrum the stopped error is within the tolerance and one block fewer would not have
    met it."""
    rng = np.random.default_rng(6)
    r = 23
    a = rand_lowrank(900, 300, r, 6, decay=0.8)
    om = rng.standard_normal((200, 900))
    out = orc.adaptive_id(a, om, 1e-10, 16, 150)
    assert out["ell"] == 48 and out["k"] == 38 and out["err"] <= 1e-12
    short = orc.interp_decomp(a, k=22, omega=om[:32])
    assert np.sqrt(orc.residual_fro2(a, short["J"], short["T"], 22) / np.sum(a * a)) > 1e-3
    sig = 10.0 ** (-np.arange(1, 301) / 20.0)
    b = wl.lowrank(900, 300, sig, 7)
    out = orc.adaptive_id(b, om, 1e-4, 16, 150)
    assert out["err"] <= 1e-4 and out["k"] == out["ell"] - 10
    # the exact Frobenius tail of the spectrum bounds any rank-k approximation from below
    assert np.sqrt(np.sum(sig[out["k"]:] ** 2) / np.sum(sig ** 2)) <= 1e-4
    prev = orc.interp_decomp(b, k=out["k"] - 16, omega=om[: out["ell"] - 16])
    e_prev = np.sqrt(orc.residual_fro2(b, prev["J"], prev["T"], prev["k"]) / np.sum(b * b))
    assert e_prev > 1e-4


def test_row_id_of_symmetric_is_column_id(orc):
    """For a symmetric matrix the row ID is the column ID."""
    b = rand_lowrank(60, 60, 60, 8, decay=0.9)
    a = np.asfortranarray((b + b.T) / 2)
    r, c = orc.row_id(a, 12), orc.interp_decomp(a, k=12)
    assert np.array_equal(r["J"], c["J"]) and np.allclose(r["T"], c["T"], rtol=0, atol=1e-12)


def test_two_sided_error_is_the_column_error(orc):
    """The rank-k row ID of the rank-k skeleton A(:,J) is exact, so the two-sided ID's
    residual equals the column ID's (to rounding), and exact rank gives an exact result."""
    a = wl.lowrank(300, 200, 10.0 ** (-np.arange(1, 201) / 30.0), 9)
    col, row = orc.two_sided_id(a, 25)
    e2 = np.linalg.norm(a - orc.two_sided_reconstruct(a, col, row, 25))
    e1 = np.linalg.norm(a - orc.reconstruct(a, col["J"], col["T"], 25))
    assert abs(e2 - e1) <= 1e-10 * np.linalg.norm(a)
    x = rand_lowrank(200, 150, 12, 10, decay=0.8)
    col, row = orc.two_sided_id(x, 12)
    assert np.linalg.norm(x - orc.two_sided_reconstruct(x, col, row, 12)) <= 1e-12 * np.linalg.norm(x)


def test_mgs_crosscheck(orc):
    """The paper's MGS column selection gives the same pivots and |R| as Householder."""
    for seed in range(3):
        a = wl.separated_matrix(70, 30, seed=200 + seed)
        k = 10
        h = orc.cpqr(a, k=k)
        g = orc.mgs_cpqr(a, k)
        assert g["info"] == 0
        assert h["J"][:k].tolist() == g["J"].tolist()
        assert np.allclose(np.abs(h["R"]), np.abs(g["R"]), rtol=1e-9, atol=1e-12)


def test_downdate_matches_exact(orc):
    """Downdated norms with the recompute test give the exact-norm pivots; on columns
    built to cancel, the recompute path is exercised and still agrees."""
    for seed in range(3):
        a = wl.separated_matrix(100, 40, seed=300 + seed)
        e = orc.cpqr(a, k=20, norm_mode="exact")
        d = orc.cpqr(a, k=20, norm_mode="downdate")
        assert e["J"].tolist() == d["J"].tolist()
        assert np.allclose(e["R"], d["R"], rtol=1e-10, atol=1e-13)
    # nearly parallel columns: residual norms drop by ~1e-10 after one step
    rng = np.random.default_rng(7)
    base = rng.standard_normal((60, 1))
    a = np.asfortranarray(np.hstack([base * (1 + 1e-10 * j) + 1e-10 * rng.standard_normal((60, 1))
                                     for j in range(6)] + [rng.standard_normal((60, 4)) * 1e-9]))
    e = orc.cpqr(a, k=5, norm_mode="exact")
    d = orc.cpqr(a, k=5, norm_mode="downdate")
    assert e["J"].tolist() == d["J"].tolist()


def test_brute_force_tiny(orc):
    """n=8, k in {2,3}: CPQR error >= best subset error; the max-volume subset obeys
    Lemma 1 (||P||_2 and error bound); CPQR obeys the 2^k bound."""
    for seed in range(6):
        rng = np.random.default_rng(400 + seed)
        a = rng.standard_normal((10, 8)) @ np.diag(0.6 ** np.arange(8))
        s = np.linalg.svd(a, compute_uv=False)
        for k in (2, 3):
            out = orc.interp_decomp(a, k=k)
            e_cpqr = np.linalg.norm(a - orc.reconstruct(a, out["J"], out["T"], k), 2)
            best, best_s, vol_s, P = orc.brute_force(a, k)
            assert e_cpqr >= best * (1 - 1e-12)
            bound = orc.lemma1_bound(k, 8, s[k])
            assert np.linalg.norm(P, 2) <= np.sqrt(1 + k * (8 - k)) * (1 + 1e-12)
            assert np.linalg.norm(a - a[:, vol_s] @ P, 2) <= bound * (1 + 1e-12)
            assert e_cpqr <= orc.cpqr_bound(k, 8, s[k])
            # the best subset error is at least sigma_{k+1} (Eckart-Young)
            assert best >= s[k] * (1 - 1e-12)


def test_cpqr_bound_config1_shape(orc):
    """The pivoted-QR ID bound ||A - A(:,J)T||_2 <= sqrt(1+k(n-k)) 2^k sigma_{k+1} at a
    config-1-like decay (smaller size)."""
    m, n, k = 300, 150, 20
    sigma = 10.0 ** (-np.arange(1, n + 1) / 25.0)
    a = wl.lowrank(m, n, sigma, 21)
    out = orc.interp_decomp(a, k=k)
    err = orc.two_norm(a - orc.reconstruct(a, out["J"], out["T"], k))
    assert err <= orc.cpqr_bound(k, n, sigma[k])
    assert err >= sigma[k] * (1 - 1e-9)


def test_k_equals_n(orc):
    a = wl.separated_matrix(20, 6, seed=5)
    out = orc.interp_decomp(a, k=6)
    assert out["k"] == 6 and out["T"].shape == (6, 0)
    assert np.allclose(orc.reconstruct(a, out["J"], out["T"], 6), a, rtol=0, atol=0)


def test_rank_by_tolerance(orc):
    """Smallest k with ||R22||_F <= tol ||A||_F, checked with the explicit residual."""
    m, n = 120, 60
    sigma = 10.0 ** (-np.arange(1, n + 1) / 6.0)
    a = wl.lowrank(m, n, sigma, 31)
    tol = 1e-4
    out = orc.interp_decomp(a, tol=tol, k_max=60)
    k = out["k"]
    fa = np.linalg.norm(a)
    assert np.sqrt(orc.residual_fro2(a, out["J"], out["T"], k)) <= tol * fa * (1 + 1e-9)
    prev = orc.interp_decomp(a, k=k - 1)
    assert np.sqrt(orc.residual_fro2(a, prev["J"], prev["T"], k - 1)) > tol * fa
    # Frobenius tail of the singular values brackets the chosen rank
    assert np.sqrt(np.sum(sigma[k:] ** 2)) <= tol * fa * (1 + 1e-9)


def test_zero_pivot_and_nonfinite(orc):
    a = np.zeros((20, 7))
    rng = np.random.default_rng(3)
    a[:, [1, 4, 5]] = rng.standard_normal((20, 3))
    out = orc.interp_decomp(a, k=5)
    assert out["info"] == 4 and out["k"] == 3
    assert sorted(out["J"][:3].tolist()) == [1, 4, 5]
    b = a.copy()
    b[0, 0] = np.inf
    assert orc.interp_decomp(b, k=2)["info"] == -1


def test_sketched_id_equals_id_of_sketch(orc):
    """With Omega given, the oracle ID is the CPQR of Y = Omega A: same J as running
    the CPQR on the LAPACK product Omega @ A."""
    a = rand_lowrank(200, 60, 30, seed=41, decay=0.8)
    om, _ = wl.gaussian_omega(40, 200, 3)
    out = orc.interp_decomp(a, k=30, omega=om)
    c = orc.cpqr(om @ a, k=30)
    assert out["J"].tolist() == c["J"].tolist()
    # exact rank 30 with ell = 40 >= 30: the sketched ID is exact too
    assert orc.rel_err(a, out["J"], out["T"], 30) <= 1e-9


# ------------------------------------------------------------------ adjoint

def test_adjoint_against_finite_differences(orc):
    """Central differences (FP64, h=1e-6) of <G, A_hat> + <Tb, T> at fixed J."""
    rng = np.random.default_rng(8)
    m, n, k = 12, 7, 3
    a = rng.standard_normal((m, n))
    J = orc.interp_decomp(a, k=k)["J"]
    G = rng.standard_normal((m, n))
    Tb = rng.standard_normal((k, n - k))

    def loss(x):
        ah, t = orc.fixed_pivot_forward(x, J, k)
        return np.sum(G * ah) + np.sum(Tb * t)

    grad = orc.adjoint_ref(a, J, k, G, Tb)
    h = 1e-6
    fd = np.zeros_like(a)
    for i, j in itertools.product(range(m), range(n)):
        e = np.zeros_like(a)
        e[i, j] = h
        fd[i, j] = (loss(a + e) - loss(a - e)) / (2 * h)
    assert np.max(np.abs(fd - grad)) <= 1e-7 * max(1.0, np.max(np.abs(grad)))
    # each term matters: dropping the T_bar part changes the gradient
    g_no_t = orc.adjoint_ref(a, J, k, G, None)
    assert np.max(np.abs(g_no_t - grad)) > 1e-3
