"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (written here, derived from the arithmetic):
  * scaled cast: bit-exact (shifts are integers, pieces are format codes decided
    in FP32 on both sides);
  * mixed sketch: |Y_gpu - Y_oracle| <= 2 (c + 2 log2(kslab count)) u32 (|Omega| |A~|)
    entrywise, c = 64 terms per chunk + chunks per slab (FP32 accumulation of exact
    products; factor 2 allows truncating rather than rounding accumulation);
  * plain FP64 sketch: 1e-12 relative to |Omega| |A|;
  * plain FP64 ID: pivots bit-exact on separated inputs, T within 1e-9 relative,
    relative reconstruction error within 1e-10 of the oracle's;
  * mixed ID: e_M <= 1.1 e_D + 10 u_low (the matched-accuracy criterion), e the
    relative 2-norm error of the reconstruction.
"""
import numpy as np
import pytest
import torch

import workloads as wl

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
U_LOW = {"mixed_bf16": 2.0 ** -8, "mixed_f16": 2.0 ** -11, "mixed_bf16x2": 2.0 ** -16,
         "mixed_bf16x3": 2.0 ** -24}
FMT = {"mixed_bf16": ("bf16", 1), "mixed_f16": ("f16", 1), "mixed_bf16x2": ("bf16", 2),
       "mixed_bf16x3": ("bf16", 3)}


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


def omega_dev(bits, dev, fmt):
    t = torch.from_numpy(np.ascontiguousarray(bits).view(np.int16)).to(dev)
    return t.view(torch.bfloat16 if fmt == "bf16" else torch.float16)


def bits_as_f64(bits, fmt):
    if fmt == "f16":
        return bits.view(np.float16).astype(np.float64)
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


# ------------------------------------------------------------------ scaled cast

def edge_matrix(dtype):
    """200 x 37 test matrix for the scaled cast: ragged last block, zero column, wide
    dynamic range, ties, FP64 -> FP32 rounding edges and range extremes (FP64 only)."""
    rng = np.random.default_rng(1)
    m, n = 200, 37
    a = rng.standard_normal((m, n)) * 10.0 ** rng.uniform(-6, 6, (m, n))
    a[:, 3] = 0.0
    a[10:20, 5] = 1e-30
    a[:, 7] = 1.0 + 2.0 ** -9            # ties for bfloat16
    a[::3, 8] = -(1.0 + 3 * 2.0 ** -12)  # ties for half
    if dtype == np.float64:
        # FP64 -> FP32 rounding edges: exact ties (to even), just above/below ties,
        # a carry into the next binade, the smallest FP64 step, signed zeros
        edges = np.array([1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, 1.0 + 2.0 ** -24 + 2.0 ** -52,
                          1.0 + 2.0 ** -24 - 2.0 ** -52, 2.0 - 2.0 ** -53, 1.0 + 2.0 ** -52, -0.0, 0.0,
                          -(1.5 + 2.0 ** -25), 0.75 - 2.0 ** -54, 1.9999999403953552, 1.0000000596046448])
        a[: len(edges), 9] = edges
        a[len(edges):2 * len(edges), 10] = -edges * 2.0 ** 40
        # scaled values below the FP32 normal range (exact fallback), subnormal doubles
        # in a block of ordinary values (signed zeros), a block near the bottom of the
        # FP64 range (shift below -872: the whole block takes the exact route, and its
        # subnormal double scales to a nonzero float), values near the FP64 maximum
        a[:64, 11] = 1.0
        a[1:9, 11] = [2.0 ** -140, -2.0 ** -130, 1.5 * 2.0 ** -126, 2.0 ** -149, 3.0 * 2.0 ** -151,
                      5e-324, -5e-324, 2.0 ** -1022]
        a[64:128, 12] = rng.standard_normal(64) * 1e-300
        a[70, 12] = 1e-310
        a[71, 12] = -0.0
        a[128:192, 13] = rng.standard_normal(64) * 1e300
        a[130:134, 13] = [1.0, -1e-20, 1e270, 2.0 ** -1074]
        # the FP32 normal-range boundary of the scaled values (block maximum 1, shift 1),
        # on rows 16q .. 16q + 3 and on the other rows of each 16
        a[:64, 14] = 1.0
        for r0 in (0, 5, 16, 21, 32, 37, 48, 53):
            a[r0 + 1: r0 + 4, 14] = [2.0 ** -125, -(2.0 ** -125) * (1 + 2.0 ** -30), 2.0 ** -126 * 1.25]
        a[64:128, 15] = 2.0 ** -100       # a block near the bottom of the FP32 range (shift -99)
        a[65:128:7, 15] = 2.0 ** -150 * 3.0
        a[66:128:5, 15] = 2.0 ** -170
    return np.asfortranarray(a.astype(dtype))


@pytest.mark.parametrize("precision", ["mixed_bf16", "mixed_f16", "mixed_bf16x2", "mixed_bf16x3"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_scale_cast_bit_exact(gid, dev, orc, precision, dtype):
    """Shifts and piece bits equal the oracle's cast (ragged last block, zero column,
    wide dynamic range, ties, range edges)."""
    a = edge_matrix(dtype)
    fmt, nsplit = FMT[precision]
    pieces, shifts, info = gid.id_scale_cast(torch.from_numpy(a).to(dev), precision)
    ref_p, ref_s, rc = orc.quantize(a, fmt, 64, nsplit)
    assert int(info.item()) == 0 and rc == 0
    assert np.array_equal(shifts.cpu().numpy(), ref_s)
    got = pieces.cpu().numpy().view(np.uint16)
    for p in range(nsplit):
        vals = bits_as_f64(np.ascontiguousarray(got[p]), fmt)
        assert np.array_equal(vals, ref_p[p]), f"piece {p} differs"


@pytest.mark.parametrize("precision", ["mixed_bf16", "mixed_f16", "mixed_bf16x2", "mixed_bf16x3"])
def test_sketch_identity_reproduces_cast(gid, dev, orc, precision):
    """The sketch kernel's own converter (the one inside the tensor-core pipeline, with
    its FP64-pipe and integer paths) against the oracle's cast, bit for bit: with Omega
    the identity every entry of Y is one product 1 x (sum of the pieces) x 2^s, exact in
    FP32.  Entries whose value is not a normal FP32 number (FP32 subnormals, whose
    handling is the tensor core's) are left out, and so is the column with values near the
    FP64 maximum: its scaled blocks reach past the FP32 range, so its FP32 sketch is not
    finite, which info reports."""
    a = edge_matrix(np.float64)
    m, n = a.shape
    fmt, nsplit = FMT[precision]
    ident = np.eye(m, dtype=np.float32)
    bits = wl.to_bf16_bits(ident) if fmt == "bf16" else wl.to_f16_bits(ident)
    y, info = gid.id_sketch(torch.from_numpy(a).to(dev), omega_dev(bits, dev, fmt), precision, return_info=True)
    y = y.cpu().numpy()
    assert int(info.item()) == -1
    ref_p, ref_s, rc = orc.quantize(a, fmt, 64, nsplit)
    assert rc == 0
    scale = np.repeat(2.0 ** ref_s, 64, axis=0)[:m]
    exact = ref_p.sum(axis=0) * scale
    with np.errstate(over="ignore"):
        ref32 = exact.astype(np.float32)
    mag = np.abs(exact)
    overflow_col = (mag >= 2.0 ** 127).any(axis=0)
    assert overflow_col.tolist() == [j == 13 for j in range(n)]
    normal = ((mag == 0) | ((mag >= 2.0 ** -126) & (mag < 2.0 ** 127))) & ~overflow_col[None, :]
    assert normal.sum() > 0.9 * normal.size
    # equal as numbers (a zero's sign is the sum's: -0 + 0 products is +0)
    bad = np.nonzero(y[normal] != ref32[normal])[0]
    assert bad.size == 0, (int(bad.size), np.argwhere(normal)[bad[:5]].tolist())


def test_widen_f32_to_f64_matches_hardware(gid, dev):
    """The integer FP32 -> FP64 widening the FP32 pivoted-QR kernels store R with equals the
    hardware conversion on all 2^32 bit patterns (zeros, subnormals, infinities, NaNs)."""
    assert gid.check_widen() == 0


def test_scale_cast_nonfinite(gid, dev):
    a = np.ones((70, 4))
    a[65, 2] = np.inf
    _, _, info = gid.id_scale_cast(torch.from_numpy(a).to(dev), "mixed_bf16")
    assert int(info.item()) == -1


# ----------------------------------------------------------------------- sketch

def lowp_bound(om, pieces, shifts, block=64, kslabs=16):
    """Entrywise bound of an FP32-accumulated evaluation: 2 (64 + nchunks + kslabs) u32 |Om| |A~| 2^s."""
    scale = np.repeat(2.0 ** shifts, block, axis=0)[: pieces.shape[1]]
    mag = np.abs(om) @ (np.abs(pieces).sum(axis=0) * scale)
    nch = (pieces.shape[1] + block - 1) // block
    return 2.0 * (64 + nch + kslabs) * U32 * mag


@pytest.mark.parametrize("precision", ["mixed_bf16", "mixed_f16", "mixed_bf16x3"])
@pytest.mark.parametrize("m,n,ell,dtype,pad", [
    (1000, 300, 40, np.float64, 0),      # ragged rows (1000 = 15*64 + 40), 3 column tiles
    (777, 129, 110, np.float64, 6),      # odd tail, lda = m + 6
    (640, 200, 200, np.float32, 0),      # N > 128
    (333, 70, 16, np.float32, 3),        # lda*4 not a multiple of 16 -> direct loads
    (129, 5, 8, np.float64, 1),          # odd lda -> direct loads
])
def test_sketch_lowp_vs_oracle(gid, dev, orc, precision, m, n, ell, dtype, pad):
    fmt, nsplit = FMT[precision]
    rng = np.random.default_rng(m + n + ell)
    a = rng.standard_normal((m, n)) * 10.0 ** rng.uniform(-2, 2, (1, n))
    a = a.astype(dtype)
    full = np.zeros((m + pad, n), dtype=dtype, order="F")
    full[:m] = a
    at = torch.from_numpy(full).to(dev)[:m]
    ldo = (m + 7) // 8 * 8
    om, bits = wl.gaussian_omega(ell, m, 3, fmt)
    bits_pad = np.zeros((ell, ldo), dtype=np.uint16)
    bits_pad[:, :m] = bits
    omt = omega_dev(bits_pad, dev, fmt)[:, :m]
    y, info = gid.id_sketch(at, omt, precision, return_info=True)
    assert int(info.item()) == 0
    y = y.cpu().numpy().astype(np.float64)
    ref, rc = orc.sketch_lowp(om, np.asfortranarray(a), fmt, nsplit, 64)
    pieces, shifts, _ = orc.quantize(np.asfortranarray(a), fmt, 64, nsplit)
    bound = lowp_bound(om, pieces, shifts)
    assert rc == 0
    err = np.abs(y - ref)
    assert np.all(err <= bound), float(np.max(err / np.maximum(bound, 1e-300)))


def test_sketch_f64_vs_oracle(gid, dev, orc):
    rng = np.random.default_rng(9)
    m, n, ell = 3001, 150, 70
    a = np.asfortranarray(rng.standard_normal((m, n)))
    om = rng.standard_normal((ell, m))
    y = gid.id_sketch(torch.from_numpy(a).to(dev), torch.from_numpy(om).to(dev), "plain_f64").cpu().numpy()
    ref = orc.sketch_f64(om, a)
    assert np.max(np.abs(y - ref) / (np.abs(om) @ np.abs(a))) <= 1e-12


# -------------------------------------------------------------- plain FP64 ID

@pytest.mark.parametrize("m,n,k", [(300, 140, 20), (1000, 500, 50), (97, 33, 33), (513, 260, 1), (64, 300, 40)])
def test_plain_f64_id_matches_oracle(gid, dev, orc, m, n, k):
    a = wl.separated_matrix(m, n, seed=m * 7 + n)
    ref = orc.interp_decomp(a, k=k)
    assert np.min(ref["gaps"]) >= 1e-8
    res = gid.id_factor(torch.from_numpy(a).to(dev), k, precision="plain_f64", estimate_error=True)
    assert res.info == 0 and res.k == k
    J = res.J.cpu().numpy()
    assert np.array_equal(J, ref["J"])
    T = res.T.cpu().numpy()
    assert T.shape == ref["T"].shape
    if T.size:
        assert np.max(np.abs(T - ref["T"])) <= 1e-9 * max(1.0, np.max(np.abs(ref["T"])))
    e_gpu = orc.rel_err(a, J, T, k, "fro")
    e_ref = orc.rel_err(a, ref["J"], ref["T"], k, "fro")
    assert abs(e_gpu - e_ref) <= 1e-10
    assert abs(res.err - e_ref) <= 1e-10


@pytest.mark.parametrize("m,n,k,dtype", [(30000, 300, 30, np.float64), (60000, 160, 24, np.float32)])
def test_plain_tall_streamed_matches_oracle(gid, dev, orc, m, n, k, dtype):
    """Tall matrices whose column slices do not fit the grid's shared memory take the
    streamed pivoted QR (the working copy updated in place in global memory): pivots equal
    the oracle's on separated inputs, T to the solve's accuracy."""
    a = wl.separated_matrix(m, n, seed=m + n, decay=0.9)
    ref = orc.interp_decomp(a, k=k)
    assert np.min(ref["gaps"]) >= 1e-3
    prec = "plain_f64" if dtype == np.float64 else "plain_f32"
    res = gid.id_factor(torch.from_numpy(a.astype(dtype)).to(dev), k, precision=prec)
    assert res.info == 0 and res.k == k
    J = res.J.cpu().numpy()
    assert np.array_equal(J, ref["J"])
    T = res.T.cpu().numpy()
    tol = 1e-9 if dtype == np.float64 else 1e-3
    assert np.max(np.abs(T - ref["T"])) <= tol * max(1.0, np.max(np.abs(ref["T"])))


@pytest.mark.parametrize("m,n,k,dtype", [(3000, 2600, 20, np.float64), (9000, 2500, 16, np.float64),
                                         (5000, 2500, 20, np.float32), (3001, 2600, 20, np.float32)])
def test_plain_wide_column_mode_matches_oracle(gid, dev, orc, m, n, k, dtype):
    """Wide matrices whose slices hold at least a column per warp take the streamed pivoted
    QR's column mode (a warp per column, no CTA barrier inside a step), with the pivot column
    staged in shared memory (3000 and 5000 rows) or read from L2 (9000 FP64 rows, 72 KB), by
    16-byte vectors where the columns are aligned and element by element where they are not
    (3001 FP32 rows): pivots equal the oracle's on separated inputs, T to the solve's accuracy."""
    a = wl.separated_matrix(m, n, seed=m + n, decay=0.97)
    a = a.astype(dtype).astype(np.float64)
    ref = orc.interp_decomp(a, k=k)
    assert np.min(ref["gaps"]) >= 1e-3
    prec = "plain_f64" if dtype == np.float64 else "plain_f32"
    res = gid.id_factor(torch.from_numpy(a.astype(dtype)).to(dev), k, precision=prec)
    assert res.info == 0 and res.k == k
    assert np.array_equal(res.J.cpu().numpy(), ref["J"])
    T = res.T.cpu().numpy()
    tol = 1e-9 if dtype == np.float64 else 1e-3
    assert np.max(np.abs(T - ref["T"])) <= tol * max(1.0, np.max(np.abs(ref["T"])))


def test_plain_f64_config1_full(gid, dev, orc):
    """Config 1 (1000 x 500, sigma_i = 10^(-i/25), k = 50): pivots equal the oracle's up
    to its first step whose two leading norms are within 1e-8 (none on this matrix),
    reconstruction error within 1e-10 of the oracle's in every case."""
    c = wl.config1()
    a = c["A"]
    ref = orc.interp_decomp(a, k=c["k"])
    res = gid.id_factor(torch.from_numpy(a).to(dev), c["k"], precision="plain_f64")
    assert res.info == 0 and res.k == 50
    J = res.J.cpu().numpy()
    gaps = ref["gaps"]
    first_tie = int(np.argmax(gaps < 1e-8)) if np.any(gaps < 1e-8) else 50
    assert np.array_equal(J[:first_tie], ref["J"][:first_tie])
    e_gpu = orc.rel_err(a, J, res.T.cpu().numpy(), 50)
    e_ref = orc.rel_err(a, ref["J"], ref["T"], 50)
    assert abs(e_gpu - e_ref) <= 1e-10 * max(1.0, e_ref)


def test_f32_solve_ill_conditioned_r11(gid, dev, orc):
    """FP32 pivoted QR (one cluster) of a matrix whose Householder QR is exact in FP32, so
    the GPU's R equals the oracle's; R11 has kappa near 1e7, where an FP32 solve refined
    once leaves T wrong in the leading digits.  The solve must detect it and give the
    oracle's T = R11^-1 R12 to FP64-solve accuracy."""
    k = 24
    w, perm = wl.exact_triangular_id_matrix(k=k, n=224, rows=40)
    w64 = w.astype(np.float64)
    kappa = np.linalg.cond(w64[:k, perm[:k]])
    assert 1e6 <= kappa <= 1e10, kappa
    ref = orc.interp_decomp(w64, k=k)
    assert np.array_equal(ref["J"][:k], perm[:k])
    res = gid.id_factor(torch.from_numpy(w).to(dev), k, precision="plain_f32")
    assert res.info == 0 and res.k == k
    assert np.array_equal(res.J.cpu().numpy(), ref["J"])
    T = res.T.cpu().numpy()
    assert np.max(np.abs(T - ref["T"])) <= 1e-6 * np.max(np.abs(ref["T"]))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_plain_f32_id(gid, dev, orc, dtype):
    a = wl.separated_matrix(400, 120, seed=31, decay=0.9)
    ref = orc.interp_decomp(a, k=25)
    res = gid.id_factor(torch.from_numpy(a.astype(dtype)).to(dev), 25, precision="plain_f32")
    assert res.info == 0
    assert np.array_equal(res.J.cpu().numpy()[:25], ref["J"][:25])
    e = orc.rel_err(a, res.J.cpu().numpy(), res.T.cpu().numpy(), 25)
    e_ref = orc.rel_err(a, ref["J"], ref["T"], 25)
    assert e <= 1.1 * e_ref + 10 * U32


def test_rank_by_tolerance(gid, dev, orc):
    m, n = 400, 120
    sigma = 10.0 ** (-np.arange(1, n + 1) / 6.0)
    a = wl.lowrank(m, n, sigma, 31)
    ref = orc.interp_decomp(a, tol=1e-5, k_max=80)
    res = gid.id_factor(torch.from_numpy(a).to(dev), tol=1e-5, k_max=80, precision="plain_f64")
    assert res.info == 0 and res.k == ref["k"]
    assert np.array_equal(res.J.cpu().numpy(), ref["J"])


def test_info_codes(gid, dev):
    a = np.zeros((50, 9))
    rng = np.random.default_rng(0)
    a[:, [2, 5]] = rng.standard_normal((50, 2))
    res = gid.id_factor(torch.from_numpy(a).to(dev), 4, precision="plain_f64")
    assert res.info == 3 and res.k == 2
    assert sorted(res.J.cpu().numpy()[:2].tolist()) == [2, 5]
    b = rng.standard_normal((50, 9))
    b[7, 3] = np.nan
    res = gid.id_factor(torch.from_numpy(b).to(dev), 4, precision="plain_f64")
    assert res.info == -1


# ----------------------------------------------------------------- mixed ID

@pytest.mark.parametrize("precision", ["mixed_bf16", "mixed_f16", "mixed_bf16x2", "mixed_bf16x3"])
def test_mixed_id_tolerance(gid, dev, orc, precision):
    """Config-2-shaped (smaller): e_M <= 1.1 e_D + 10 u_low with the same Omega."""
    fmt, _ = FMT[precision]
    m, n, k, ell = 4000, 400, 40, 50
    sigma = np.arange(1, n + 1, dtype=np.float64) ** -2.0
    a = wl.lowrank(m, n, sigma, 77)
    om, bits = wl.gaussian_omega(ell, m, 78, fmt)
    res = gid.id_factor(torch.from_numpy(a).to(dev), k, precision=precision, omega=omega_dev(bits, dev, fmt))
    assert res.info == 0 and res.k == k
    J, T = res.J.cpu().numpy(), res.T.cpu().numpy()
    ref = orc.interp_decomp(a, k=k, omega=om)
    e_m = orc.rel_err(a, J, T, k)
    e_d = orc.rel_err(a, ref["J"], ref["T"], k)
    assert e_m <= 1.1 * e_d + 10 * U_LOW[precision] * 1.0, (e_m, e_d)
    if precision == "mixed_bf16x3":
        # FP32-accurate sketch: same skeleton at separated steps
        ok = ref["gaps"] >= 1e-3
        first = int(np.argmax(~ok)) if np.any(~ok) else k
        assert np.array_equal(J[:first], ref["J"][:first])


def test_plain_f64_sketched_id(gid, dev, orc):
    m, n, k, ell = 3000, 250, 30, 40
    sigma = np.arange(1, n + 1, dtype=np.float64) ** -2.0
    a = wl.lowrank(m, n, sigma, 90)
    rng = np.random.default_rng(91)
    om = rng.standard_normal((ell, m))
    ref = orc.interp_decomp(a, k=k, omega=om)
    res = gid.id_factor(torch.from_numpy(a).to(dev), k, precision="plain_f64", omega=torch.from_numpy(om).to(dev))
    assert res.info == 0
    sep = ref["gaps"] >= 1e-8
    first = int(np.argmax(~sep)) if np.any(~sep) else k
    assert np.array_equal(res.J.cpu().numpy()[:first], ref["J"][:first])
    if first == k:
        assert np.max(np.abs(res.T.cpu().numpy() - ref["T"])) <= 1e-8 * max(1.0, np.max(np.abs(ref["T"])))


def test_plain_f64_rank_128(gid, dev, orc):
    """The largest rank of the warp-per-column solve (k = 128) in FP64: one FP64 copy
    of R11 fits shared memory."""
    m, n, k, ell = 1500, 400, 128, 138
    a = wl.separated_matrix(m, n, seed=128, decay=0.97)
    rng = np.random.default_rng(129)
    om = rng.standard_normal((ell, m))
    ref = orc.interp_decomp(a, k=k, omega=om)
    res = gid.id_factor(torch.from_numpy(a).to(dev), k, precision="plain_f64", omega=torch.from_numpy(om).to(dev))
    assert res.info == 0 and res.k == k
    sep = ref["gaps"] >= 1e-8
    first = int(np.argmax(~sep)) if np.any(~sep) else k
    assert np.array_equal(res.J.cpu().numpy()[:first], ref["J"][:first])
    if first == k:
        assert np.max(np.abs(res.T.cpu().numpy() - ref["T"])) <= 1e-8 * max(1.0, np.max(np.abs(ref["T"])))
    e = orc.rel_err(a, res.J.cpu().numpy(), res.T.cpu().numpy(), k)
    e_d = orc.rel_err(a, ref["J"], ref["T"], k)
    assert abs(e - e_d) <= 1e-10


# --------------------------------------------------- cluster pivoted QR (FP32, <= 128 rows)

@pytest.mark.parametrize("m,n,k", [(20, 300, 15), (50, 37, 30), (100, 700, 50), (110, 2000, 100), (128, 3000, 60)])
def test_cluster_cpqr_f32_short_matrix(gid, dev, orc, m, n, k):
    """PLAIN_F32 on a float matrix of <= 128 rows runs the thread-block-cluster kernel:
    pivots equal the oracle's while the oracle's gaps stay above FP32 resolution,
    and the ID error meets e <= 1.1 e_D + 10 u32."""
    a = wl.separated_matrix(m, n, seed=m + 3 * n, decay=0.97).astype(np.float32)
    ref = orc.interp_decomp(a.astype(np.float64), k=k)
    res = gid.id_factor(torch.from_numpy(np.asfortranarray(a)).to(dev), k, precision="plain_f32")
    assert res.info == 0 and res.k == k
    J = res.J.cpu().numpy()
    assert sorted(J.tolist()) == list(range(n))
    sep = ref["gaps"] >= 1e-3
    first = int(np.argmax(~sep)) if np.any(~sep) else k
    assert first > 0
    assert np.array_equal(J[:first], ref["J"][:first])
    e = orc.rel_err(a.astype(np.float64), J, res.T.cpu().numpy(), k)
    e_d = orc.rel_err(a.astype(np.float64), ref["J"], ref["T"], k)
    assert e <= 1.1 * e_d + 10 * U32


def test_cluster_cpqr_rank_by_tolerance(gid, dev, orc):
    m, n = 96, 800
    sigma = 10.0 ** (-np.arange(1, m + 1) / 8.0)
    a = wl.lowrank(m, n, sigma, 12).astype(np.float32)
    ref = orc.interp_decomp(a.astype(np.float64), tol=1e-3, k_max=90)
    res = gid.id_factor(torch.from_numpy(np.asfortranarray(a)).to(dev), tol=1e-3, k_max=90, precision="plain_f32")
    assert res.info == 0
    assert abs(res.k - ref["k"]) <= 1


def test_cluster_cpqr_zero_columns(gid, dev):
    a = np.zeros((40, 500), dtype=np.float32)
    rng = np.random.default_rng(2)
    cols = [3, 77, 200, 499]
    a[:, cols] = rng.standard_normal((40, 4))
    res = gid.id_factor(torch.from_numpy(np.asfortranarray(a)).to(dev), 6, precision="plain_f32")
    assert res.info == 5 and res.k == 4
    assert sorted(res.J.cpu().numpy()[:4].tolist()) == cols
