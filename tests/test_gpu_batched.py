"""Batched IDs (id_factor_batched) against the FP64 oracle, through the C ABI.

Every matrix of an uneven batch is checked on its own against the oracle's
sketched ID with the same Omega (the leading ell_i x m_i block of the shared
one): the relative 2-norm error meets e_M <= 1.1 e_D + 10 u_low, and where the
oracle's pivot gaps are well above the sketch's resolution the pivots equal the
oracle's.  Also: ragged and degenerate shapes (k = n, m < 64, n not a multiple
of 128, padded leading dimensions, float input), rejection of matrices TMA
cannot address,
rank by tolerance, equality with one id_factor call per matrix, replay of a
captured CUDA graph on new data, and the autotuner's cache round trip.  The FP64
twin (precision plain_f64) equals the oracle's FP64 ID of every matrix and one
id_factor call per matrix, also when replayed from a captured graph.
"""
import json
import os

import numpy as np
import pytest
import torch

import workloads as wl

pytestmark = pytest.mark.gpu

U_LOW = {"mixed_bf16": 2.0 ** -8, "mixed_f16": 2.0 ** -11, "mixed_bf16x2": 2.0 ** -16,
         "mixed_bf16x3": 2.0 ** -24}
FMT = {"mixed_bf16": "bf16", "mixed_f16": "f16", "mixed_bf16x2": "bf16", "mixed_bf16x3": "bf16"}


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


def to_dev(a, dev, lda=None, dtype=np.float64):
    """Column-major device copy of a with leading dimension lda (>= m)."""
    m, n = a.shape
    lda = lda or m
    buf = torch.zeros((n, lda), dtype=torch.float64 if dtype == np.float64 else torch.float32, device=dev)
    buf[:, :m] = torch.from_numpy(np.ascontiguousarray(a.T.astype(dtype))).to(dev)
    return buf, buf.t()[:m]


def small_batch(count, seed, m_range=(100, 900), n_range=(30, 300), r_range=(4, 40)):
    """Uneven shapes in the style of the 512-matrix batch, scaled down for the oracle."""
    shapes = wl.config4_shapes(count, seed, m_range=m_range, n_range=n_range, r_range=r_range)
    mats = []
    for i, (m, n, r) in enumerate(shapes):
        mats.append(wl.separated_matrix(m, n, seed=seed * 1000 + i, decay=0.9))
    return shapes, mats


def aligned_ld(m, dtype=np.float64):
    """Smallest leading dimension >= m whose byte stride is a multiple of 16 (TMA)."""
    per = 2 if dtype == np.float64 else 4
    return (m + per - 1) // per * per


def run_batch(gid, dev, mats, ranks, precision, lda=None, dtype=np.float64, **kw):
    shapes = [a.shape for a in mats]
    ldas = lda or [aligned_ld(a.shape[0], dtype) for a in mats]
    plan = gid.BatchPlan(shapes, ranks, precision=precision, lda=ldas,
                         dtype=torch.float64 if dtype == np.float64 else torch.float32, **kw)
    fmt = FMT[precision]
    om, bits = wl.gaussian_omega(plan.ell_max, (plan.m_max + 7) // 8 * 8, 4242, fmt)
    omd = omega_dev(bits, dev, fmt)
    bufs = [to_dev(a, dev, l, dtype) for a, l in zip(mats, ldas)]
    plan.bind([v for _, v in bufs])
    plan.run(omd)
    torch.cuda.synchronize()
    return plan, om, bufs, omd


def check_against_oracle(orc, mats, ranks, plan, om, precision, oversample=10, strict_pivots=True, cast=None):
    for i, (a, r, res) in enumerate(zip(mats, ranks, plan.results())):
        m, n = a.shape
        ell = min(r + oversample, m)
        a64 = a.astype(np.float64) if cast is None else cast(a)
        ref = orc.interp_decomp(a64, k=r, omega=om[:ell, :m])
        assert res.info == 0 and res.k == r, (i, res.info, res.k)
        J = res.J.cpu().numpy()
        assert sorted(J.tolist()) == list(range(n)), i
        assert np.array_equal(J[r:], np.sort(J[r:]))
        T = res.T.cpu().numpy()
        assert T.shape == (r, n - r)
        e_m = orc.rel_err(a64, J, T, r)
        e_d = orc.rel_err(a64, ref["J"], ref["T"], r)
        assert e_m <= 1.1 * e_d + 10 * U_LOW[precision], (i, e_m, e_d)
        if strict_pivots:
            ok = ref["gaps"] >= 1e-2
            first = int(np.argmax(~ok)) if np.any(~ok) else r
            assert np.array_equal(J[:first], ref["J"][:first]), i


@pytest.mark.parametrize("precision", ["mixed_bf16", "mixed_f16", "mixed_bf16x3"])
def test_batched_uneven_vs_oracle(gid, dev, orc, precision):
    shapes, mats = small_batch(40, 11)
    ranks = [r for _, _, r in shapes]
    plan, om, *_ = run_batch(gid, dev, mats, ranks, precision)
    check_against_oracle(orc, mats, ranks, plan, om, precision, strict_pivots=precision == "mixed_bf16x3")


def test_batched_ragged_and_degenerate_shapes(gid, dev, orc):
    """k = n, m < 64, single column tile with 1 valid column, n just past a tile,
    padded leading dimensions, a tall matrix spanning many slabs."""
    rng = np.random.default_rng(5)
    dims = [(40, 12, 12), (63, 20, 5), (257, 129, 17), (300, 1, 1), (1000, 128, 30), (5000, 200, 25),
            (65, 64, 64), (777, 333, 128)]
    mats = [wl.separated_matrix(m, n, seed=int(rng.integers(1 << 30)), decay=0.9) for m, n, _ in dims]
    ranks = [r for _, _, r in dims]
    ldas = [aligned_ld(m) + (6 if i % 2 else 0) for i, (m, _, _) in enumerate(dims)]
    plan, om, *_ = run_batch(gid, dev, mats, ranks, "mixed_bf16x3", lda=ldas)
    check_against_oracle(orc, mats, ranks, plan, om, "mixed_bf16x3")


def test_batched_float_input(gid, dev, orc):
    shapes, mats = small_batch(16, 21)
    mats = [a.astype(np.float32) for a in mats]
    ranks = [r for _, _, r in shapes]
    plan, om, *_ = run_batch(gid, dev, mats, ranks, "mixed_f16", dtype=np.float32)
    check_against_oracle(orc, mats, ranks, plan, om, "mixed_f16", strict_pivots=False)


def test_batched_matches_single_calls(gid, dev):
    """Each matrix of the batch gives the same pivots as id_factor on that matrix with
    the same Omega block, and T agrees to FP32 accuracy."""
    shapes, mats = small_batch(12, 31)
    ranks = [r for _, _, r in shapes]
    plan, om, bufs, omd = run_batch(gid, dev, mats, ranks, "mixed_bf16x3")
    for i, (a, r, res) in enumerate(zip(mats, ranks, plan.results())):
        m, n = a.shape
        ell = min(r + 10, m)
        one = gid.id_factor(bufs[i][1], r, precision="mixed_bf16x3", omega=omd[:ell, :m])
        assert one.k == res.k == r
        assert np.array_equal(one.J.cpu().numpy(), res.J.cpu().numpy()), i
        t1, t2 = one.T.cpu().numpy(), res.T.cpu().numpy()
        # the two sketches add their split-K partial sums in different slabs, so T
        # differs by FP32 rounding of Y amplified by the conditioning of R11
        assert np.max(np.abs(t1 - t2)) <= 1e4 * 2.0 ** -24 * max(1.0, np.max(np.abs(t1))), i


def test_batched_rank_by_tolerance(gid, dev, orc):
    rng = np.random.default_rng(8)
    mats, caps = [], []
    for i in range(10):
        m, n = int(rng.integers(200, 700)), int(rng.integers(60, 250))
        sigma = 10.0 ** (-np.arange(1, n + 1) / 6.0)
        mats.append(wl.lowrank(m, n, sigma, 500 + i))
        caps.append(min(60, n))
    plan, om, *_ = run_batch(gid, dev, mats, caps, "mixed_bf16x3", tol=1e-4)
    for i, (a, cap, res) in enumerate(zip(mats, caps, plan.results())):
        m, n = a.shape
        ref = orc.interp_decomp(a, tol=1e-4, k_max=cap, omega=om[:min(cap + 10, m), :m])
        assert res.info == 0
        assert abs(res.k - ref["k"]) <= 1, (i, res.k, ref["k"])
        assert res.T.shape == (res.k, n - res.k)


def test_batched_graph_replay(gid, dev):
    """The launch sequence captured once replays on new matrices at the same addresses."""
    shapes, mats = small_batch(10, 41)
    ranks = [r for _, _, r in shapes]
    plan, om, bufs, omd = run_batch(gid, dev, mats, ranks, "mixed_bf16")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        plan.run(omd, stream=s)       # warm-up outside the capture
        s.synchronize()
        with torch.cuda.graph(g, stream=s):
            plan.run(omd, stream=s)
    torch.cuda.synchronize()
    new = [wl.separated_matrix(a.shape[0], a.shape[1], seed=900 + i, decay=0.9) for i, a in enumerate(mats)]
    for (buf, view), a in zip(bufs, new):
        view.copy_(torch.from_numpy(np.asfortranarray(a)).to(dev))
    g.replay()
    torch.cuda.synchronize()
    got = [(r.J.cpu().numpy().copy(), r.T.cpu().numpy().copy(), r.k) for r in plan.results()]
    plan.run(omd)
    torch.cuda.synchronize()
    for (J1, T1, k1), r in zip(got, plan.results()):
        assert k1 == r.k
        assert np.array_equal(J1, r.J.cpu().numpy())
        assert np.array_equal(T1, r.T.cpu().numpy())


def test_batched_autotune_cache_roundtrip(gid, dev, orc, tmp_path):
    shapes, mats = small_batch(24, 51)
    ranks = [r for _, _, r in shapes]
    plan, om, bufs, omd = run_batch(gid, dev, mats, ranks, "mixed_bf16x3")
    cache = str(tmp_path / "tune.jsonl")
    best = plan.autotune(omd, reps=2, cache_path=cache)
    assert best > 0
    lines = open(cache).read().strip().splitlines()
    assert len(lines) == 1
    entry = json.loads(lines[0])
    tuned = plan.describe()
    for key in ("slab_chunks", "tpc32", "tpc64", "solve_warps", "solve_cols"):
        assert entry[key] == tuned[key]
    # the tuned plan still gives the oracle's answers
    plan.run(omd)
    torch.cuda.synchronize()
    check_against_oracle(orc, mats, ranks, plan, om, "mixed_bf16x3")
    # a new plan for the same batch reads the cache
    again = gid.BatchPlan([a.shape for a in mats], ranks, precision="mixed_bf16x3", tune_cache=cache,
                          lda=[aligned_ld(a.shape[0]) for a in mats])
    d = again.describe()
    for key in ("slab_chunks", "tpc32", "tpc64", "solve_warps", "solve_cols"):
        assert d[key] == tuned[key]
    # tuning again replaces the entry instead of appending
    plan.autotune(omd, reps=1, cache_path=cache)
    assert len(open(cache).read().strip().splitlines()) == 1


def test_batched_argument_errors(gid, dev):
    plan = gid.BatchPlan([(100, 50), (200, 80)], [5, 7], precision="mixed_bf16")
    om, bits = wl.gaussian_omega(plan.ell_max, plan.m_max + 8, 1, "bf16")
    omd = omega_dev(bits, dev, "bf16")
    a = [torch.zeros((50, 100), dtype=torch.float64, device=dev).t(),
         torch.zeros((80, 200), dtype=torch.float64, device=dev).t()]
    # not bound yet
    with pytest.raises(gid.IDError):
        plan.run(omd)
    plan.bind(a)
    # Omega narrower than the widest matrix
    with pytest.raises(gid.IDError):
        plan.run(omd[:, :96].contiguous())
    # zero matrices: rank 0 at the first step, reported per matrix
    plan.run(omd)
    torch.cuda.synchronize()
    assert plan.info.cpu().tolist() == [1, 1]
    assert plan.k_out.cpu().tolist() == [0, 0]
    # a leading dimension TMA cannot address is refused at bind time
    odd = gid.BatchPlan([(101, 50)], [5], precision="mixed_bf16")
    buf = torch.zeros((50, 101), dtype=torch.float64, device=dev)
    with pytest.raises(gid.IDError):
        odd.bind([buf.t()])


def test_batched_plain_f64(gid, dev, orc):
    """The FP64 twin: each matrix's pivots equal the oracle's sketched FP64 ID with the
    same Omega block (separated columns: every gap well above FP64 rounding), T within
    1e-9, and J / T equal one id_factor(plain_f64) call bit for bit, also from a graph."""
    shapes, mats = small_batch(12, 61)
    ranks = [r for _, _, r in shapes]
    plan = gid.BatchPlan([a.shape for a in mats], ranks, precision="plain_f64")
    om, _ = wl.gaussian_omega(plan.ell_max, plan.m_max, 4343, "bf16")
    omd = torch.from_numpy(om).to(dev)
    bufs = [to_dev(a, dev) for a in mats]
    plan.bind([v for _, v in bufs])
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        plan.run(omd, stream=s)
        s.synchronize()
        with torch.cuda.graph(g, stream=s):
            plan.run(omd, stream=s)
    torch.cuda.synchronize()
    plan.J.zero_()
    plan.T.zero_()
    g.replay()
    torch.cuda.synchronize()
    for i, (a, r, res) in enumerate(zip(mats, ranks, plan.results())):
        m, n = a.shape
        ell = min(r + 10, m)
        ref = orc.interp_decomp(a, k=r, omega=om[:ell, :m])
        assert np.min(ref["gaps"]) >= 1e-8, i
        assert res.info == 0 and res.k == r, (i, res.info, res.k)
        J, T = res.J.cpu().numpy(), res.T.cpu().numpy()
        assert np.array_equal(J, ref["J"]), i
        assert np.max(np.abs(T - ref["T"])) <= 1e-9 * max(1.0, np.max(np.abs(ref["T"]))), i
        one = gid.id_factor(bufs[i][1], r, precision="plain_f64", omega=omd[:ell, :m])
        assert np.array_equal(one.J.cpu().numpy(), J), i
        assert np.array_equal(one.T.cpu().numpy(), T), i


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_batched_plain_f32(gid, dev, orc, dtype):
    """The unsketched FP32 plan (grouped pivoted QRs in waves, then the batched solve):
    uneven shapes over two waves (six 4000 x 1000 working copies of 16 MB do not fit one
    64 MB wave) plus ragged small ones.  Every matrix's pivots equal the oracle's
    unsketched ID of the same data (separated columns), its 2-norm error meets
    e <= 1.1 e_D + 10 u32, and J and T agree with one id_factor(plain_f32) call."""
    shapes = [(4000, 1000, 30)] * 6 + [(300, 77, 12), (1000, 33, 33), (2048, 512, 32)]
    mats = [wl.separated_matrix(m, n, seed=700 + i, decay=0.9).astype(dtype) for i, (m, n, _) in enumerate(shapes)]
    ranks = [r for _, _, r in shapes]
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    plan = gid.BatchPlan([a.shape for a in mats], ranks, dtype=tdt, precision="plain_f32")
    assert plan.describe()["waves"] >= 2
    bufs = [to_dev(a, dev, dtype=dtype) for a in mats]
    plan.bind([v for _, v in bufs])
    plan.run()
    torch.cuda.synchronize()
    for i, (a, r, res) in enumerate(zip(mats, ranks, plan.results())):
        a64 = a.astype(np.float32).astype(np.float64)      # the values the FP32 pivoting sees
        ref = orc.interp_decomp(a64, k=r)
        assert res.info == 0 and res.k == r, (i, res.info, res.k)
        J, T = res.J.cpu().numpy(), res.T.cpu().numpy()
        assert np.array_equal(J, ref["J"]), i
        scale = max(1.0, np.max(np.abs(ref["T"]), initial=0.0))
        assert np.max(np.abs(T - ref["T"]), initial=0.0) <= 1e-4 * scale, i
        e_m = orc.rel_err(a64, J, T, r)
        e_d = orc.rel_err(a64, ref["J"], ref["T"], r)
        assert e_m <= 1.1 * e_d + 10 * 2.0 ** -24, (i, e_m, e_d)
        one = gid.id_factor(bufs[i][1], r, precision="plain_f32")
        assert np.array_equal(one.J.cpu().numpy(), J), i
        assert np.max(np.abs(one.T.cpu().numpy() - T), initial=0.0) <= 1e-4 * scale, i


def test_batched_plain_f32_row_mode(gid, dev, orc):
    """A PLAIN_F32 wave whose slices are narrower than a CTA's warps runs the grouped kernel in
    row mode (each column one update behind, the pivot column brought up to date on the fly and
    kept in the group's two pivot-column slots): pivots equal the oracle's on separated columns,
    T agrees with the oracle's, tall ragged shapes included."""
    shapes = [(5000, 40, 8), (4099, 37, 12), (6001, 45, 20), (3000, 33, 33)]
    mats = [wl.separated_matrix(m, n, seed=760 + i, decay=0.9).astype(np.float32)
            for i, (m, n, _) in enumerate(shapes)]
    ranks = [r for _, _, r in shapes]
    plan = gid.BatchPlan([a.shape for a in mats], ranks, dtype=torch.float32, precision="plain_f32")
    d = plan.describe()
    assert d["column_mode"] == [0] and d["waves"] == 1, d
    bufs = [to_dev(a, dev, dtype=np.float32) for a in mats]
    plan.bind([v for _, v in bufs])
    plan.run()
    torch.cuda.synchronize()
    for i, (a, r, res) in enumerate(zip(mats, ranks, plan.results())):
        a64 = a.astype(np.float64)
        ref = orc.interp_decomp(a64, k=r)
        assert res.info == 0 and res.k == r, (i, res.info, res.k)
        J, T = res.J.cpu().numpy(), res.T.cpu().numpy()
        assert np.array_equal(J, ref["J"]), i
        scale = max(1.0, np.max(np.abs(ref["T"]), initial=0.0))
        assert np.max(np.abs(T - ref["T"]), initial=0.0) <= 1e-4 * scale, i


def test_batched_solve_ill_conditioned_r11(gid, dev, orc):
    """The batch's solve takes the products for well-conditioned R11 and the warp solve with
    six refinement steps where the largest diagonal of R11 exceeds 2^24 / 100 times the
    smallest: a PLAIN_F32 batch holding a matrix whose Householder QR is exact in FP32 (so
    the GPU's R equals the oracle's) with diagonal ratio 2^19 between two separated ones.
    Every T equals the oracle's; the ill-conditioned one to 1e-6 of its largest entry."""
    w, perm = wl.exact_triangular_id_matrix(k=20, n=150, rows=40)
    mats = [wl.separated_matrix(300, 80, seed=91, decay=0.9).astype(np.float32), w,
            wl.separated_matrix(500, 120, seed=92, decay=0.9).astype(np.float32)]
    ranks = [10, 20, 15]
    plan = gid.BatchPlan([a.shape for a in mats], ranks, dtype=torch.float32, precision="plain_f32")
    bufs = [to_dev(a, dev, dtype=np.float32) for a in mats]
    plan.bind([v for _, v in bufs])
    plan.run()
    torch.cuda.synchronize()
    for i, (a, r, res) in enumerate(zip(mats, ranks, plan.results())):
        a64 = a.astype(np.float64)
        ref = orc.interp_decomp(a64, k=r)
        assert res.info == 0 and res.k == r, (i, res.info, res.k)
        assert np.array_equal(res.J.cpu().numpy(), ref["J"]), i
        tol = 1e-6 if i == 1 else 1e-4
        T = res.T.cpu().numpy()
        assert np.max(np.abs(T - ref["T"])) <= tol * max(1.0, np.max(np.abs(ref["T"]))), (i, np.max(np.abs(T - ref["T"])))
    d = np.abs(np.diag(w.astype(np.float64)[:20, perm[:20]]))
    assert d.max() / d.min() > 2.0 ** 24 / 100
