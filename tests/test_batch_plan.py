"""Host-side logic of the batched ID plan (no GPU needed): argument checks, output
offsets, workspace sizing, and the unit tables the plan derives from the shapes."""
import ctypes

import pytest
import torch

import workloads as wl


@pytest.fixture(scope="module")
def gid():
    import paper_2012_00706_gb300 as g
    g.load()
    return g


def plan_status(gid, m, n, k, lda=None, dtype=0, **opts):
    lib = gid.load()
    b = len(m)
    o = lib.id_batch_opts_default()
    for key, v in opts.items():
        setattr(o, key, v)
    i64a = ctypes.c_int64 * b
    h = ctypes.c_void_p(0)
    code = lib.id_batch_plan_create(b, dtype, i64a(*m), i64a(*n), i64a(*(lda or m)), (ctypes.c_int32 * b)(*k),
                                    ctypes.byref(o), ctypes.byref(h))
    if h.value:
        lib.id_batch_plan_destroy(h)
    return code


def test_plan_offsets_fixed_rank(gid):
    shapes = [(300, 40), (1000, 700), (64, 64), (5000, 2048)]
    ranks = [10, 128, 64, 1]
    p = gid.BatchPlan(shapes, ranks, device="cpu")
    j = [0]
    t = [0]
    for (m, n), k in zip(shapes, ranks):
        j.append(j[-1] + n)
        t.append(t[-1] + k * (n - k))
    assert p.j_off == j
    assert p.t_off == t
    assert p.ell_max == 138          # 128 + 10
    assert p.m_max == 5000
    d = p.describe()
    assert d["work_bytes"] == p.work_bytes > 0
    # one unit per (128-column tile, 32-chunk row slab)
    assert d["sketch_units"] == sum(((n + 127) // 128) * (((m + 63) // 64 + 31) // 32) for m, n in shapes)


def test_plan_offsets_tolerance(gid):
    shapes = [(300, 40), (100, 90)]
    p = gid.BatchPlan(shapes, [20, 30], tol=1e-6, device="cpu")
    assert p.t_off == [0, 20 * 39, 20 * 39 + 30 * 89]


def test_plan_config4_shapes(gid):
    """The 512-matrix uneven batch plans; every unit table is sized and the outputs
    hold sum(n) pivots and sum(k (n - k)) coefficients."""
    shapes = wl.config4_shapes(512, 4)
    p = gid.BatchPlan([(m, n) for m, n, _ in shapes], [r for _, _, r in shapes], precision="mixed_bf16x3",
                      device="cpu")
    assert p.j_off[-1] == sum(n for _, n, _ in shapes)
    assert p.t_off[-1] == sum(r * (n - r) for _, n, r in shapes)
    d = p.describe()
    # each (tile, 32-chunk slab) is one unit
    assert d["sketch_units"] == sum(((n + 127) // 128) * (((m + 63) // 64 + 31) // 32) for m, n, _ in shapes)
    assert d["solve_units"] == sum((n - r + 31) // 32 for _, n, r in shapes)


@pytest.mark.parametrize("slab,units_of", [(16, 16), (64, 64)])
def test_plan_slab_option(gid, slab, units_of):
    shapes = [(4096, 1000), (300, 200)]
    p = gid.BatchPlan(shapes, [50, 8], slab_chunks=slab, device="cpu")
    d = p.describe()
    assert d["slab_chunks"] == slab
    assert d["sketch_units"] == sum(((n + 127) // 128) * (((m + 63) // 64 + units_of - 1) // units_of)
                                    for m, n in shapes)


def test_plan_argument_errors(gid):
    ok = plan_status(gid, [100], [50], [5])
    assert ok == 0
    assert plan_status(gid, [100], [50], [0]) == 1            # k < 1
    assert plan_status(gid, [100], [50], [51]) == 1           # k > n
    assert plan_status(gid, [30], [50], [31]) == 1            # k > m
    assert plan_status(gid, [100], [50], [5], lda=[99]) == 1  # lda < m
    assert plan_status(gid, [1000], [500], [129]) == 5        # k > 128
    assert plan_status(gid, [1000], [3000], [50]) == 5        # n > 2048
    assert plan_status(gid, [1000], [500], [128], oversample=40) == 5   # ell > 160
    assert plan_status(gid, [100], [50], [5], slab_chunks=7) == 1       # not a tuner candidate
    assert plan_status(gid, [100], [50], [5], cpqr_tpc=3) == 1


def test_plan_reads_tune_cache(gid, tmp_path):
    """A cache line with this batch's key sets the unit shapes; other keys are ignored."""
    shapes = [(500, 100), (800, 300)]
    ranks = [10, 20]
    base = gid.BatchPlan(shapes, ranks, device="cpu")
    cache = tmp_path / "c.jsonl"
    # no entry yet: defaults
    cache.write_text('{"key": "other|sm1|f64|p2|os10|tol0|b2|0", "slab_chunks": 64}\n')
    p = gid.BatchPlan(shapes, ranks, tune_cache=str(cache), device="cpu")
    assert p.describe()["slab_chunks"] == base.describe()["slab_chunks"]


def test_plan_plain_f64(gid):
    """The FP64 twin: any shape id_factor takes, the packed offsets of a mixed plan, and
    one workspace slice per matrix; FP32 input and rank by tolerance are refused."""
    shapes = [(300, 40), (1000, 700), (64, 64), (5000, 3000)]
    ranks = [10, 200, 64, 1]
    p = gid.BatchPlan(shapes, ranks, precision="plain_f64", device="cpu")
    assert p.j_off == [0, 40, 740, 804, 3804]
    assert p.t_off == [0, 300, 300 + 200 * 500, 100300, 100300 + 2999]
    assert p.ell_max == 210 and p.m_max == 5000
    d = p.describe()
    assert d["precision"] == "plain_f64" and d["ids"] == 4 and d["work_bytes"] == p.work_bytes
    lib = gid.load()
    total = 0
    for (m, n), k in zip(shapes, ranks):
        o = gid.IDOpts()
        lib.id_opts_default(ctypes.byref(o))
        o.k, o.sketch, o.ell, o.precision = k, 1, min(k + 10, m), 0
        o.omega, o.omega_ld = 256, m        # sizing reads neither; it only has to be set
        nb = ctypes.c_size_t(0)
        assert lib.id_workspace_size(0, m, n, ctypes.byref(o), ctypes.byref(nb)) == 0
        total = (total + nb.value + 255) // 256 * 256
    assert p.work_bytes == total
    assert plan_status(gid, [100], [50], [5], precision=0) == 0
    assert plan_status(gid, [1000], [3000], [129], precision=0) == 0     # beyond the mixed kernels' limits
    assert plan_status(gid, [100], [50], [5], precision=0, dtype=1) == 1  # FP32 input
    assert plan_status(gid, [100], [50], [5], precision=0, rel_tol=1e-6) == 1


def test_plan_plain_f32_waves(gid):
    """The unsketched FP32 plan: waves whose FP32 working copies fit 64 MiB, the SMs
    shared evenly within a wave, and the packed offsets of the other plans."""
    p = gid.BatchPlan([(2048, 512)] * 64, [32] * 64, dtype=torch.float32, precision="plain_f32", device="cpu")
    d = p.describe()
    assert d["precision"] == "plain_f32"
    assert d["ids_per_wave"] == [16, 16, 16, 16]          # 4 MiB each
    assert d["ctas_per_id"] == [9, 9, 9, 9]               # 152 SMs // 16
    assert p.j_off[-1] == 64 * 512 and p.t_off[-1] == 64 * 32 * 480
    q = gid.BatchPlan([(300, 3000), (5000, 40), (300, 7)], [128, 40, 7], precision="plain_f32", tol=1e-3,
                      device="cpu")
    d = q.describe()
    assert d["waves"] == 1 and d["ids_per_wave"] == [3] and d["ctas_per_id"] == [7]   # at most n of the narrowest
    # one slice mode per wave (a launch): a warp per column as soon as one matrix has a column
    # per warp (429 columns per CTA here), rows split over all threads only when none has
    assert d["column_mode"] == [1]
    assert p.describe()["column_mode"] == [1, 1, 1, 1]     # 57 columns per CTA
    r = gid.BatchPlan([(5000, 40)] * 4, [8] * 4, precision="plain_f32", device="cpu")
    assert r.describe()["ctas_per_id"] == [38] and r.describe()["column_mode"] == [0]   # 2 columns per CTA
    assert q.t_off == [0, 128 * 2999, 128 * 2999 + 40 * 39, 128 * 2999 + 40 * 39 + 7 * 6]
    assert plan_status(gid, [100], [50], [5], precision=1) == 0
    assert plan_status(gid, [100], [50], [5], precision=1, dtype=1) == 0
    assert plan_status(gid, [1000], [500], [129], precision=1) == 5      # the batched solve's rank limit
