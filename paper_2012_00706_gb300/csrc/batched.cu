// Batched mixed-precision column IDs: the plan (task and unit tables), the
// launch sequence, and the autotuner of the unit shapes.
//
// One call runs three stages over all matrices of the batch:
//   1. the tensor-core sketch, one CTA per (matrix, 128-column tile, row slab)
//      unit, the units ordered largest first so that the block scheduler hands
//      the longest ones out first (longest-processing-time order), each unit
//      leaving split-K partial sums; every matrix is read through its own TMA
//      tensor map, encoded when the matrices are bound;
//   2. the truncated pivoted QR, one thread-block cluster per matrix, which adds
//      the partial sums while loading; matrices are grouped by cluster size and
//      row class, and the groups run concurrently on the plan's streams;
//   3. the coefficient solve, one CTA per block of T columns.
// Everything the launches need is in the tables the plan writes into the
// caller's workspace once (id_batch_bind), so a call enqueues kernels only.
//
// Two plain twins share the call: PLAIN_F64 issues each matrix's FP64 ID as id_factor
// computes it, and PLAIN_F32 pivots the matrices themselves (no sketch) in waves, each
// wave one cooperative launch whose CTA groups factor one matrix each, followed by the
// batched solve of stage 3.
#include "common.cuh"
#include "cpqr_grid.cuh"
#include "internal.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <functional>
#include <queue>
#include <sstream>
#include <string>
#include <vector>

using namespace gid;

namespace {

constexpr int kSlabCandidates[] = {16, 32, 64};
constexpr int kMinSlabChunks = 16;
constexpr int kMaxAuxStreams = 32;
constexpr int kMaxClusterBatch = 16;    // CTAs of one matrix's pivoted QR (non-portable cluster size)
constexpr int kRowClasses[] = {32, 64, 96, 128, 160};
constexpr size_t kWaveBytes = size_t(64) << 20;   // PLAIN_F32 working copies of one wave (half of L2)
constexpr int kNumRowClasses = 5;

int row_class(int ell) {
    for (int i = 0; i < kNumRowClasses; ++i)
        if (ell <= kRowClasses[i]) return i;
    return -1;
}

bool is_mixed(int p) {
    return p == ID_MIXED_BF16 || p == ID_MIXED_F16 || p == ID_MIXED_BF16X2 || p == ID_MIXED_BF16X3;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Tuning {
    int slab_chunks = 32;
    int tpc[kNumRowClasses] = {4, 4, 4, 4, 4};   // per row class
    int solve_warps = 8;
    int solve_cols = 32;
};

struct CqGroup {
    ClusterCpqrPlan shape;
    int32_t first = 0, count = 0;
};

struct SolveClass {
    int kmax = 0;
    int32_t first = 0, count = 0;
};

// PLAIN_F32: matrices wave_order[first, first + count) in one grouped launch of gsize
// CTAs per matrix.
struct Wave {
    int32_t first = 0, count = 0, gsize = 1, colmode = 0;
    size_t smem = 0;
    size_t x_bytes = 0, ctrl_stride = 0;
};

}  // namespace

struct id_batch_plan {
    int32_t batch = 0;
    int a_f64 = 1;
    id_batch_opts_t opts{};
    std::vector<int64_t> m, n, lda;
    std::vector<int32_t> k;
    int device = 0;
    Tuning tune;
    // derived from shapes and tuning
    std::vector<BatchTask> tasks;
    std::vector<SketchUnit> sunits;
    std::vector<CUtensorMap> maps;   // one per matrix, encoded by id_batch_bind
    SketchPlan spipe;
    std::vector<int32_t> cq_order;
    std::vector<CqGroup> cq_groups;
    std::vector<SolveUnit> solve_units;
    std::vector<SolveClass> solve_classes;
    int ell_max = 0, lp_max = 0;
    int64_t m_max = 0;
    std::vector<int64_t> j_offsets, t_offsets;
    // workspace layout (bytes)
    size_t off_tasks = 0, off_maps = 0, off_sunits = 0, off_cq = 0, off_solve = 0, off_partial = 0, off_r = 0,
           off_sel = 0, off_inv = 0;
    int kcap_max = 0;      // the largest rank cap of the batch (the product solve's inverses)
    BatchTotals tot;
    size_t work_bytes = 0;
    size_t table_bytes = 0;
    std::vector<uint8_t> tables;    // host image of the table region
    void* bound_work = nullptr;
    // PLAIN_F64 plans: one FP64 id_factor per matrix in its own slice of the workspace
    bool plain = false;
    std::vector<size_t> woff, wbytes;
    std::vector<const void*> mats;
    // PLAIN_F32 plans: waves of grouped pivoted QRs, then the batched solve
    bool plain32 = false;
    std::vector<int32_t> wave_order;
    std::vector<Wave> waves;
    size_t off_params = 0, off_x = 0, off_ctrl = 0;
    // fork/join of the pivoted-QR groups
    cudaStream_t aux[kMaxAuxStreams] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kMaxAuxStreams] = {};
    bool streams_ready = false;
};

namespace {

// Sketch units: (matrix, tile, slab) with slab height S chunks, ordered by cost,
// largest first; CTA b computes unit b, and the block scheduler starts CTAs in
// index order as SMs free up, which deals the units out longest-processing-time.
void build_sketch_units(id_batch_plan* p) {
    const int S = p->tune.slab_chunks;
    struct U {
        SketchUnit su;
        double cost;
    };
    std::vector<U> all;
    for (int32_t i = 0; i < p->batch; ++i) {
        const BatchTask& t = p->tasks[i];
        const int64_t nch = (t.m + kChunkRows - 1) / kChunkRows;
        const int64_t tiles = (t.n + kTileCols - 1) / kTileCols;
        for (int64_t tile = 0; tile < tiles; ++tile)
            for (int32_t s = 0; s < t.kslabs; ++s) {
                SketchUnit su{};
                su.task = i;
                su.tile = static_cast<int32_t>(tile);
                su.c0 = s * S;
                su.nloc = static_cast<int32_t>(std::min<int64_t>(S, nch - su.c0));
                su.slab = s;
                // a chunk costs ~1; a unit adds its pipeline fill and the store of its sums
                all.push_back({su, su.nloc + 2.0 + t.lp / 64.0});
            }
    }
    std::stable_sort(all.begin(), all.end(), [](const U& a, const U& b) { return a.cost > b.cost; });
    p->sunits.clear();
    for (const U& u : all) p->sunits.push_back(u.su);
}

// Pivoted-QR groups: one launch per (row class, cluster size); matrices in a group
// ordered by rank, largest first.
bool build_cq_groups(id_batch_plan* p) {
    p->cq_order.clear();
    p->cq_groups.clear();
    std::vector<std::vector<int32_t>> buckets(kNumRowClasses * (kMaxClusterBatch + 1));
    for (int32_t i = 0; i < p->batch; ++i) {
        const BatchTask& t = p->tasks[i];
        const int rc = row_class(t.ell);
        if (rc < 0) return false;
        const int64_t cpb = 512 / p->tune.tpc[rc];
        const int64_t cs = (t.n + cpb - 1) / cpb;
        if (cs > kMaxClusterBatch) return false;
        buckets[rc * (kMaxClusterBatch + 1) + cs].push_back(i);
    }
    for (int rc = 0; rc < kNumRowClasses; ++rc)
        for (int cs = 1; cs <= kMaxClusterBatch; ++cs) {
            auto& v = buckets[rc * (kMaxClusterBatch + 1) + cs];
            if (v.empty()) continue;
            std::stable_sort(v.begin(), v.end(), [&](int32_t a, int32_t b) { return p->k[a] > p->k[b]; });
            CqGroup g;
            const int tpc = p->tune.tpc[rc];
            if (!cpqr_cluster_shape(kRowClasses[rc], cs, 512 / tpc, tpc, &g.shape)) return false;
            g.first = static_cast<int32_t>(p->cq_order.size());
            g.count = static_cast<int32_t>(v.size());
            p->cq_order.insert(p->cq_order.end(), v.begin(), v.end());
            p->cq_groups.push_back(g);
        }
    // largest groups (by total steps) first, so their streams start early
    std::stable_sort(p->cq_groups.begin(), p->cq_groups.end(), [&](const CqGroup& a, const CqGroup& b) {
        int64_t wa = 0, wb = 0;
        for (int32_t i = 0; i < a.count; ++i) wa += p->k[p->cq_order[a.first + i]] * a.shape.csize;
        for (int32_t i = 0; i < b.count; ++i) wb += p->k[p->cq_order[b.first + i]] * b.shape.csize;
        return wa > wb;
    });
    return true;
}

// Solve units: blocks of solve_cols columns of T, grouped by rank class (32, 64,
// 96, 128 rows per warp column); units of the heaviest matrices first.
void build_solve_units(id_batch_plan* p) {
    p->solve_units.clear();
    p->solve_classes.clear();
    const int C = p->tune.solve_cols;
    for (int kq = 1; kq <= 4; ++kq) {
        std::vector<int32_t> ids;
        int kmax = 0;
        for (int32_t i = 0; i < p->batch; ++i)
            if ((p->k[i] + 31) / 32 == kq) {
                ids.push_back(i);
                kmax = std::max(kmax, p->k[i]);
            }
        if (ids.empty()) continue;
        std::stable_sort(ids.begin(), ids.end(), [&](int32_t a, int32_t b) {
            return static_cast<double>(p->k[a]) * p->k[a] > static_cast<double>(p->k[b]) * p->k[b];
        });
        SolveClass sc;
        sc.kmax = kmax;
        sc.first = static_cast<int32_t>(p->solve_units.size());
        for (int32_t i : ids) {
            const int64_t cols = p->tasks[i].tcols;
            for (int64_t c = 0; c < cols; c += C) {
                SolveUnit u{};
                u.task = i;
                u.c0 = static_cast<int32_t>(c);
                u.ncols = static_cast<int32_t>(std::min<int64_t>(C, cols - c));
                p->solve_units.push_back(u);
            }
        }
        sc.count = static_cast<int32_t>(p->solve_units.size()) - sc.first;
        p->solve_classes.push_back(sc);
    }
}

// Tasks, offsets and the workspace layout for the current tuning.
bool build_plan(id_batch_plan* p) {
    const int nsplit = precision_nsplit(p->opts.precision);
    p->tasks.assign(p->batch, BatchTask{});
    p->j_offsets.assign(p->batch + 1, 0);
    p->t_offsets.assign(p->batch + 1, 0);
    int64_t partial = 0, rr = 0, sel = 0, inv = 0;
    p->kcap_max = 0;
    p->ell_max = 0;
    p->m_max = 0;
    for (int32_t i = 0; i < p->batch; ++i) {
        BatchTask& t = p->tasks[i];
        t.m = p->m[i];
        t.n = p->n[i];
        t.lda = p->lda[i];
        t.kcap = p->k[i];
        t.ell = static_cast<int32_t>(std::min<int64_t>(p->k[i] + p->opts.oversample, p->m[i]));
        t.lp = (t.ell + 15) / 16 * 16;
        const int64_t nch = (t.m + kChunkRows - 1) / kChunkRows;
        t.kslabs = static_cast<int32_t>((nch + p->tune.slab_chunks - 1) / p->tune.slab_chunks);
        t.partial_off = partial;
        // room for the smallest slab height the tuner tries, so any tuning fits the workspace
        const int64_t max_slabs = (nch + kMinSlabChunks - 1) / kMinSlabChunks;
        partial += max_slabs * t.n * t.lp;
        t.r_off = rr;
        rr += static_cast<int64_t>(t.kcap) * t.n;
        t.sel_off = sel;
        sel += (t.n + 15) / 16 * 16;
        t.inv_off = inv;
        inv += static_cast<int64_t>(batch_inverse_floats(t.kcap));
        p->kcap_max = std::max(p->kcap_max, t.kcap);
        t.j_off = p->j_offsets[i];
        p->j_offsets[i + 1] = p->j_offsets[i] + t.n;
        t.tcols = p->opts.rel_tol > 0.0 ? t.n - 1 : t.n - t.kcap;
        t.t_off = p->t_offsets[i];
        p->t_offsets[i + 1] = p->t_offsets[i] + static_cast<int64_t>(t.kcap) * t.tcols;
        t.rel_tol = p->opts.rel_tol;
        p->ell_max = std::max(p->ell_max, t.ell);
        p->m_max = std::max(p->m_max, t.m);
    }
    p->lp_max = (p->ell_max + 15) / 16 * 16;
    if (!sketch_pipeline_plan(p->lp_max, p->a_f64, nsplit, &p->spipe)) return false;
    build_sketch_units(p);
    if (!build_cq_groups(p)) return false;
    build_solve_units(p);

    // workspace: tables, then sketch partial sums, R, selection flags
    size_t off = 0;
    p->off_tasks = off;
    off = align256(off + p->tasks.size() * sizeof(BatchTask));
    p->off_maps = off;
    off = align256(off + p->tasks.size() * sizeof(CUtensorMap));
    p->off_sunits = off;
    // sized for the most units any slab candidate produces
    size_t max_units = 0;
    for (int S : kSlabCandidates) {
        size_t units = 0;
        for (const BatchTask& t : p->tasks) {
            const int64_t nch = (t.m + kChunkRows - 1) / kChunkRows;
            units += ((t.n + kTileCols - 1) / kTileCols) * ((nch + S - 1) / S);
        }
        max_units = std::max(max_units, units);
    }
    max_units = std::max(max_units, p->sunits.size());
    off = align256(off + max_units * sizeof(SketchUnit));
    p->off_cq = off;
    off = align256(off + p->cq_order.size() * sizeof(int32_t));
    p->off_solve = off;
    size_t max_solve = 0;
    for (const BatchTask& t : p->tasks) max_solve += (t.tcols + 15) / 16;   // smallest solve_cols tried
    max_solve = std::max(max_solve, p->solve_units.size());
    off = align256(off + max_solve * sizeof(SolveUnit));
    p->table_bytes = off;
    p->off_partial = off;
    off = align256(off + static_cast<size_t>(partial) * sizeof(float));
    p->off_r = off;
    off = align256(off + static_cast<size_t>(rr) * sizeof(double));
    p->off_sel = off;
    off = align256(off + static_cast<size_t>(sel));
    p->off_inv = off;
    off = align256(off + static_cast<size_t>(inv) * sizeof(float));
    p->work_bytes = off;
    p->tot.ntasks = p->batch;
    p->tot.partial = static_cast<int64_t>((p->off_r - p->off_partial) / sizeof(float));
    p->tot.r = static_cast<int64_t>((p->off_sel - p->off_r) / sizeof(double));
    p->tot.j = p->j_offsets.back();
    p->tot.t = p->t_offsets.back();
    p->tot.sel = static_cast<int64_t>(p->off_inv - p->off_sel);
    p->tot.inv = static_cast<int64_t>((p->work_bytes - p->off_inv) / sizeof(float));

    // host image of the table region
    p->tables.assign(p->table_bytes, 0);
    memcpy(p->tables.data() + p->off_tasks, p->tasks.data(), p->tasks.size() * sizeof(BatchTask));
    if (p->maps.size() == p->tasks.size())
        memcpy(p->tables.data() + p->off_maps, p->maps.data(), p->maps.size() * sizeof(CUtensorMap));
    memcpy(p->tables.data() + p->off_sunits, p->sunits.data(), p->sunits.size() * sizeof(SketchUnit));
    memcpy(p->tables.data() + p->off_cq, p->cq_order.data(), p->cq_order.size() * sizeof(int32_t));
    memcpy(p->tables.data() + p->off_solve, p->solve_units.data(), p->solve_units.size() * sizeof(SolveUnit));
    return true;
}

// PLAIN_F32: tasks and offsets as for a mixed plan (no sketch), the solve units, and the
// waves.  Matrices are taken in decreasing order of pivoting work (m n k); a wave holds as
// many as keep their FP32 working copies within kWaveBytes (and at most one per SM), and
// shares the SMs evenly between them (gsize CTAs each, at most n of the narrowest).
bool build_plan_plain32(id_batch_plan* p) {
    const int sms = device_info().sm_count;
    p->tasks.assign(p->batch, BatchTask{});
    p->j_offsets.assign(p->batch + 1, 0);
    p->t_offsets.assign(p->batch + 1, 0);
    int64_t rr = 0, sel = 0, inv = 0;
    p->kcap_max = 0;
    p->ell_max = 0;
    p->m_max = 0;
    for (int32_t i = 0; i < p->batch; ++i) {
        BatchTask& t = p->tasks[i];
        t.m = p->m[i];
        t.n = p->n[i];
        t.lda = p->lda[i];
        t.kcap = p->k[i];
        t.r_off = rr;
        rr += static_cast<int64_t>(t.kcap) * t.n;
        t.sel_off = sel;
        sel += (t.n + 15) / 16 * 16;
        t.inv_off = inv;
        inv += static_cast<int64_t>(batch_inverse_floats(t.kcap));
        p->kcap_max = std::max(p->kcap_max, t.kcap);
        t.j_off = p->j_offsets[i];
        p->j_offsets[i + 1] = p->j_offsets[i] + t.n;
        t.tcols = p->opts.rel_tol > 0.0 ? t.n - 1 : t.n - t.kcap;
        t.t_off = p->t_offsets[i];
        p->t_offsets[i + 1] = p->t_offsets[i] + static_cast<int64_t>(t.kcap) * t.tcols;
        t.rel_tol = p->opts.rel_tol;
        p->m_max = std::max(p->m_max, t.m);
    }
    build_solve_units(p);

    std::vector<int32_t> order(p->batch);
    for (int32_t i = 0; i < p->batch; ++i) order[i] = i;
    auto work = [&](int32_t i) { return static_cast<double>(p->m[i]) * p->n[i] * p->k[i]; };
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return work(a) > work(b); });
    p->wave_order = order;
    p->waves.clear();
    size_t x_max = 0, ctrl_max = 0, smem_max = 0;
    for (int32_t q = 0; q < p->batch;) {
        Wave w;
        w.first = q;
        size_t bytes = 0;
        int64_t nmin = INT64_MAX, mmax = 1;
        while (q < p->batch && w.count < sms) {
            const int32_t i = order[q];
            const size_t b = align256(static_cast<size_t>(p->m[i]) * p->n[i] * sizeof(float));
            if (w.count > 0 && bytes + b > kWaveBytes) break;
            bytes += b;
            nmin = std::min(nmin, p->n[i]);
            mmax = std::max(mmax, p->m[i]);
            ++w.count;
            ++q;
        }
        w.gsize = static_cast<int32_t>(std::max<int64_t>(1, std::min<int64_t>(sms / w.count, nmin)));
        int64_t cpb = 1, rst = 0;
        for (int32_t e = w.first; e < w.first + w.count; ++e) {
            const int64_t ci = (p->n[order[e]] + w.gsize - 1) / w.gsize;
            cpb = std::max<int64_t>(cpb, ci);
            rst = std::max<int64_t>(rst, cpqr_grouped_rstage(ci, p->m[order[e]], 4));
        }
        // one mode per wave (a launch): a warp per column when any matrix has a column per
        // warp (the others leave warps idle), else the rows split over all threads
        w.colmode = cpqr_grouped_colmode(cpb);
        w.smem = cpqr_grouped_smem(cpb, rst, 0);
        if (w.smem > static_cast<size_t>(device_info().max_smem_optin) - 8 * 1024) return false;
        w.x_bytes = bytes;
        // barrier word and candidate tables, then the row mode's two pivot-column slots
        w.ctrl_stride = cpqr_pub_offset(w.gsize) + align256(2 * static_cast<size_t>(mmax) * sizeof(float));
        x_max = std::max(x_max, bytes);
        ctrl_max = std::max(ctrl_max, w.ctrl_stride * w.count);
        smem_max = std::max(smem_max, w.smem);
        p->waves.push_back(w);
    }

    // workspace: tables (tasks, solve units, parameter blocks), then the wave's working
    // copies and control words, R, selection flags
    size_t off = 0;
    p->off_tasks = off;
    off = align256(off + p->tasks.size() * sizeof(BatchTask));
    p->off_solve = off;
    off = align256(off + p->solve_units.size() * sizeof(SolveUnit));
    p->off_params = off;
    off = align256(off + static_cast<size_t>(p->batch) * sizeof(CpqrParams<float>));
    p->table_bytes = off;
    p->off_x = off;
    off = align256(off + x_max);
    p->off_ctrl = off;
    off = align256(off + ctrl_max);
    p->off_r = off;
    off = align256(off + static_cast<size_t>(rr) * sizeof(double));
    p->off_sel = off;
    off = align256(off + static_cast<size_t>(sel));
    p->off_inv = off;
    off = align256(off + static_cast<size_t>(inv) * sizeof(float));
    p->work_bytes = off;
    p->tot.ntasks = p->batch;
    p->tot.partial = 0;
    p->tot.r = static_cast<int64_t>((p->off_sel - p->off_r) / sizeof(double));
    p->tot.j = p->j_offsets.back();
    p->tot.t = p->t_offsets.back();
    p->tot.sel = static_cast<int64_t>(p->off_inv - p->off_sel);
    p->tot.inv = static_cast<int64_t>((p->work_bytes - p->off_inv) / sizeof(float));
    p->tables.assign(p->table_bytes, 0);
    memcpy(p->tables.data() + p->off_tasks, p->tasks.data(), p->tasks.size() * sizeof(BatchTask));
    memcpy(p->tables.data() + p->off_solve, p->solve_units.data(), p->solve_units.size() * sizeof(SolveUnit));
    return true;
}

// PLAIN_F32: one parameter block per matrix, in wave order, for the bound matrices and
// workspace (the outputs are the call's, added by the kernel from their bases).
void write_params_plain32(id_batch_plan* p, const void* const* A, void* work) {
    uint8_t* w = static_cast<uint8_t*>(work);
    const int64_t ms = p->opts.watchdog_ms > 0 ? p->opts.watchdog_ms : 4000;
    CpqrParams<float>* params = reinterpret_cast<CpqrParams<float>*>(p->tables.data() + p->off_params);
    for (const Wave& wv : p->waves) {
        size_t xoff = 0;
        for (int32_t e = 0; e < wv.count; ++e) {
            const int32_t i = p->wave_order[wv.first + e];
            const BatchTask& t = p->tasks[i];
            CpqrParams<float> P{};
            P.X = reinterpret_cast<float*>(w + p->off_x + xoff);
            xoff += align256(static_cast<size_t>(t.m) * t.n * sizeof(float));
            P.r = t.m;
            P.n = t.n;
            P.ldx = t.m;
            P.src = A[i];
            P.src_f64 = p->a_f64;
            P.ldsrc = t.lda;
            P.kcap = t.kcap;
            P.rel_tol = p->opts.rel_tol;
            P.R = reinterpret_cast<double*>(w + p->off_r) + t.r_off;
            P.ldr = t.kcap;
            P.sel = w + p->off_sel + t.sel_off;
            P.ctrl = reinterpret_cast<CpqrCtrl*>(w + p->off_ctrl + e * wv.ctrl_stride);
            P.cand = reinterpret_cast<Cand*>(w + p->off_ctrl + e * wv.ctrl_stride + sizeof(CpqrCtrl));
            P.pub = reinterpret_cast<float*>(w + p->off_ctrl + e * wv.ctrl_stride + cpqr_pub_offset(wv.gsize));
            P.resident = 0;
            P.cpb_max = (t.n + wv.gsize - 1) / wv.gsize;
            P.colmode = wv.colmode;
            P.rstage = cpqr_grouped_rstage(P.cpb_max, t.m, 4);
            P.limit_ns = static_cast<uint64_t>(ms) * 1000000ull;
            P.out_j = t.j_off;
            P.out_i = i;
            params[wv.first + e] = P;
        }
    }
}

uint64_t fnv1a(uint64_t h, const void* data, size_t len) {
    const uint8_t* b = static_cast<const uint8_t*>(data);
    for (size_t i = 0; i < len; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

std::string device_name(int dev) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return "unknown";
    }
    std::string s(prop.name);
    for (char& c : s)
        if (c == '"' || c == '\\') c = '_';
    return s;
}

// Cache key: device, SM count, input type, precision, options and every shape.
std::string tune_key(const id_batch_plan* p) {
    uint64_t h = 1469598103934665603ull;
    h = fnv1a(h, p->m.data(), p->m.size() * sizeof(int64_t));
    h = fnv1a(h, p->n.data(), p->n.size() * sizeof(int64_t));
    h = fnv1a(h, p->lda.data(), p->lda.size() * sizeof(int64_t));
    h = fnv1a(h, p->k.data(), p->k.size() * sizeof(int32_t));
    char buf[256];
    snprintf(buf, sizeof(buf), "%s|sm%d|%s|p%d|os%d|tol%d|b%d|%016llx", device_name(p->device).c_str(),
             device_info().sm_count, p->a_f64 ? "f64" : "f32", p->opts.precision, p->opts.oversample,
             p->opts.rel_tol > 0.0 ? 1 : 0, p->batch, static_cast<unsigned long long>(h));
    return std::string(buf);
}

bool json_int(const std::string& line, const char* name, int* out) {
    const std::string pat = std::string("\"") + name + "\":";
    size_t pos = line.find(pat);
    if (pos == std::string::npos) return false;
    pos += pat.size();
    while (pos < line.size() && line[pos] == ' ') ++pos;
    char* end = nullptr;
    const long v = strtol(line.c_str() + pos, &end, 10);
    if (end == line.c_str() + pos) return false;
    *out = static_cast<int>(v);
    return true;
}

bool json_key_is(const std::string& line, const std::string& key) {
    return line.find(std::string("\"key\": \"") + key + "\"") != std::string::npos;
}

std::string tuning_json(const id_batch_plan* p, double ms) {
    char buf[512];
    snprintf(buf, sizeof(buf),
             "\"slab_chunks\": %d, \"tpc32\": %d, \"tpc64\": %d, \"tpc96\": %d, \"tpc128\": %d, "
             "\"tpc160\": %d, \"solve_warps\": %d, \"solve_cols\": %d, \"ms\": %.4f",
             p->tune.slab_chunks, p->tune.tpc[0], p->tune.tpc[1], p->tune.tpc[2], p->tune.tpc[3], p->tune.tpc[4],
             p->tune.solve_warps, p->tune.solve_cols, ms);
    return std::string(buf);
}

bool valid_tuning(const Tuning& t) {
    bool slab_ok = false;
    for (int S : kSlabCandidates) slab_ok |= (t.slab_chunks == S);
    if (!slab_ok) return false;
    for (int rc = 0; rc < kNumRowClasses; ++rc)
        if (t.tpc[rc] != 2 && t.tpc[rc] != 4) return false;
    if (t.tpc[kNumRowClasses - 1] != 4) return false;   // 160 rows: 2 threads per column would spill
    return t.solve_warps >= 1 && t.solve_warps <= 16 && t.solve_cols >= 16 && t.solve_cols <= 4096;
}

void read_cache(id_batch_plan* p, const char* path) {
    std::ifstream f(path);
    if (!f) return;
    const std::string key = tune_key(p);
    std::string line;
    while (std::getline(f, line)) {
        if (!json_key_is(line, key)) continue;
        Tuning t = p->tune;
        json_int(line, "slab_chunks", &t.slab_chunks);
        json_int(line, "tpc32", &t.tpc[0]);
        json_int(line, "tpc64", &t.tpc[1]);
        json_int(line, "tpc96", &t.tpc[2]);
        json_int(line, "tpc128", &t.tpc[3]);
        json_int(line, "tpc160", &t.tpc[4]);
        json_int(line, "solve_warps", &t.solve_warps);
        json_int(line, "solve_cols", &t.solve_cols);
        if (valid_tuning(t)) p->tune = t;
    }
}

bool write_cache(const id_batch_plan* p, const char* path, double ms) {
    const std::string key = tune_key(p);
    std::vector<std::string> keep;
    {
        std::ifstream f(path);
        std::string line;
        while (f && std::getline(f, line))
            if (!line.empty() && !json_key_is(line, key)) keep.push_back(line);
    }
    std::ofstream f(path, std::ios::trunc);
    if (!f) return false;
    for (const auto& l : keep) f << l << "\n";
    f << "{\"key\": \"" << key << "\", " << tuning_json(p, ms) << "}\n";
    return static_cast<bool>(f);
}

bool ensure_streams(id_batch_plan* p) {
    if (p->streams_ready) return true;
    if (cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming) != cudaSuccess) return false;
    for (int i = 0; i < kMaxAuxStreams; ++i) {
        if (cudaStreamCreateWithFlags(&p->aux[i], cudaStreamNonBlocking) != cudaSuccess) return false;
        if (cudaEventCreateWithFlags(&p->join[i], cudaEventDisableTiming) != cudaSuccess) return false;
    }
    p->streams_ready = true;
    return true;
}

id_status_t enqueue(const id_batch_plan* p, const void* omega, int64_t omega_ld, int32_t* J, double* T,
                    int32_t* k_out, int32_t* info, void* work, cudaStream_t s) {
    uint8_t* w = static_cast<uint8_t*>(work);
    const BatchTask* d_tasks = reinterpret_cast<const BatchTask*>(w + p->off_tasks);
    const CUtensorMap* d_maps = reinterpret_cast<const CUtensorMap*>(w + p->off_maps);
    const SketchUnit* d_units = reinterpret_cast<const SketchUnit*>(w + p->off_sunits);
    const int32_t* d_order = reinterpret_cast<const int32_t*>(w + p->off_cq);
    const SolveUnit* d_solve = reinterpret_cast<const SolveUnit*>(w + p->off_solve);
    float* partial = reinterpret_cast<float*>(w + p->off_partial);
    double* R = reinterpret_cast<double*>(w + p->off_r);
    uint8_t* sel = w + p->off_sel;
    const int64_t ms = p->opts.watchdog_ms > 0 ? p->opts.watchdog_ms : 4000;
    const uint64_t lim = static_cast<uint64_t>(ms) * 1000000ull;

    record_stage(0, s);
    if (cudaMemsetAsync(info, 0, sizeof(int32_t) * p->batch, s) != cudaSuccess) return ID_ERR_CUDA;
    cudaError_t e = launch_sketch_lowp_batched(d_units, static_cast<int64_t>(p->sunits.size()), d_tasks, d_maps,
                                               p->a_f64, static_cast<const uint16_t*>(omega), omega_ld, p->m_max,
                                               p->ell_max, p->opts.precision, p->spipe, partial, p->tot.partial,
                                               p->batch, info, lim, s);
    if (e != cudaSuccess) return ID_ERR_CUDA;
    record_stage(1, s);
    record_stage(2, s);
    // pivoted QR: groups fork onto the plan's streams and join back
    const int ng = static_cast<int>(p->cq_groups.size());
    const int naux = std::min(ng, kMaxAuxStreams);
    if (naux > 1) {
        if (cudaEventRecord(p->fork, s) != cudaSuccess) return ID_ERR_CUDA;
        for (int i = 0; i < naux; ++i)
            if (cudaStreamWaitEvent(p->aux[i], p->fork, 0) != cudaSuccess) return ID_ERR_CUDA;
    }
    for (int g = 0; g < ng; ++g) {
        const CqGroup& G = p->cq_groups[g];
        cudaStream_t gs = naux > 1 ? p->aux[g % naux] : s;
        e = launch_cpqr_cluster_batched(d_tasks, d_order + G.first, G.count, partial, R, sel, J, k_out, info,
                                        p->tot, G.shape, lim, gs);
        if (e != cudaSuccess) return ID_ERR_CUDA;
    }
    if (naux > 1) {
        for (int i = 0; i < naux; ++i) {
            if (cudaEventRecord(p->join[i], p->aux[i]) != cudaSuccess) return ID_ERR_CUDA;
            if (cudaStreamWaitEvent(s, p->join[i], 0) != cudaSuccess) return ID_ERR_CUDA;
        }
    }
    record_stage(3, s);
    // one refinement step: the solve as products, every R11 inverted first
    float* inv = reinterpret_cast<float*>(w + p->off_inv);
    const bool product = p->opts.refine_steps == 1;
    if (product && launch_r11_inverse_batched(d_tasks, p->batch, p->kcap_max, R, J, k_out, p->tot, inv, s) != cudaSuccess)
        return ID_ERR_CUDA;
    record_stage(4, s);     // the inverses (nothing on the warp solve's path)
    // solve classes (by rank) run concurrently on the plan's streams as well
    const int nsc = static_cast<int>(p->solve_classes.size());
    const int naux2 = std::min(nsc, kMaxAuxStreams);
    if (naux2 > 1) {
        if (cudaEventRecord(p->fork, s) != cudaSuccess) return ID_ERR_CUDA;
        for (int i = 0; i < naux2; ++i)
            if (cudaStreamWaitEvent(p->aux[i], p->fork, 0) != cudaSuccess) return ID_ERR_CUDA;
    }
    for (int ci = 0; ci < nsc; ++ci) {
        const SolveClass& c = p->solve_classes[ci];
        cudaStream_t cs = naux2 > 1 ? p->aux[ci % naux2] : s;
        e = product ? launch_solve_T_batched_product(d_tasks, d_solve + c.first, c.count, c.kmax, R, J, k_out, info, T,
                                                     p->tot, p->opts.refine_steps, inv, cs)
                    : launch_solve_T_batched(d_tasks, d_solve + c.first, c.count, c.kmax, p->tune.solve_warps, R, J,
                                             k_out, info, T, p->tot, p->opts.refine_steps, cs);
        if (e != cudaSuccess) return ID_ERR_CUDA;
    }
    if (naux2 > 1) {
        for (int i = 0; i < naux2; ++i) {
            if (cudaEventRecord(p->join[i], p->aux[i]) != cudaSuccess) return ID_ERR_CUDA;
            if (cudaStreamWaitEvent(s, p->join[i], 0) != cudaSuccess) return ID_ERR_CUDA;
        }
    }
    record_stage(5, s);
    return ID_OK;
}

// The options of matrix i's FP64 ID in a PLAIN_F64 plan.
id_opts_t plain_opts(const id_batch_plan* p, int32_t i, const void* omega, int64_t omega_ld) {
    id_opts_t o;
    id_opts_default(&o);
    o.k = p->k[i];
    o.sketch = 1;
    o.ell = static_cast<int32_t>(std::min<int64_t>(p->k[i] + p->opts.oversample, p->m[i]));
    o.precision = ID_PLAIN_F64;
    o.omega = omega;
    o.omega_ld = omega_ld;
    o.refine_steps = p->opts.refine_steps;
    o.watchdog_ms = p->opts.watchdog_ms;
    return o;
}

// PLAIN_F64: the matrices' FP64 IDs (FP64 sketch by DFMA, FP64 pivoted QR and solve) in
// order on the caller's stream, each in its own workspace slice.  One stream because the
// FP64 pivoted QR is a cooperative grid launch, and two of those running side by side on
// other streams are not guaranteed to be co-resident.
id_status_t enqueue_plain(const id_batch_plan* p, const void* omega, int64_t omega_ld, int32_t* J, double* T,
                          int32_t* k_out, int32_t* info, void* work, cudaStream_t s) {
    uint8_t* w = static_cast<uint8_t*>(work);
    record_stage(0, s);
    const int stages = pause_stages();
    id_status_t st = ID_OK;
    for (int32_t i = 0; i < p->batch && st == ID_OK; ++i) {
        const id_opts_t o = plain_opts(p, i, omega, omega_ld);
        st = id_factor(p->mats[i], ID_F64, p->m[i], p->n[i], p->lda[i], &o, J + p->j_offsets[i], T + p->t_offsets[i],
                       p->k[i], k_out + i, info + i, nullptr, w + p->woff[i], p->wbytes[i], s);
    }
    resume_stages(stages);
    if (st != ID_OK) return st;
    for (int i = 1; i < 6; ++i) record_stage(i, s);
    return ID_OK;
}

// PLAIN_F32: per wave, zero the groups' control words and launch the grouped pivoted QR;
// then the solve classes as in stage 3 of the mixed call.
id_status_t enqueue_plain32(const id_batch_plan* p, int32_t* J, double* T, int32_t* k_out, int32_t* info, void* work,
                            cudaStream_t s) {
    uint8_t* w = static_cast<uint8_t*>(work);
    const BatchTask* d_tasks = reinterpret_cast<const BatchTask*>(w + p->off_tasks);
    const SolveUnit* d_solve = reinterpret_cast<const SolveUnit*>(w + p->off_solve);
    const CpqrParams<float>* d_params = reinterpret_cast<const CpqrParams<float>*>(w + p->off_params);
    const double* R = reinterpret_cast<const double*>(w + p->off_r);
    record_stage(0, s);
    if (cudaMemsetAsync(info, 0, sizeof(int32_t) * p->batch, s) != cudaSuccess) return ID_ERR_CUDA;
    record_stage(1, s);
    record_stage(2, s);
    for (const Wave& wv : p->waves) {
        if (cudaMemsetAsync(w + p->off_ctrl, 0, wv.ctrl_stride * wv.count, s) != cudaSuccess) return ID_ERR_CUDA;
        if (launch_cpqr_grouped<float>(d_params + wv.first, wv.count, wv.gsize, wv.colmode, wv.smem, J, k_out, info,
                                       s) !=
            cudaSuccess)
            return ID_ERR_CUDA;
    }
    record_stage(3, s);
    float* inv = reinterpret_cast<float*>(w + p->off_inv);
    const bool product = p->opts.refine_steps == 1;
    if (product && launch_r11_inverse_batched(d_tasks, p->batch, p->kcap_max, R, J, k_out, p->tot, inv, s) != cudaSuccess)
        return ID_ERR_CUDA;
    record_stage(4, s);     // the inverses (nothing on the warp solve's path)
    for (const SolveClass& c : p->solve_classes) {
        const cudaError_t e =
            product ? launch_solve_T_batched_product(d_tasks, d_solve + c.first, c.count, c.kmax, R, J, k_out, info, T,
                                                     p->tot, p->opts.refine_steps, inv, s)
                    : launch_solve_T_batched(d_tasks, d_solve + c.first, c.count, c.kmax, p->tune.solve_warps, R, J,
                                             k_out, info, T, p->tot, p->opts.refine_steps, s);
        if (e != cudaSuccess) return ID_ERR_CUDA;
    }
    record_stage(5, s);
    return ID_OK;
}

id_status_t check_call(const id_batch_plan* p, const void* omega, int64_t omega_ld, const int32_t* J,
                       const double* T, const int32_t* k_out, const int32_t* info, const void* work,
                       size_t work_bytes) {
    if (!p || !J || !T || !k_out || !info || !work) return ID_ERR_ARG;
    if (!omega && !p->plain32) return ID_ERR_ARG;
    if (work_bytes < p->work_bytes) return ID_ERR_WORKSPACE;
    if (p->plain32) {
        if (work != p->bound_work || p->mats.size() != static_cast<size_t>(p->batch)) return ID_ERR_ARG;
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return ID_ERR_ARG;
        return ID_OK;
    }
    if (p->plain) {
        if (work != p->bound_work || p->mats.size() != static_cast<size_t>(p->batch) || omega_ld < p->m_max)
            return ID_ERR_ARG;
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return ID_ERR_ARG;
        return ID_OK;
    }
    if (work != p->bound_work || p->maps.size() != static_cast<size_t>(p->batch)) return ID_ERR_ARG;
    if (omega_ld < p->m_max || (omega_ld % 8) != 0 || (reinterpret_cast<uintptr_t>(omega) & 15u) != 0)
        return ID_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return ID_ERR_ARG;
    return ID_OK;
}

id_status_t upload(id_batch_plan* p, void* work, cudaStream_t s) {
    if (cudaMemcpyAsync(work, p->tables.data(), p->table_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return ID_ERR_CUDA;
    p->bound_work = work;
    return ID_OK;
}

}  // namespace

extern "C" {

id_batch_opts_t id_batch_opts_default(void) {
    id_batch_opts_t o;
    memset(&o, 0, sizeof(o));
    o.precision = ID_MIXED_BF16;
    o.oversample = 10;
    o.refine_steps = 1;
    o.rel_tol = 0.0;
    o.watchdog_ms = 0;
    o.tune_cache = nullptr;
    return o;
}

id_status_t id_batch_plan_create(int32_t batch, id_dtype_t a_dtype, const int64_t* m, const int64_t* n,
                                 const int64_t* lda, const int32_t* k, const id_batch_opts_t* opts,
                                 id_batch_plan_t** plan) {
    if (!plan) return ID_ERR_ARG;
    *plan = nullptr;
    if (batch < 1 || !m || !n || !lda || !k) return ID_ERR_ARG;
    if (a_dtype != ID_F64 && a_dtype != ID_F32) return ID_ERR_ARG;
    id_batch_opts_t o = opts ? *opts : id_batch_opts_default();
    const bool plain = o.precision == ID_PLAIN_F64;
    const bool plain32 = o.precision == ID_PLAIN_F32;
    if ((!is_mixed(o.precision) && !plain && !plain32) || o.oversample < 0 || o.refine_steps < 0 || o.rel_tol < 0.0 ||
        !std::isfinite(o.rel_tol))
        return ID_ERR_ARG;
    if (plain && (a_dtype != ID_F64 || o.rel_tol > 0.0)) return ID_ERR_ARG;
    for (int32_t i = 0; i < batch; ++i) {
        if (m[i] < 1 || n[i] < 1 || lda[i] < m[i] || k[i] < 1 || k[i] > m[i] || k[i] > n[i]) return ID_ERR_ARG;
        if (plain) continue;   // the single-matrix FP64 path takes any shape
        if (plain32) {
            if (k[i] > 128) return ID_ERR_UNSUPPORTED;   // the batched solve's rank limit
            continue;
        }
        if (k[i] > 128 || n[i] > kMaxClusterBatch * 128 || m[i] > (int64_t(1) << 31) / 2) return ID_ERR_UNSUPPORTED;
        if (std::min<int64_t>(k[i] + o.oversample, m[i]) > 160) return ID_ERR_UNSUPPORTED;
    }
    auto* p = new id_batch_plan;
    p->batch = batch;
    p->a_f64 = a_dtype == ID_F64 ? 1 : 0;
    p->opts = o;
    p->opts.tune_cache = nullptr;
    p->m.assign(m, m + batch);
    p->n.assign(n, n + batch);
    p->lda.assign(lda, lda + batch);
    p->k.assign(k, k + batch);
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        cudaGetLastError();
        p->device = 0;
    }
    if (o.slab_chunks > 0) p->tune.slab_chunks = o.slab_chunks;
    if (o.cpqr_tpc > 0)
        for (int rc = 0; rc < kNumRowClasses - 1; ++rc) p->tune.tpc[rc] = o.cpqr_tpc;
    if (o.solve_warps > 0) p->tune.solve_warps = o.solve_warps;
    if (o.solve_cols > 0) p->tune.solve_cols = o.solve_cols;
    if (!valid_tuning(p->tune)) {
        delete p;
        return ID_ERR_ARG;
    }
    if (plain) {
        // per-matrix FP64 IDs: workspace slices, the packed J / T offsets and Omega's extent
        p->plain = true;
        p->j_offsets.assign(batch + 1, 0);
        p->t_offsets.assign(batch + 1, 0);
        size_t off = 0;
        for (int32_t i = 0; i < batch; ++i) {
            const double fake = 0.0;
            const id_opts_t oi = plain_opts(p, i, &fake, p->m[i]);
            size_t b = 0;
            const id_status_t st = id_workspace_size(ID_F64, p->m[i], p->n[i], &oi, &b);
            if (st != ID_OK) {
                delete p;
                return st;
            }
            p->woff.push_back(off);
            p->wbytes.push_back(b);
            off = align256(off + b);
            p->j_offsets[i + 1] = p->j_offsets[i] + p->n[i];
            p->t_offsets[i + 1] = p->t_offsets[i] + static_cast<int64_t>(p->k[i]) * (p->n[i] - p->k[i]);
            p->ell_max = std::max(p->ell_max, oi.ell);
            p->m_max = std::max(p->m_max, p->m[i]);
        }
        p->work_bytes = off;
        *plan = p;
        return ID_OK;
    }
    if (plain32) {
        p->plain32 = true;
        if (!build_plan_plain32(p)) {
            delete p;
            return ID_ERR_UNSUPPORTED;
        }
        *plan = p;
        return ID_OK;
    }
    if (o.tune_cache) read_cache(p, o.tune_cache);
    if (!build_plan(p)) {
        delete p;
        return ID_ERR_UNSUPPORTED;
    }
    *plan = p;
    return ID_OK;
}

void id_batch_plan_destroy(id_batch_plan_t* p) {
    if (!p) return;
    if (p->streams_ready) {
        cudaEventDestroy(p->fork);
        for (int i = 0; i < kMaxAuxStreams; ++i) {
            cudaEventDestroy(p->join[i]);
            cudaStreamDestroy(p->aux[i]);
        }
    }
    delete p;
}

id_status_t id_batch_plan_query(const id_batch_plan_t* p, size_t* work_bytes, int64_t* j_offsets,
                                int64_t* t_offsets, int32_t* ell_max, int64_t* m_max) {
    if (!p) return ID_ERR_ARG;
    if (work_bytes) *work_bytes = p->work_bytes;
    if (j_offsets) std::copy(p->j_offsets.begin(), p->j_offsets.end(), j_offsets);
    if (t_offsets) std::copy(p->t_offsets.begin(), p->t_offsets.end(), t_offsets);
    if (ell_max) *ell_max = p->ell_max;
    if (m_max) *m_max = p->m_max;
    return ID_OK;
}

int64_t id_batch_plan_describe(const id_batch_plan_t* p, char* buf, int64_t len) {
    if (!p) return 0;
    std::ostringstream os;
    if (p->plain)
        os << "{\"precision\": \"plain_f64\", \"ids\": " << p->batch << ", \"work_bytes\": " << p->work_bytes
           << "}";
    else if (p->plain32) {
        os << "{\"precision\": \"plain_f32\", \"waves\": " << p->waves.size() << ", \"ids_per_wave\": [";
        for (size_t i = 0; i < p->waves.size(); ++i) os << (i ? ", " : "") << p->waves[i].count;
        os << "], \"ctas_per_id\": [";
        for (size_t i = 0; i < p->waves.size(); ++i) os << (i ? ", " : "") << p->waves[i].gsize;
        os << "], \"column_mode\": [";
        for (size_t i = 0; i < p->waves.size(); ++i) os << (i ? ", " : "") << p->waves[i].colmode;
        os << "], \"solve_units\": " << p->solve_units.size() << ", \"work_bytes\": " << p->work_bytes << "}";
    }
    else
        os << "{" << tuning_json(p, 0.0).substr(0, tuning_json(p, 0.0).rfind(", \"ms\""))
       << ", \"sketch_units\": " << p->sunits.size()
       << ", \"sketch_stages\": " << p->spipe.stages << ", \"cpqr_groups\": " << p->cq_groups.size()
       << ", \"solve_units\": " << p->solve_units.size() << ", \"work_bytes\": " << p->work_bytes << "}";
    const std::string s = os.str();
    if (buf && len > 0) {
        const size_t nc = std::min<size_t>(s.size(), static_cast<size_t>(len - 1));
        memcpy(buf, s.data(), nc);
        buf[nc] = '\0';
    }
    return static_cast<int64_t>(s.size()) + 1;
}

id_status_t id_batch_workspace_size(const id_batch_plan_t* p, size_t* bytes) {
    if (!p || !bytes) return ID_ERR_ARG;
    *bytes = p->work_bytes;
    return ID_OK;
}

id_status_t id_batch_bind(id_batch_plan_t* p, const void* const* A, void* work, size_t work_bytes, void* stream) {
    if (!p || !A || !work) return ID_ERR_ARG;
    if (work_bytes < p->work_bytes) return ID_ERR_WORKSPACE;
    if ((reinterpret_cast<uintptr_t>(work) & 255u) != 0) return ID_ERR_ARG;
    if (p->plain || p->plain32) {
        for (int32_t i = 0; i < p->batch; ++i)
            if (!A[i]) return ID_ERR_ARG;
        p->mats.assign(A, A + p->batch);
        p->bound_work = work;
        if (!p->plain32) return ID_OK;
        write_params_plain32(p, A, work);
        return upload(p, work, static_cast<cudaStream_t>(stream));
    }
    std::vector<CUtensorMap> maps(p->batch);
    for (int32_t i = 0; i < p->batch; ++i)
        if (!A[i] || !encode_a_map(A[i], p->a_f64, p->m[i], p->n[i], p->lda[i], &maps[i])) return ID_ERR_ARG;
    p->maps.swap(maps);
    memcpy(p->tables.data() + p->off_maps, p->maps.data(), p->maps.size() * sizeof(CUtensorMap));
    return upload(p, work, static_cast<cudaStream_t>(stream));
}

id_status_t id_factor_batched(const id_batch_plan_t* p, const void* omega, int64_t omega_ld, int32_t* J, double* T,
                              int32_t* k_out, int32_t* info, void* work, size_t work_bytes, void* stream) {
    const id_status_t st = check_call(p, omega, omega_ld, J, T, k_out, info, work, work_bytes);
    if (st != ID_OK) return st;
    if (p->plain) return enqueue_plain(p, omega, omega_ld, J, T, k_out, info, work, static_cast<cudaStream_t>(stream));
    if (p->plain32) return enqueue_plain32(p, J, T, k_out, info, work, static_cast<cudaStream_t>(stream));
    if (!ensure_streams(const_cast<id_batch_plan*>(p))) return ID_ERR_CUDA;
    return enqueue(p, omega, omega_ld, J, T, k_out, info, work, static_cast<cudaStream_t>(stream));
}

id_status_t id_batch_shard(int32_t batch, const int64_t* m, const int64_t* n, const int32_t* k, int32_t oversample,
                           int32_t world, int32_t* rank_of, double* load) {
    if (batch < 0 || world < 1 || (batch > 0 && (!m || !n || !k || !rank_of)) || oversample < 0) return ID_ERR_ARG;
    std::vector<std::pair<double, int32_t>> work(batch);
    for (int32_t i = 0; i < batch; ++i) {
        if (m[i] < 1 || n[i] < 1 || k[i] < 1) return ID_ERR_ARG;
        const double ell = static_cast<double>(std::min<int64_t>(k[i] + oversample, m[i]));
        const double kk = k[i], nn = static_cast<double>(n[i]), mm = static_cast<double>(m[i]);
        const double f = 2.0 * ell * mm * nn + 4.0 * ell * nn * kk - 2.0 * kk * kk * (ell + nn) +
                         4.0 * kk * kk * kk / 3.0 + kk * kk * std::max(0.0, nn - kk);
        work[i] = {f, i};
    }
    std::stable_sort(work.begin(), work.end(),
                     [](const std::pair<double, int32_t>& a, const std::pair<double, int32_t>& b) {
                         return a.first > b.first;
                     });
    std::vector<double> acc(world, 0.0);
    for (const auto& w : work) {
        int best = 0;
        for (int r = 1; r < world; ++r)
            if (acc[r] < acc[best]) best = r;
        rank_of[w.second] = best;
        acc[best] += w.first;
    }
    if (load)
        for (int r = 0; r < world; ++r) load[r] = acc[r];
    return ID_OK;
}

id_status_t id_batch_autotune(id_batch_plan_t* p, const void* omega, int64_t omega_ld, int32_t* J, double* T,
                              int32_t* k_out, int32_t* info, void* work, size_t work_bytes, void* stream, int32_t reps,
                              const char* cache_path, double* best_ms) {
    id_status_t st = check_call(p, omega, omega_ld, J, T, k_out, info, work, work_bytes);
    if (st != ID_OK) return st;
    if (p->plain || p->plain32) return ID_ERR_ARG;   // nothing to tune: the plain IDs run with their own shapes
    if (!ensure_streams(p)) return ID_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (reps < 1) reps = 5;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return ID_ERR_CUDA;
    // the stage events of this thread would be recorded by every timed call
    auto time_current = [&](double* out) -> id_status_t {
        if (upload(p, work, s) != ID_OK) return ID_ERR_CUDA;
        id_status_t r = enqueue(p, omega, omega_ld, J, T, k_out, info, work, s);   // warm-up
        if (r != ID_OK) return r;
        std::vector<float> t(reps);
        for (int i = 0; i < reps; ++i) {
            cudaEventRecord(e0, s);
            r = enqueue(p, omega, omega_ld, J, T, k_out, info, work, s);
            if (r != ID_OK) return r;
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) return ID_ERR_CUDA;
            cudaEventElapsedTime(&t[i], e0, e1);
        }
        std::sort(t.begin(), t.end());
        *out = t[reps / 2];
        return ID_OK;
    };
    const Tuning start = p->tune;
    Tuning best = start;
    double best_t = 0.0;
    auto apply = [&](const Tuning& t) -> bool {
        p->tune = t;
        return build_plan(p);
    };
    auto fail = [&](id_status_t r) {
        apply(best);
        upload(p, work, s);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return r;
    };
    if (!apply(best)) return fail(ID_ERR_UNSUPPORTED);
    st = time_current(&best_t);
    if (st != ID_OK) return fail(st);
    auto consider = [&](const Tuning& cand) -> id_status_t {
        if (!valid_tuning(cand)) return ID_OK;
        if (!apply(cand)) return ID_OK;   // a shape the kernels do not cover: skip
        double t = 0.0;
        const id_status_t r = time_current(&t);
        if (r != ID_OK) return r;
        if (t < best_t) {
            best_t = t;
            best = cand;
        }
        return ID_OK;
    };
    // coordinate search: sketch unit height, then pivoted-QR threads per column for
    // each row class present, then the solve CTA shape
    for (int S : kSlabCandidates) {
        Tuning c = best;
        c.slab_chunks = S;
        if (S != best.slab_chunks && (st = consider(c)) != ID_OK) return fail(st);
    }
    bool present[kNumRowClasses] = {};
    for (const BatchTask& t : p->tasks) present[row_class(t.ell)] = true;
    for (int rc = 0; rc < kNumRowClasses - 1; ++rc) {
        if (!present[rc]) continue;
        Tuning c = best;
        c.tpc[rc] = best.tpc[rc] == 4 ? 2 : 4;
        if ((st = consider(c)) != ID_OK) return fail(st);
    }
    const int warps_c[] = {4, 8, 16};
    const int cols_c[] = {16, 32, 64, 128};
    for (int wv : warps_c)
        for (int cv : cols_c) {
            if (cv < wv) continue;
            Tuning c = best;
            c.solve_warps = wv;
            c.solve_cols = cv;
            if ((wv != best.solve_warps || cv != best.solve_cols) && (st = consider(c)) != ID_OK) return fail(st);
        }
    if (!apply(best)) return fail(ID_ERR_UNSUPPORTED);
    if (upload(p, work, s) != ID_OK) return fail(ID_ERR_CUDA);
    cudaStreamSynchronize(s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_ms) *best_ms = best_t;
    if (cache_path && !write_cache(p, cache_path, best_t)) return ID_ERR_ARG;
    return ID_OK;
}

}  // extern "C"
