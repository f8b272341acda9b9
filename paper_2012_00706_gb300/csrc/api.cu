// C ABI of the GB300 column-ID library: argument checks, workspace planning
// and the launch sequence of one ID (sketch -> pivoted QR -> coefficient solve
// -> optional error estimate), all enqueued on the caller's stream.
#include "common.cuh"
#include "internal.h"

#include <algorithm>
#include <mutex>
#include <vector>

namespace gid {

const DeviceInfo& device_info() {
    static std::mutex mu;
    static std::vector<DeviceInfo> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        dev = 0;
        cudaGetLastError();
    }
    std::lock_guard<std::mutex> lock(mu);
    if (static_cast<int>(cache.size()) <= dev) cache.resize(dev + 1);
    DeviceInfo& d = cache[dev];
    if (d.sm_count == 0) {
        cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&d.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaDeviceGetAttribute(&d.cc_major, cudaDevAttrComputeCapabilityMajor, dev);
        cudaDeviceGetAttribute(&d.cc_minor, cudaDevAttrComputeCapabilityMinor, dev);
        // without a device (host-only planning) assume the GB300 target: 152 SMs, 227 KB
        if (d.sm_count <= 0) d.sm_count = 152;
        if (d.max_smem_optin <= 0) d.max_smem_optin = 232448;
    }
    return d;
}

static thread_local cudaEvent_t t_stage_events[8];
static thread_local int t_stage_count = 0;

void record_stage(int i, cudaStream_t s) {
    if (i < t_stage_count) cudaEventRecord(t_stage_events[i], s);
}

cudaEvent_t stage_event(int i) { return i < t_stage_count ? t_stage_events[i] : nullptr; }

int pause_stages() {
    const int c = t_stage_count;
    t_stage_count = 0;
    return c;
}

void resume_stages(int count) { t_stage_count = count; }

namespace {

uint64_t limit_ns_of(const id_opts_t& o) {
    const int64_t ms = o.watchdog_ms > 0 ? o.watchdog_ms : 4000;
    return static_cast<uint64_t>(ms) * 1000000ull;
}

bool is_mixed(int p) {
    return p == ID_MIXED_BF16 || p == ID_MIXED_F16 || p == ID_MIXED_BF16X2 || p == ID_MIXED_BF16X3;
}

bool is_low(int p) { return p == ID_LOW_BF16 || p == ID_LOW_F16; }

// Everything id_factor derives from its arguments before touching the GPU.
struct FactorPlan {
    int64_t rows = 0;       // rows of the matrix being pivoted (ell or m)
    int kcap = 0;           // rank capacity (k or k_max)
    int w_f64 = 1;          // working precision of the pivoted QR
    int mixed = 0, sketch = 0;
    int low = 0;            // Algorithm 2 on the whole matrix: pivot the cast A_L
    int64_t omega_ld = 0;
    SketchPlan sp;
    SketchF64Plan sp64;
    CpqrPlan cp;
    ClusterCpqrPlan ccp;
    int use_cluster = 0;    // FP32 pivoting of at most 128 rows: one thread-block cluster
    size_t ctrl_bytes = 0;  // the grid kernels' control region (the largest any launch of the plan needs)
    size_t bytes = 0;
};

struct FactorPtrs {
    void* ctrl;
    uint8_t* sel;
    void* nu;
    void* nuref;
    void* W;
    void* partial;
    double* R64;
    double* tscr;
    double* acc;
};

size_t carve_factor(void* base, int64_t n, const FactorPlan& p, FactorPtrs* out) {
    Carver c(base);
    const int elem = p.w_f64 ? 8 : 4;
    FactorPtrs f{};
    f.ctrl = c.take<uint8_t>(p.ctrl_bytes);
    f.sel = c.take<uint8_t>(static_cast<size_t>(n));
    f.nu = c.take<uint8_t>(static_cast<size_t>(n) * elem);
    f.nuref = c.take<uint8_t>(static_cast<size_t>(n) * elem);
    f.W = c.take<uint8_t>(static_cast<size_t>(p.rows) * n * elem);
    if (p.sketch) {
        if (p.mixed) f.partial = c.take<uint8_t>(sketch_partial_bytes_lowp(p.sp, n));
        else f.partial = c.take<double>(static_cast<size_t>(p.sp64.kslabs) * n * p.sp64.lp);
    }
    f.R64 = c.take<double>(static_cast<size_t>(p.kcap) * n);
    f.tscr = c.take<double>(solve_T_scratch_doubles(p.kcap, n));
    f.acc = c.take<double>(4);
    if (out) *out = f;
    return c.off + 256;
}

id_status_t plan_factor(id_dtype_t a_dtype, int64_t m, int64_t n, int64_t lda, const id_opts_t* o,
                        FactorPlan* plan) {
    if (!o || m < 1 || n < 1 || lda < m) return ID_ERR_ARG;
    if (a_dtype != ID_F64 && a_dtype != ID_F32) return ID_ERR_ARG;
    if (n > (int64_t(1) << 31) - 1) return ID_ERR_UNSUPPORTED;
    FactorPlan p;
    const int prec = o->precision;
    if (prec < ID_PLAIN_F64 || prec > ID_LOW_F16) return ID_ERR_ARG;
    p.mixed = is_mixed(prec);
    p.low = is_low(prec);
    p.sketch = o->sketch ? 1 : 0;
    if (p.mixed && !p.sketch) return ID_ERR_ARG;
    if ((prec == ID_PLAIN_F32 || p.low) && p.sketch) return ID_ERR_ARG;
    p.w_f64 = (prec == ID_PLAIN_F64) ? 1 : 0;
    if (p.sketch) {
        if (o->ell < 1 || o->ell > m || !o->omega) return ID_ERR_ARG;
        if (p.mixed && o->ell > ID_MAX_ELL) return ID_ERR_ARG;
        if (prec == ID_PLAIN_F64 && a_dtype != ID_F64) return ID_ERR_ARG;
        p.rows = o->ell;
        p.omega_ld = o->omega_ld > 0 ? o->omega_ld : m;
        if (p.omega_ld < m) return ID_ERR_ARG;
        if (p.mixed && ((p.omega_ld % 8) != 0 || (reinterpret_cast<uintptr_t>(o->omega) & 15u) != 0))
            return ID_ERR_ARG;
    } else {
        p.rows = m;
    }
    const int64_t kmax_possible = std::min<int64_t>(p.rows, n);
    if (o->rel_tol > 0.0) {
        if (o->k_max < 1 || o->k_max > kmax_possible) return ID_ERR_ARG;
        p.kcap = o->k_max;
    } else {
        if (o->rel_tol < 0.0 || o->k < 1 || o->k > kmax_possible) return ID_ERR_ARG;
        p.kcap = o->k;
    }
    if (o->refine_steps < 0) return ID_ERR_ARG;
    if (p.sketch) {
        if (p.mixed) {
            if (!sketch_plan_lowp(m, n, o->ell, a_dtype == ID_F64, precision_nsplit(prec), &p.sp))
                return ID_ERR_UNSUPPORTED;
        } else {
            sketch_plan_f64(m, n, o->ell, &p.sp64);
        }
    }
    if (!cpqr_plan(p.rows, n, p.w_f64 ? 8 : 4, &p.cp)) return ID_ERR_UNSUPPORTED;
    // the cluster kernel reads A directly when it is a short float matrix (PLAIN_F32, no
    // sketch), or the sketch Y, or the cast A_L
    const bool short_f32 = !p.w_f64 && (p.sketch || p.low || a_dtype == ID_F32);
    p.use_cluster = short_f32 && cpqr_cluster_plan(p.rows, n, &p.ccp) ? 1 : 0;
    p.ctrl_bytes = cpqr_ctrl_bytes(p.cp, p.rows, p.w_f64 ? 8 : 4);
    p.bytes = carve_factor(nullptr, n, p, nullptr);
    *plan = p;
    return ID_OK;
}

}  // namespace
}  // namespace gid

using namespace gid;

extern "C" {

void id_opts_default(id_opts_t* o) {
    if (!o) return;
    o->k = 0;
    o->rel_tol = 0.0;
    o->k_max = 0;
    o->sketch = 0;
    o->ell = 0;
    o->precision = ID_PLAIN_F64;
    o->omega = nullptr;
    o->omega_ld = 0;
    o->refine_steps = 1;
    o->estimate_error = 0;
    o->watchdog_ms = 0;
}

const char* id_status_string(id_status_t s) {
    switch (s) {
        case ID_OK: return "ID_OK: success";
        case ID_ERR_ARG: return "ID_ERR_ARG: invalid argument";
        case ID_ERR_WORKSPACE: return "ID_ERR_WORKSPACE: workspace smaller than id_workspace_size()";
        case ID_ERR_CUDA: return "ID_ERR_CUDA: a CUDA runtime call failed";
        case ID_ERR_TIMEOUT: return "ID_ERR_TIMEOUT: a device wait gave up (watchdog)";
        case ID_ERR_UNSUPPORTED: return "ID_ERR_UNSUPPORTED: shape or option not supported";
    }
    return "unknown status";
}

const char* id_version(void) { return "gb300-id 0.1 (sm_103a)"; }

id_status_t id_set_stage_events(void* const* events, int32_t count) {
    if (!events || count <= 0) {
        t_stage_count = 0;
        return ID_OK;
    }
    t_stage_count = count > 8 ? 8 : count;
    for (int i = 0; i < t_stage_count; ++i) t_stage_events[i] = static_cast<cudaEvent_t>(events[i]);
    return ID_OK;
}

id_status_t id_workspace_size(id_dtype_t a_dtype, int64_t m, int64_t n, const id_opts_t* opts, size_t* bytes) {
    if (!bytes) return ID_ERR_ARG;
    FactorPlan p;
    const id_status_t st = plan_factor(a_dtype, m, n, m, opts, &p);
    if (st != ID_OK) return st;
    *bytes = p.bytes;
    return ID_OK;
}

id_status_t id_factor(const void* A, id_dtype_t a_dtype, int64_t m, int64_t n, int64_t lda, const id_opts_t* opts,
                      int32_t* J, double* T, int64_t ldt, int32_t* k_out, int32_t* info, double* err_out,
                      void* work, size_t work_bytes, void* stream) {
    if (!A || !J || !T || !k_out || !info || !work) return ID_ERR_ARG;
    FactorPlan p;
    id_status_t st = plan_factor(a_dtype, m, n, lda, opts, &p);
    if (st != ID_OK) return st;
    if (ldt < p.kcap) return ID_ERR_ARG;
    if (opts->estimate_error && !err_out) return ID_ERR_ARG;
    if (work_bytes < p.bytes) return ID_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FactorPtrs f;
    void* aligned = reinterpret_cast<void*>((reinterpret_cast<uintptr_t>(work) + 255) & ~uintptr_t(255));
    carve_factor(aligned, n, p, &f);
    const uint64_t lim = limit_ns_of(*opts);
    const int a_f64 = a_dtype == ID_F64;

    cudaError_t e = cudaMemsetAsync(info, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(k_out, 0, sizeof(int32_t), s);
    record_stage(0, s);
    const void* cpqr_src = nullptr;
    int64_t ldsrc = 0;
    if (e == cudaSuccess && p.sketch) {
        if (p.mixed) {
            // the split-K partial sums are reduced by a whole-GPU pass: the pivoted QR runs on
            // one cluster, too few SMs to gather the slabs quickly itself
            e = launch_sketch_lowp(A, a_f64, m, n, lda, static_cast<const uint16_t*>(opts->omega), p.omega_ld,
                                   opts->ell, opts->precision, p.sp, static_cast<float*>(f.partial),
                                   static_cast<float*>(f.W), opts->ell, info, lim, s, stage_event(1));
        } else {
            e = launch_sketch_f64(static_cast<const double*>(A), m, n, lda,
                                  static_cast<const double*>(opts->omega), p.omega_ld, opts->ell, p.sp64,
                                  static_cast<double*>(f.partial), static_cast<double*>(f.W), opts->ell, info, s,
                                  stage_event(1));
        }
    } else if (e == cudaSuccess && p.low) {
        // Algorithm 2's A_L: the scaled low-precision cast of A, as FP32 values, in W
        e = launch_low_cast(A, a_f64, m, n, lda, opts->precision == ID_LOW_F16 ? 1 : 0, static_cast<float*>(f.W),
                            m, info, s);
        record_stage(1, s);
    } else if (e == cudaSuccess) {
        record_stage(1, s);
        cpqr_src = A;
        ldsrc = lda;
    }
    record_stage(2, s);
    const double rel_tol = opts->rel_tol > 0.0 ? opts->rel_tol : 0.0;
    if (e == cudaSuccess) {
        if (p.use_cluster) {
            // short FP32 matrix: the sketch Y (or a short A) goes straight to the cluster kernel
            const float* Wf = static_cast<const float*>(f.W);
            int64_t ldw = p.rows;
            if (!p.sketch && !p.low) {
                Wf = static_cast<const float*>(A);
                ldw = lda;
            }
            e = launch_cpqr_cluster(Wf, p.rows, n, ldw, 1, 0, p.kcap, rel_tol, J, k_out, info, f.R64, p.kcap, f.sel,
                                    p.ccp, lim, s);
        } else {
            e = launch_cpqr(f.W, p.w_f64, p.rows, n, p.rows, cpqr_src, a_f64, ldsrc, p.kcap, rel_tol, J, k_out, info,
                            f.R64, p.kcap, f.nu, f.nuref, f.sel, f.ctrl, p.cp, lim, s);
        }
    }
    record_stage(3, s);
    if (e == cudaSuccess)
        e = launch_solve_T(f.R64, p.kcap, J, k_out, p.kcap, n, T, ldt, f.tscr, opts->refine_steps, p.w_f64 ? 0 : 1,
                           s);
    record_stage(4, s);
    if (e == cudaSuccess && opts->estimate_error)
        e = launch_residual_fro(A, a_f64, m, n, lda, J, k_out, T, ldt, p.kcap, f.acc, err_out,
                                reinterpret_cast<float*>(f.tscr), s);
    record_stage(5, s);
    return e == cudaSuccess ? ID_OK : ID_ERR_CUDA;
}

id_status_t id_sketch_workspace_size(id_dtype_t a_dtype, int64_t m, int64_t n, int32_t ell, int32_t precision,
                                     size_t* bytes) {
    if (!bytes || m < 1 || n < 1 || ell < 1 || ell > m) return ID_ERR_ARG;
    if (precision == ID_PLAIN_F64) {
        if (a_dtype != ID_F64) return ID_ERR_ARG;
        SketchF64Plan sp;
        sketch_plan_f64(m, n, ell, &sp);
        *bytes = static_cast<size_t>(sp.kslabs) * n * sp.lp * sizeof(double) + 512;
        return ID_OK;
    }
    if (!is_mixed(precision) || ell > ID_MAX_ELL) return ID_ERR_ARG;
    SketchPlan sp;
    if (!sketch_plan_lowp(m, n, ell, a_dtype == ID_F64, precision_nsplit(precision), &sp)) return ID_ERR_UNSUPPORTED;
    *bytes = sketch_partial_bytes_lowp(sp, n) + 512;
    return ID_OK;
}

id_status_t id_sketch(const void* A, id_dtype_t a_dtype, int64_t m, int64_t n, int64_t lda, const void* omega,
                      int64_t omega_ld, int32_t ell, int32_t precision, void* Y, int64_t ldy, int32_t* info,
                      void* work, size_t work_bytes, void* stream) {
    if (!A || !omega || !Y || !work || lda < m || ldy < ell) return ID_ERR_ARG;
    size_t need = 0;
    id_status_t st = id_sketch_workspace_size(a_dtype, m, n, ell, precision, &need);
    if (st != ID_OK) return st;
    if (work_bytes < need) return ID_ERR_WORKSPACE;
    const int64_t ldo = omega_ld > 0 ? omega_ld : m;
    if (ldo < m) return ID_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void* aligned = reinterpret_cast<void*>((reinterpret_cast<uintptr_t>(work) + 255) & ~uintptr_t(255));
    cudaError_t e = cudaSuccess;
    if (info) e = cudaMemsetAsync(info, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return ID_ERR_CUDA;
    if (precision == ID_PLAIN_F64) {
        SketchF64Plan sp;
        sketch_plan_f64(m, n, ell, &sp);
        e = launch_sketch_f64(static_cast<const double*>(A), m, n, lda, static_cast<const double*>(omega), ldo, ell,
                              sp, static_cast<double*>(aligned), static_cast<double*>(Y), ldy, info, s);
    } else {
        if ((ldo % 8) != 0 || (reinterpret_cast<uintptr_t>(omega) & 15u) != 0) return ID_ERR_ARG;
        SketchPlan sp;
        sketch_plan_lowp(m, n, ell, a_dtype == ID_F64, precision_nsplit(precision), &sp);
        e = launch_sketch_lowp(A, a_dtype == ID_F64, m, n, lda, static_cast<const uint16_t*>(omega), ldo, ell,
                               precision, sp, static_cast<float*>(aligned), static_cast<float*>(Y), ldy, info,
                               4000000000ull, s);
    }
    return e == cudaSuccess ? ID_OK : ID_ERR_CUDA;
}

id_status_t id_scale_cast(const void* A, id_dtype_t a_dtype, int64_t m, int64_t n, int64_t lda, int32_t precision,
                          uint16_t* pieces, int32_t* shifts, int32_t* info, void* stream) {
    if (!A || !pieces || !shifts || m < 1 || n < 1 || lda < m || !is_mixed(precision)) return ID_ERR_ARG;
    if (a_dtype != ID_F64 && a_dtype != ID_F32) return ID_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (info) e = cudaMemsetAsync(info, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = launch_scale_cast(A, a_dtype == ID_F64, m, n, lda, precision, pieces, shifts, info, s);
    return e == cudaSuccess ? ID_OK : ID_ERR_CUDA;
}

// ---------------------------------------------------------- rank-adaptive ID

namespace {
struct AdaptivePlan {
    FactorPlan f;
    size_t y_off = 0, partial_off = 0, bytes = 0;
};

// Split-K partial sums of one round's sketch of b rows.
size_t adaptive_partial_bytes(id_dtype_t a_dtype, int64_t m, int64_t n, int b, int precision) {
    if (precision == ID_PLAIN_F64) {
        SketchF64Plan sp;
        sketch_plan_f64(m, n, b, &sp);
        return static_cast<size_t>(sp.kslabs) * n * sp.lp * sizeof(double);
    }
    SketchPlan sp;
    if (!sketch_plan_lowp(m, n, b, a_dtype == ID_F64, precision_nsplit(precision), &sp)) return 0;
    return sketch_partial_bytes_lowp(sp, n);
}

id_status_t plan_adaptive(id_dtype_t a_dtype, int64_t m, int64_t n, const id_opts_t* o, int32_t block,
                          int32_t oversample, AdaptivePlan* ap) {
    if (!o || block < 1 || oversample < 0 || !(o->rel_tol > 0.0) || !o->sketch) return ID_ERR_ARG;
    if (o->precision != ID_PLAIN_F64 && !is_mixed(o->precision)) return ID_ERR_ARG;
    if (o->k_max < 1 || o->k_max > o->ell - oversample || o->k_max > n) return ID_ERR_ARG;
    id_opts_t fo = *o;
    fo.rel_tol = 0.0;
    fo.k = o->k_max;
    AdaptivePlan p;
    const id_status_t st = plan_factor(a_dtype, m, n, m, &fo, &p.f);
    if (st != ID_OK) return st;
    const size_t elem = p.f.w_f64 ? 8 : 4;
    // the rounds pivot ell = block, 2 block, ..., ell_max rows: a shorter round may take the
    // resident kernel, whose control region holds published columns, where ell_max does not
    for (int64_t e = std::min<int64_t>(block, o->ell);; e = std::min<int64_t>(e + block, o->ell)) {
        CpqrPlan cp;
        if (cpqr_plan(e, n, static_cast<int>(elem), &cp))
            p.f.ctrl_bytes = std::max(p.f.ctrl_bytes, cpqr_ctrl_bytes(cp, e, static_cast<int>(elem)));
        if (e >= o->ell) break;
    }
    p.f.bytes = carve_factor(nullptr, n, p.f, nullptr);
    // the rounds sketch `block` rows, the last one the remainder
    const int rem = static_cast<int>(o->ell % block);
    size_t part = adaptive_partial_bytes(a_dtype, m, n, std::min<int>(block, o->ell), o->precision);
    if (rem > 0) part = std::max(part, adaptive_partial_bytes(a_dtype, m, n, rem, o->precision));
    if (part == 0) return ID_ERR_UNSUPPORTED;
    p.y_off = (p.f.bytes + 255) & ~size_t(255);
    p.partial_off = (p.y_off + static_cast<size_t>(o->ell) * n * elem + 255) & ~size_t(255);
    p.bytes = p.partial_off + part + 256;
    *ap = p;
    return ID_OK;
}
}  // namespace

id_status_t id_adaptive_workspace_size(id_dtype_t a_dtype, int64_t m, int64_t n, const id_opts_t* opts,
                                       int32_t block, int32_t oversample, size_t* bytes) {
    if (!bytes) return ID_ERR_ARG;
    AdaptivePlan ap;
    const id_status_t st = plan_adaptive(a_dtype, m, n, opts, block, oversample, &ap);
    if (st == ID_OK) *bytes = ap.bytes;
    return st;
}

id_status_t id_factor_adaptive(const void* A, id_dtype_t a_dtype, int64_t m, int64_t n, int64_t lda,
                               const id_opts_t* opts, int32_t block, int32_t oversample, int32_t* J, double* T,
                               int64_t ldt, int32_t* k_out, int32_t* info, double* err_out, int32_t* ell_out,
                               void* work, size_t work_bytes, void* stream) {
    if (!A || !J || !T || !k_out || !info || !err_out || !work || lda < m) return ID_ERR_ARG;
    AdaptivePlan ap;
    id_status_t st = plan_adaptive(a_dtype, m, n, opts, block, oversample, &ap);
    if (st != ID_OK) return st;
    const FactorPlan& p = ap.f;
    if (ldt < opts->k_max) return ID_ERR_ARG;
    if (work_bytes < ap.bytes) return ID_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* aligned = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(work) + 255) & ~uintptr_t(255));
    FactorPtrs f;
    carve_factor(aligned, n, p, &f);
    void* Y = aligned + ap.y_off;
    void* partial = aligned + ap.partial_off;
    const int64_t ell_max = opts->ell, ldo = p.omega_ld, ldy = ell_max;
    const uint64_t lim = limit_ns_of(*opts);
    const int a_f64 = a_dtype == ID_F64;
    const int elem = p.w_f64 ? 8 : 4;
    int64_t ell = 0;
    int32_t h_info = 0;
    while (ell < ell_max) {
        const int64_t e0 = ell;
        ell = std::min<int64_t>(ell + block, ell_max);
        const int b = static_cast<int>(ell - e0);
        const int k = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>({opts->k_max, ell - oversample, n})));
        cudaError_t e = cudaMemsetAsync(info, 0, sizeof(int32_t), s);
        // the block's rows of the sketch: Y(e0:ell, :) = Omega(e0:ell, :) A
        if (e == cudaSuccess) {
            if (p.mixed) {
                SketchPlan sp;
                if (!sketch_plan_lowp(m, n, b, a_f64, precision_nsplit(opts->precision), &sp)) return ID_ERR_UNSUPPORTED;
                e = launch_sketch_lowp(A, a_f64, m, n, lda, static_cast<const uint16_t*>(opts->omega) + e0 * ldo, ldo,
                                       b, opts->precision, sp, static_cast<float*>(partial),
                                       static_cast<float*>(Y) + e0, ldy, info, lim, s);
            } else {
                SketchF64Plan sp;
                sketch_plan_f64(m, n, b, &sp);
                e = launch_sketch_f64(static_cast<const double*>(A), m, n, lda,
                                      static_cast<const double*>(opts->omega) + e0 * ldo, ldo, b, sp,
                                      static_cast<double*>(partial), static_cast<double*>(Y) + e0, ldy, info, s);
            }
        }
        // rank-k pivoted QR of Y(0:ell, :) (the kernels read Y and leave it as it is)
        if (e == cudaSuccess) {
            ClusterCpqrPlan ccp;
            if (p.mixed && cpqr_cluster_plan(ell, n, &ccp)) {
                e = launch_cpqr_cluster(static_cast<const float*>(Y), ell, n, ldy, 1, 0, k, 0.0, J, k_out, info,
                                        f.R64, opts->k_max, f.sel, ccp, lim, s);
            } else {
                CpqrPlan cp;
                if (!cpqr_plan(ell, n, elem, &cp)) return ID_ERR_UNSUPPORTED;
                e = launch_cpqr(f.W, p.w_f64, ell, n, ell, Y, p.w_f64, ldy, k, 0.0, J, k_out, info, f.R64,
                                opts->k_max, f.nu, f.nuref, f.sel, f.ctrl, cp, lim, s);
            }
        }
        if (e == cudaSuccess)
            e = launch_solve_T(f.R64, opts->k_max, J, k_out, k, n, T, ldt, f.tscr, opts->refine_steps,
                               p.w_f64 ? 0 : 1, s);
        if (e == cudaSuccess)
            e = launch_residual_fro(A, a_f64, m, n, lda, J, k_out, T, ldt, k, f.acc, err_out,
                                    reinterpret_cast<float*>(f.tscr), s);
        double h_err = 0.0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err_out, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h_info, info, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return ID_ERR_CUDA;
        if (h_info < 0) break;                      // non-finite data or a watchdog: report, stop
        if (h_err <= opts->rel_tol) break;
    }
    if (ell_out) *ell_out = static_cast<int32_t>(ell);
    return h_info == kInfoWatchdog ? ID_ERR_TIMEOUT : ID_OK;
}

// ------------------------------------------------------- row and two-sided IDs

namespace {
int64_t round_up8(int64_t x) { return (x + 7) / 8 * 8; }
size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
}  // namespace

id_status_t id_rows_workspace_size(id_dtype_t a_dtype, int64_t m, int64_t n, const id_opts_t* opts, size_t* bytes) {
    if (!bytes || (a_dtype != ID_F64 && a_dtype != ID_F32)) return ID_ERR_ARG;
    size_t fb = 0;
    const id_status_t st = id_workspace_size(a_dtype, n, m, opts, &fb);   // the column ID of A^T (n x m)
    if (st != ID_OK) return st;
    const size_t elem = a_dtype == ID_F64 ? 8 : 4;
    *bytes = align256(static_cast<size_t>(round_up8(n)) * m * elem) + fb + 512;
    return ID_OK;
}

id_status_t id_factor_rows(const void* A, id_dtype_t a_dtype, int64_t m, int64_t n, int64_t lda, const id_opts_t* opts,
                           int32_t* I, double* T, int64_t ldt, int32_t* k_out, int32_t* info, double* err_out,
                           void* work, size_t work_bytes, void* stream) {
    if (!A || !work || m < 1 || n < 1 || lda < m) return ID_ERR_ARG;
    size_t need = 0;
    id_status_t st = id_rows_workspace_size(a_dtype, m, n, opts, &need);
    if (st != ID_OK) return st;
    if (work_bytes < need) return ID_ERR_WORKSPACE;
    char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(work) + 255) & ~uintptr_t(255));
    const size_t elem = a_dtype == ID_F64 ? 8 : 4;
    const int64_t ldb = round_up8(n);
    const size_t tb = align256(static_cast<size_t>(ldb) * m * elem);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (launch_transpose(A, a_dtype == ID_F64, m, n, lda, base, ldb, s) != cudaSuccess) return ID_ERR_CUDA;
    return id_factor(base, a_dtype, n, m, ldb, opts, I, T, ldt, k_out, info, err_out, base + tb,
                     work_bytes - tb - static_cast<size_t>(base - static_cast<char*>(work)), stream);
}

namespace {
// The row stage of the two-sided ID: the rank-k row ID of the m x k skeleton, plain precision.
id_opts_t two_sided_row_opts(id_dtype_t a_dtype, int32_t k) {
    id_opts_t o;
    id_opts_default(&o);
    o.k = k;
    o.precision = a_dtype == ID_F64 ? ID_PLAIN_F64 : ID_PLAIN_F32;
    return o;
}
}  // namespace

id_status_t id_two_sided_workspace_size(id_dtype_t a_dtype, int64_t m, int64_t n, const id_opts_t* opts,
                                        size_t* bytes) {
    if (!bytes || !opts || opts->rel_tol != 0.0) return ID_ERR_ARG;
    size_t cb = 0, rb = 0;
    id_status_t st = id_workspace_size(a_dtype, m, n, opts, &cb);
    if (st != ID_OK) return st;
    const int32_t k = opts->k;
    if (k > m) return ID_ERR_ARG;
    const id_opts_t ro = two_sided_row_opts(a_dtype, k);
    st = id_rows_workspace_size(a_dtype, m, k, &ro, &rb);
    if (st != ID_OK) return st;
    const size_t elem = a_dtype == ID_F64 ? 8 : 4;
    *bytes = align256(cb) + align256(static_cast<size_t>(round_up8(m)) * k * elem) + rb + 512;
    return ID_OK;
}

id_status_t id_factor_two_sided(const void* A, id_dtype_t a_dtype, int64_t m, int64_t n, int64_t lda,
                                const id_opts_t* opts, int32_t* J, double* Tc, int64_t ldtc, int32_t* I, double* Tr,
                                int64_t ldtr, int32_t* k_out, int32_t* info, void* work, size_t work_bytes,
                                void* stream) {
    if (!A || !J || !Tc || !I || !Tr || !k_out || !info || !work || lda < m) return ID_ERR_ARG;
    size_t need = 0;
    id_status_t st = id_two_sided_workspace_size(a_dtype, m, n, opts, &need);
    if (st != ID_OK) return st;
    if (work_bytes < need) return ID_ERR_WORKSPACE;
    char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(work) + 255) & ~uintptr_t(255));
    const size_t avail = work_bytes - static_cast<size_t>(base - static_cast<char*>(work));
    size_t cb = 0;
    id_workspace_size(a_dtype, m, n, opts, &cb);
    const size_t elem = a_dtype == ID_F64 ? 8 : 4;
    const int32_t k = opts->k;
    const int64_t ldc = round_up8(m);
    const size_t c_off = align256(cb), r_off = c_off + align256(static_cast<size_t>(ldc) * k * elem);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // column stage: A ~= A(:,J[0:k]) Pc
    st = id_factor(A, a_dtype, m, n, lda, opts, J, Tc, ldtc, k_out, info, nullptr, base, cb, stream);
    if (st != ID_OK) return st;
    // row stage: the skeleton C = A(:,J[0:k]) ~= X C(I[0:k], :), a rank-k row ID
    if (launch_gather_cols(A, a_dtype == ID_F64, m, lda, J, k, base + c_off, ldc, s) != cudaSuccess)
        return ID_ERR_CUDA;
    const id_opts_t ro = two_sided_row_opts(a_dtype, k);
    return id_factor_rows(base + c_off, a_dtype, m, k, ldc, &ro, I, Tr, ldtr, k_out + 1, info + 1, nullptr,
                          base + r_off, avail - r_off, stream);
}

id_status_t id_low_cast(const void* A, id_dtype_t a_dtype, int64_t m, int64_t n, int64_t lda, int32_t precision,
                        float* AL, int64_t ldal, int32_t* info, void* stream) {
    if (!A || !AL || m < 1 || n < 1 || lda < m || ldal < m) return ID_ERR_ARG;
    if (a_dtype != ID_F64 && a_dtype != ID_F32) return ID_ERR_ARG;
    if (!is_low(precision) && !is_mixed(precision)) return ID_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (info) e = cudaMemsetAsync(info, 0, sizeof(int32_t), s);
    const int f16 = (precision == ID_LOW_F16 || precision == ID_MIXED_F16) ? 1 : 0;
    if (e == cudaSuccess) e = launch_low_cast(A, a_dtype == ID_F64, m, n, lda, f16, AL, ldal, info, s);
    return e == cudaSuccess ? ID_OK : ID_ERR_CUDA;
}

id_status_t id_reconstruct_one(const void* A, id_dtype_t a_dtype, int64_t m, int64_t n, int64_t lda,
                               const int32_t* J, int32_t k, const double* T, int64_t ldt, void* Ahat, int64_t ldh,
                               void* stream) {
    if (!A || !J || !Ahat || m < 1 || n < 1 || lda < m || ldh < m || k < 1 || k > n) return ID_ERR_ARG;
    if (a_dtype != ID_F64 && a_dtype != ID_F32) return ID_ERR_ARG;
    if (k < n && (!T || ldt < k)) return ID_ERR_ARG;
    const cudaError_t e = launch_reconstruct_one(A, a_dtype == ID_F64, m, n, lda, J, k, T, ldt, Ahat, ldh,
                                                 static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ID_OK : ID_ERR_CUDA;
}

}  // extern "C"
