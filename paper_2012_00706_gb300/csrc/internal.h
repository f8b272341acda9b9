// Host-side declarations shared by the translation units of the library.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/gb300_id.h"

namespace gid {

// Rows of one scaling / pipeline chunk of the tensor-core sketch.
constexpr int kChunkRows = ID_SCALE_BLOCK_ROWS;
// Columns of A per sketch CTA (the MMA's M).
constexpr int kTileCols = 128;

struct DeviceInfo {
    int sm_count = 0;
    int max_smem_optin = 0;
    int cc_major = 0, cc_minor = 0;
};
const DeviceInfo& device_info();   // current device, cached

// Stage-boundary events set with id_set_stage_events (this host thread): record event i.
void record_stage(int i, cudaStream_t s);
cudaEvent_t stage_event(int i);
// Stop recording stage events (returns how many were set) and start again; a call made of
// several id_factor calls keeps its own boundaries this way.
int pause_stages();
void resume_stages(int count);

// Bump allocator over the caller's workspace (256-byte alignment).
struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(void* b) : base(static_cast<char*>(b)) {}
    template <typename T>
    T* take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

// ---- batched ID: task and work-unit tables (device copies built by the batch plan)
struct BatchTask {
    int64_t m, n, lda;
    int32_t kcap;          // fixed rank, or the rank cap under a tolerance
    int32_t ell, lp;       // sketch rows and the MMA N (ell rounded up to 16)
    int32_t kslabs;        // row slabs of the split-K sketch
    int64_t partial_off;   // floats: sketch partial sums [kslabs][n][lp]
    int64_t r_off;         // doubles: R rows 0..kcap-1 of every column (ldr = kcap)
    int64_t j_off;         // int32: J (n entries)
    int64_t t_off;         // doubles: T (ldt = kcap, tcols columns reserved)
    int64_t tcols;
    int64_t sel_off;       // bytes: selected-column flags (n)
    double rel_tol;
    int64_t inv_off;       // floats: the product solve's R11 inverse, packed R11 and flag
};
// Element counts of the batch workspace regions and outputs (bounds the kernels check
// every table entry against before using it).
struct BatchTotals {
    int64_t ntasks = 0, partial = 0, r = 0, j = 0, t = 0, sel = 0, inv = 0;
};
struct SolveUnit {
    int32_t task, c0, ncols, pad;   // columns [c0, c0 + ncols) of T
};
struct SketchUnit {
    int32_t task, tile;    // matrix and 128-column tile
    int32_t c0, nloc;      // first 64-row chunk and chunk count
    int32_t slab, pad;     // row slab (partial-sum slot)
};

// ---- sketch (sketch.cu); launch_sketch_lowp with Y == nullptr leaves only the partial sums
struct SketchPlan {
    int lp = 0;             // MMA N: ell rounded up to 16
    int tiles = 0;          // ceil(n / 128)
    int64_t nchunks = 0;    // ceil(m / 64)
    int64_t chunks_per_slab = 0;
    int kslabs = 0;
    int stages = 0, aop_bufs = 0, omega_bufs = 0, acc_bufs = 0;
    int aop_in_stage = 0;
    size_t smem_bytes = 0;
};
int precision_nsplit(int precision);
int precision_is_f16(int precision);
bool sketch_plan_lowp(int64_t m, int64_t n, int ell, int a_f64, int nsplit, SketchPlan* plan);
size_t sketch_partial_bytes_lowp(const SketchPlan& p, int64_t n);
cudaError_t launch_sketch_lowp(const void* A, int a_f64, int64_t m, int64_t n, int64_t lda,
                               const uint16_t* omega, int64_t ldo, int ell, int precision,
                               const SketchPlan& plan, float* partial, float* Y, int64_t ldy,
                               int32_t* info, uint64_t limit_ns, cudaStream_t s,
                               cudaEvent_t after_main = nullptr);
// Pipeline depth and shared memory of the tensor-core sketch for MMA width lp.
bool sketch_pipeline_plan(int lp, int a_f64, int nsplit, SketchPlan* plan);
// Batched sketch: one CTA per unit of the table (units ordered largest first); matrix i
// is read through maps[i] (encode_a_map), all matrices share the leading
// ell_rows x m_rows part of Omega.
bool encode_a_map(const void* A, int a_f64, int64_t m, int64_t n, int64_t lda, CUtensorMap* map);
cudaError_t launch_sketch_lowp_batched(const SketchUnit* units, int64_t nunits, const BatchTask* tasks,
                                       const CUtensorMap* maps, int a_f64, const uint16_t* omega, int64_t ldo,
                                       int64_t m_rows, int ell_rows, int precision, const SketchPlan& plan,
                                       float* partial, int64_t partial_total, int64_t ntasks, int32_t* infos,
                                       uint64_t limit_ns, cudaStream_t s);

struct SketchF64Plan {
    int kslabs = 0;
    int64_t k_per_slab = 0;
    int lp = 0;
};
void sketch_plan_f64(int64_t m, int64_t n, int ell, SketchF64Plan* plan);
cudaError_t launch_sketch_f64(const double* A, int64_t m, int64_t n, int64_t lda,
                              const double* omega, int64_t ldo, int ell,
                              const SketchF64Plan& plan, double* partial, double* Y, int64_t ldy,
                              int32_t* info, cudaStream_t s, cudaEvent_t after_main = nullptr);
cudaError_t launch_scale_cast(const void* A, int a_f64, int64_t m, int64_t n, int64_t lda,
                              int precision, uint16_t* pieces, int32_t* shifts, int32_t* info,
                              cudaStream_t s);
// A_L of Algorithm 2 as FP32 values (2^s fl_low(x 2^-s) per 64-row block and column), out: m x n, ldo.
cudaError_t launch_low_cast(const void* A, int a_f64, int64_t m, int64_t n, int64_t lda, int f16, float* out,
                            int64_t ldo, int32_t* info, cudaStream_t s);

// ---- pivoted QR (cpqr.cu)
struct CpqrPlan {
    int grid = 0;
    int threads = 0;
    int resident = 0;     // the CTAs keep their columns in shared memory
    size_t smem = 0;      // dynamic shared memory per CTA
};
bool cpqr_plan(int64_t r, int64_t n, int elem_bytes, CpqrPlan* plan);
size_t cpqr_ctrl_bytes(const CpqrPlan& plan, int64_t r, int elem_bytes);
size_t cpqr_pub_offset(int grid);   // offset of the column slots in the control region
cudaError_t launch_cpqr(void* W, int w_f64, int64_t r, int64_t n, int64_t ldw, const void* src,
                        int src_f64, int64_t ldsrc, int kcap, double rel_tol, int32_t* J,
                        int32_t* k_out, int32_t* info, double* R64, int64_t ldr, void* nu,
                        void* nuref, uint8_t* sel, void* ctrl, const CpqrPlan& plan,
                        uint64_t limit_ns, cudaStream_t s);

// ---- pivoted QR of a short FP32 matrix on one thread-block cluster (cpqr_cluster.cu)
struct ClusterCpqrPlan {
    int csize = 0;
    int64_t cpb = 0;
    int threads = 0;
    int maxr = 0;
    int tpc = 0;          // threads per column
};
bool cpqr_cluster_plan(int64_t r, int64_t n, ClusterCpqrPlan* plan);
// A fixed shape (csize CTAs of cpb columns, tpc threads per column) for rows <= r.
bool cpqr_cluster_shape(int64_t r, int csize, int64_t cpb, int tpc, ClusterCpqrPlan* plan);
// One cluster per listed task: cluster c factors tasks[order[c]] from its sketch partial sums.
cudaError_t launch_cpqr_cluster_batched(const BatchTask* tasks, const int32_t* order, int ntasks,
                                        const float* partial, double* R_base, uint8_t* sel_base,
                                        int32_t* J_base, int32_t* k_out_base, int32_t* infos,
                                        const BatchTotals& tot, const ClusterCpqrPlan& plan,
                                        uint64_t limit_ns, cudaStream_t s);
// Y: r x n (ldy), or the sum of kslabs such arrays slab_stride floats apart (the
// sketch's split-K partial sums, added in slab order while loading).
cudaError_t launch_cpqr_cluster(const float* Y, int64_t r, int64_t n, int64_t ldy, int kslabs, int64_t slab_stride,
                                int kcap, double rel_tol, int32_t* J, int32_t* k_out, int32_t* info, double* R64,
                                int64_t ldr, uint8_t* sel, const ClusterCpqrPlan& plan, uint64_t limit_ns,
                                cudaStream_t s);

// ---- coefficient solve and error estimate (trsm.cu)
cudaError_t launch_solve_T(const double* R64, int64_t ldr, const int32_t* J, const int32_t* k_ptr,
                           int kcap, int64_t n, double* T, int64_t ldt, double* scratch,
                           int refine_steps, int low_solve, cudaStream_t s);
size_t solve_T_scratch_doubles(int kcap, int64_t n);
// Batched mixed-precision solve (FP32 solves, FP64 residual): one CTA of `warps` warps
// per unit; kmax bounds the ranks of the listed tasks (<= 128).
cudaError_t launch_solve_T_batched(const BatchTask* tasks, const SolveUnit* units, int nunits, int kmax,
                                   int warps, const double* R_base, const int32_t* J_base,
                                   const int32_t* k_out, int32_t* infos, double* T_base,
                                   const BatchTotals& tot, int refine_steps, cudaStream_t s);
// The batch's solve as products (one refinement step, ranks <= 128): the inverses of every
// task's R11 (kmax bounds all ranks of the batch), then the listed units (kmax bounds theirs).
// inv: the workspace's inverse region, batch_inverse_floats(kcap) floats per task.
size_t batch_inverse_floats(int kcap);
cudaError_t launch_r11_inverse_batched(const BatchTask* tasks, int ntasks, int kmax, const double* R_base,
                                       const int32_t* J_base, const int32_t* k_out, const BatchTotals& tot, float* inv,
                                       cudaStream_t s);
cudaError_t launch_solve_T_batched_product(const BatchTask* tasks, const SolveUnit* units, int nunits, int kmax,
                                           const double* R_base, const int32_t* J_base, const int32_t* k_out,
                                           int32_t* infos, double* T_base, const BatchTotals& tot, int refine_steps,
                                           const float* inv, cudaStream_t s);
cudaError_t launch_reconstruct_one(const void* A, int a_f64, int64_t m, int64_t n, int64_t lda, const int32_t* J,
                                   int k, const double* T, int64_t ldt, void* Ahat, int64_t ldh, cudaStream_t s);
// ||A - A(:,J) P||_F / ||A||_F into err_out (acc2: 4 doubles of scratch).  FP32 A: the
// products in exact float pairs, with T split into FP32 parts in tsplit (2 kcap (n - 1) floats,
// free space such as the solve's scratch once the solve has run); FP64 A: DFMA (tsplit unused).
cudaError_t launch_residual_fro(const void* A, int a_f64, int64_t m, int64_t n, int64_t lda,
                                const int32_t* J, const int32_t* k_ptr, const double* T,
                                int64_t ldt, int kcap, double* acc2, double* err_out, float* tsplit,
                                cudaStream_t s);

// ---- transpose and column gather (transform.cu)
cudaError_t launch_transpose(const void* A, int f64, int64_t m, int64_t n, int64_t lda, void* B, int64_t ldb,
                             cudaStream_t s);
cudaError_t launch_gather_cols(const void* A, int f64, int64_t m, int64_t lda, const int32_t* J, int k, void* C,
                               int64_t ldc, cudaStream_t s);

// ---- adjoint and reconstruction (backward.cu)
size_t backward_workspace_bytes(int64_t batch, int64_t m, int64_t n, int k);
size_t reconstruct_workspace_bytes(int64_t batch, int64_t n, int k);
cudaError_t launch_backward(int64_t batch, const float* A, int64_t m, int64_t n, int64_t lda, int64_t strideA,
                            const int32_t* J, int64_t strideJ, int k, const double* T, int64_t ldt, int64_t strideT,
                            const float* G, int64_t ldg, int64_t strideG, const double* Tb, int64_t ldtb,
                            int64_t strideTb, float* dA, int64_t ldd, int64_t strideD, void* work, cudaStream_t s);
cudaError_t launch_reconstruct(int64_t batch, const float* A, int64_t m, int64_t n, int64_t lda, int64_t strideA,
                               const int32_t* J, int64_t strideJ, int k, const double* T, int64_t ldt, int64_t strideT,
                               float* Ahat, int64_t ldh, int64_t strideH, void* work, cudaStream_t s);

}  // namespace gid
