// Truncated column-pivoted Householder QR of a short FP32 matrix on one thread-block
// cluster (Sec. 1.1 / Algorithm 1, its pivoted QR, applied to the sketch Y of the mixed path).
//
// The sketch Y has ell <= 160 rows, so a column fits in the registers of a few
// threads: TPC threads own one column, each a contiguous block of MAXR / TPC
// rows.  The n columns are split over the C CTAs of a cluster (up to 16).
//
// Every pivot step needs one global argmax.  Each warp stages its best candidate's
// current column in shared memory; after one CTA barrier the CTA's best record (norm,
// index, sum of norms, exact squared norm, then the column) goes into every peer's shared
// memory by 16-byte st.async stores, completing on the peer's mbarrier in bytes.  Each
// CTA waits (bounded) on its own mbarrier, reduces the C records in the same order, and
// so all CTAs agree on the pivot and hold its column locally: one exchange per step, no
// grid barrier and no memory fences.
//
// Per step each column forms w = v^T x(j:r) with the reflector
// v = x_p / (alpha - beta) (v_j = 1), applies x -= tau w v, records
// R(j, i) = x_j, and downdates its squared norm with the Drmac-Bujanovic
// recompute test.  With S = x_p(j:r)^T x(j:r) - beta x_j the reflector's
// coefficient is tau w = -S / beta, so a step needs the two reciprocals 1 / beta
// and 1 / (alpha - beta) and no division.
#include "common.cuh"
#include "internal.h"

#include <algorithm>

namespace gid {

constexpr int kCqMaxCluster = 16;
constexpr int kCqMaxThreads = 512;
constexpr int kCqMaxRows = 160;

struct CqParams {
    const float* Y;
    int64_t r, n, ldy;
    int kcap;
    double rel_tol;
    int32_t* J;
    int32_t* k_out;
    int32_t* info;
    double* R;
    int64_t ldr;
    uint8_t* sel;
    int64_t cpb;          // columns per CTA
    uint64_t limit_ns;
    int kslabs;           // Y given as kslabs split-K partial sums, slab_stride apart (1: Y itself)
    int64_t slab_stride;
    // batch mode (tasks != nullptr): cluster c factors task order[c]; Y is the sketch's
    // split-K partial sums, added in slab order while loading
    const BatchTask* tasks;
    const int32_t* order;
    const float* partial;
    double* R_base;
    uint8_t* sel_base;
    int32_t* J_base;
    int32_t* k_out_base;
    int32_t* infos;
    int64_t ntasks, partial_total, r_total, j_total, sel_total;
};

// The matrix one cluster factors.
struct CqTask {
    const float* Y;
    int64_t r, n, ldy, slab_stride;
    int kslabs, kcap;
    double rel_tol;
    int32_t* J;
    int32_t* k_out;
    int32_t* info;
    double* R;
    int64_t ldr;
    uint8_t* sel;
    bool ok;              // the task fits its regions and this launch's shape
};

template <int MAXR>
__device__ __forceinline__ CqTask cq_task(const CqParams& P, uint32_t C) {
    CqTask W;
    W.ok = true;
    if (!P.tasks) {
        W.Y = P.Y; W.r = P.r; W.n = P.n; W.ldy = P.ldy; W.slab_stride = P.slab_stride;
        W.kslabs = P.kslabs > 0 ? P.kslabs : 1;
        W.kcap = P.kcap; W.rel_tol = P.rel_tol; W.J = P.J; W.k_out = P.k_out; W.info = P.info;
        W.R = P.R; W.ldr = P.ldr; W.sel = P.sel;
        return W;
    }
    const int task = P.order[blockIdx.x / C];
    W.ok = task >= 0 && task < P.ntasks;
    const BatchTask& bt = P.tasks[W.ok ? task : 0];
    W.Y = P.partial + bt.partial_off; W.r = bt.ell; W.n = bt.n; W.ldy = bt.lp;
    W.slab_stride = bt.n * bt.lp; W.kslabs = bt.kslabs;
    W.kcap = bt.kcap; W.rel_tol = bt.rel_tol; W.J = P.J_base + bt.j_off; W.k_out = P.k_out_base + task;
    W.info = P.infos + task; W.R = P.R_base + bt.r_off; W.ldr = bt.kcap; W.sel = P.sel_base + bt.sel_off;
    W.ok = W.ok && bt.ell >= 1 && bt.ell <= MAXR && bt.ell <= bt.lp && bt.n >= 1 && bt.n <= C * P.cpb &&
           bt.kcap >= 1 && bt.kcap <= bt.ell && bt.kcap <= bt.n && bt.kslabs >= 1 && bt.partial_off >= 0 &&
           bt.partial_off + static_cast<int64_t>(bt.kslabs) * bt.n * bt.lp <= P.partial_total &&
           bt.r_off >= 0 && bt.r_off + static_cast<int64_t>(bt.kcap) * bt.n <= P.r_total && bt.j_off >= 0 &&
           bt.j_off + bt.n <= P.j_total && bt.sel_off >= 0 && bt.sel_off + bt.n <= P.sel_total;
    return W;
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t cluster_nrank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t map_peer(uint32_t local_addr, uint32_t rank) {
    uint32_t out;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(local_addr), "r"(rank));
    return out;
}

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Candidate key: larger residual norm first, ties to the smaller column index.  Norms
// are non-negative, so their float bits order like the values; 0 means "none".
__device__ __forceinline__ uint64_t cand_key(float nu, int64_t i) {
    return (static_cast<uint64_t>(__float_as_uint(nu)) << 32) | static_cast<uint32_t>(0x7FFFFFFF - static_cast<int>(i));
}
__device__ __forceinline__ int key_index(uint64_t key) {
    return key ? 0x7FFFFFFF - static_cast<int>(static_cast<uint32_t>(key)) : -1;
}
__device__ __forceinline__ float key_norm(uint64_t key) { return __uint_as_float(static_cast<uint32_t>(key >> 32)); }

// Warp maximum of candidate keys with two 32-bit warp reductions (norm bits, then the
// index word among the lanes holding the largest norm).
__device__ __forceinline__ uint64_t warp_max_key(uint64_t key) {
    const uint32_t kh = static_cast<uint32_t>(key >> 32);
    const uint32_t hi = __reduce_max_sync(0xffffffffu, kh);
    const uint32_t lo = __reduce_max_sync(0xffffffffu, kh == hi ? static_cast<uint32_t>(key) : 0u);
    return (static_cast<uint64_t>(hi) << 32) | lo;
}

// 16 bytes from registers into a peer CTA's shared memory, counted in bytes on the
// peer's mbarrier.
__device__ __forceinline__ void st_async_peer(uint32_t dst_cluster, float4 v, uint32_t bar_cluster) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                     dst_cluster),
                 "r"(__float_as_uint(v.x)), "r"(__float_as_uint(v.y)), "r"(__float_as_uint(v.z)),
                 "r"(__float_as_uint(v.w)), "r"(bar_cluster)
                 : "memory");
}

// End of a pivot step for a warp-uniform register index u (a uniform switch, no local
// memory): x[u] = 0 where `own` holds (the step's row leaves the column), and x[(u + 1) % RPT]
// is returned (the next step's row, held by this thread or by the next one of the group).
template <int RPT>
__device__ __forceinline__ float zero_and_next(float (&x)[RPT], int u, bool own) {
    switch (u) {
        case 0: if constexpr (RPT > 0) { x[0] = own ? 0.f : x[0]; return x[(0 + 1) % RPT]; } return 0.f;
        case 1: if constexpr (RPT > 1) { x[1] = own ? 0.f : x[1]; return x[(1 + 1) % RPT]; } return 0.f;
        case 2: if constexpr (RPT > 2) { x[2] = own ? 0.f : x[2]; return x[(2 + 1) % RPT]; } return 0.f;
        case 3: if constexpr (RPT > 3) { x[3] = own ? 0.f : x[3]; return x[(3 + 1) % RPT]; } return 0.f;
        case 4: if constexpr (RPT > 4) { x[4] = own ? 0.f : x[4]; return x[(4 + 1) % RPT]; } return 0.f;
        case 5: if constexpr (RPT > 5) { x[5] = own ? 0.f : x[5]; return x[(5 + 1) % RPT]; } return 0.f;
        case 6: if constexpr (RPT > 6) { x[6] = own ? 0.f : x[6]; return x[(6 + 1) % RPT]; } return 0.f;
        case 7: if constexpr (RPT > 7) { x[7] = own ? 0.f : x[7]; return x[(7 + 1) % RPT]; } return 0.f;
        case 8: if constexpr (RPT > 8) { x[8] = own ? 0.f : x[8]; return x[(8 + 1) % RPT]; } return 0.f;
        case 9: if constexpr (RPT > 9) { x[9] = own ? 0.f : x[9]; return x[(9 + 1) % RPT]; } return 0.f;
        case 10: if constexpr (RPT > 10) { x[10] = own ? 0.f : x[10]; return x[(10 + 1) % RPT]; } return 0.f;
        case 11: if constexpr (RPT > 11) { x[11] = own ? 0.f : x[11]; return x[(11 + 1) % RPT]; } return 0.f;
        case 12: if constexpr (RPT > 12) { x[12] = own ? 0.f : x[12]; return x[(12 + 1) % RPT]; } return 0.f;
        case 13: if constexpr (RPT > 13) { x[13] = own ? 0.f : x[13]; return x[(13 + 1) % RPT]; } return 0.f;
        case 14: if constexpr (RPT > 14) { x[14] = own ? 0.f : x[14]; return x[(14 + 1) % RPT]; } return 0.f;
        case 15: if constexpr (RPT > 15) { x[15] = own ? 0.f : x[15]; return x[(15 + 1) % RPT]; } return 0.f;
        case 16: if constexpr (RPT > 16) { x[16] = own ? 0.f : x[16]; return x[(16 + 1) % RPT]; } return 0.f;
        case 17: if constexpr (RPT > 17) { x[17] = own ? 0.f : x[17]; return x[(17 + 1) % RPT]; } return 0.f;
        case 18: if constexpr (RPT > 18) { x[18] = own ? 0.f : x[18]; return x[(18 + 1) % RPT]; } return 0.f;
        case 19: if constexpr (RPT > 19) { x[19] = own ? 0.f : x[19]; return x[(19 + 1) % RPT]; } return 0.f;
        case 20: if constexpr (RPT > 20) { x[20] = own ? 0.f : x[20]; return x[(20 + 1) % RPT]; } return 0.f;
        case 21: if constexpr (RPT > 21) { x[21] = own ? 0.f : x[21]; return x[(21 + 1) % RPT]; } return 0.f;
        case 22: if constexpr (RPT > 22) { x[22] = own ? 0.f : x[22]; return x[(22 + 1) % RPT]; } return 0.f;
        case 23: if constexpr (RPT > 23) { x[23] = own ? 0.f : x[23]; return x[(23 + 1) % RPT]; } return 0.f;
        case 24: if constexpr (RPT > 24) { x[24] = own ? 0.f : x[24]; return x[(24 + 1) % RPT]; } return 0.f;
        case 25: if constexpr (RPT > 25) { x[25] = own ? 0.f : x[25]; return x[(25 + 1) % RPT]; } return 0.f;
        case 26: if constexpr (RPT > 26) { x[26] = own ? 0.f : x[26]; return x[(26 + 1) % RPT]; } return 0.f;
        case 27: if constexpr (RPT > 27) { x[27] = own ? 0.f : x[27]; return x[(27 + 1) % RPT]; } return 0.f;
        case 28: if constexpr (RPT > 28) { x[28] = own ? 0.f : x[28]; return x[(28 + 1) % RPT]; } return 0.f;
        case 29: if constexpr (RPT > 29) { x[29] = own ? 0.f : x[29]; return x[(29 + 1) % RPT]; } return 0.f;
        case 30: if constexpr (RPT > 30) { x[30] = own ? 0.f : x[30]; return x[(30 + 1) % RPT]; } return 0.f;
        case 31: if constexpr (RPT > 31) { x[31] = own ? 0.f : x[31]; return x[(31 + 1) % RPT]; } return 0.f;
        case 32: if constexpr (RPT > 32) { x[32] = own ? 0.f : x[32]; return x[(32 + 1) % RPT]; } return 0.f;
        case 33: if constexpr (RPT > 33) { x[33] = own ? 0.f : x[33]; return x[(33 + 1) % RPT]; } return 0.f;
        case 34: if constexpr (RPT > 34) { x[34] = own ? 0.f : x[34]; return x[(34 + 1) % RPT]; } return 0.f;
        case 35: if constexpr (RPT > 35) { x[35] = own ? 0.f : x[35]; return x[(35 + 1) % RPT]; } return 0.f;
        case 36: if constexpr (RPT > 36) { x[36] = own ? 0.f : x[36]; return x[(36 + 1) % RPT]; } return 0.f;
        case 37: if constexpr (RPT > 37) { x[37] = own ? 0.f : x[37]; return x[(37 + 1) % RPT]; } return 0.f;
        case 38: if constexpr (RPT > 38) { x[38] = own ? 0.f : x[38]; return x[(38 + 1) % RPT]; } return 0.f;
        case 39: if constexpr (RPT > 39) { x[39] = own ? 0.f : x[39]; return x[(39 + 1) % RPT]; } return 0.f;
        case 40: if constexpr (RPT > 40) { x[40] = own ? 0.f : x[40]; return x[(40 + 1) % RPT]; } return 0.f;
        case 41: if constexpr (RPT > 41) { x[41] = own ? 0.f : x[41]; return x[(41 + 1) % RPT]; } return 0.f;
        case 42: if constexpr (RPT > 42) { x[42] = own ? 0.f : x[42]; return x[(42 + 1) % RPT]; } return 0.f;
        case 43: if constexpr (RPT > 43) { x[43] = own ? 0.f : x[43]; return x[(43 + 1) % RPT]; } return 0.f;
        case 44: if constexpr (RPT > 44) { x[44] = own ? 0.f : x[44]; return x[(44 + 1) % RPT]; } return 0.f;
        case 45: if constexpr (RPT > 45) { x[45] = own ? 0.f : x[45]; return x[(45 + 1) % RPT]; } return 0.f;
        case 46: if constexpr (RPT > 46) { x[46] = own ? 0.f : x[46]; return x[(46 + 1) % RPT]; } return 0.f;
        case 47: if constexpr (RPT > 47) { x[47] = own ? 0.f : x[47]; return x[(47 + 1) % RPT]; } return 0.f;
        case 48: if constexpr (RPT > 48) { x[48] = own ? 0.f : x[48]; return x[(48 + 1) % RPT]; } return 0.f;
        case 49: if constexpr (RPT > 49) { x[49] = own ? 0.f : x[49]; return x[(49 + 1) % RPT]; } return 0.f;
        case 50: if constexpr (RPT > 50) { x[50] = own ? 0.f : x[50]; return x[(50 + 1) % RPT]; } return 0.f;
        case 51: if constexpr (RPT > 51) { x[51] = own ? 0.f : x[51]; return x[(51 + 1) % RPT]; } return 0.f;
        case 52: if constexpr (RPT > 52) { x[52] = own ? 0.f : x[52]; return x[(52 + 1) % RPT]; } return 0.f;
        case 53: if constexpr (RPT > 53) { x[53] = own ? 0.f : x[53]; return x[(53 + 1) % RPT]; } return 0.f;
        case 54: if constexpr (RPT > 54) { x[54] = own ? 0.f : x[54]; return x[(54 + 1) % RPT]; } return 0.f;
        case 55: if constexpr (RPT > 55) { x[55] = own ? 0.f : x[55]; return x[(55 + 1) % RPT]; } return 0.f;
        case 56: if constexpr (RPT > 56) { x[56] = own ? 0.f : x[56]; return x[(56 + 1) % RPT]; } return 0.f;
        case 57: if constexpr (RPT > 57) { x[57] = own ? 0.f : x[57]; return x[(57 + 1) % RPT]; } return 0.f;
        case 58: if constexpr (RPT > 58) { x[58] = own ? 0.f : x[58]; return x[(58 + 1) % RPT]; } return 0.f;
        case 59: if constexpr (RPT > 59) { x[59] = own ? 0.f : x[59]; return x[(59 + 1) % RPT]; } return 0.f;
        case 60: if constexpr (RPT > 60) { x[60] = own ? 0.f : x[60]; return x[(60 + 1) % RPT]; } return 0.f;
        case 61: if constexpr (RPT > 61) { x[61] = own ? 0.f : x[61]; return x[(61 + 1) % RPT]; } return 0.f;
        case 62: if constexpr (RPT > 62) { x[62] = own ? 0.f : x[62]; return x[(62 + 1) % RPT]; } return 0.f;
        case 63: if constexpr (RPT > 63) { x[63] = own ? 0.f : x[63]; return x[(63 + 1) % RPT]; } return 0.f;
        case 64: if constexpr (RPT > 64) { x[64] = own ? 0.f : x[64]; return x[(64 + 1) % RPT]; } return 0.f;
        case 65: if constexpr (RPT > 65) { x[65] = own ? 0.f : x[65]; return x[(65 + 1) % RPT]; } return 0.f;
        case 66: if constexpr (RPT > 66) { x[66] = own ? 0.f : x[66]; return x[(66 + 1) % RPT]; } return 0.f;
        case 67: if constexpr (RPT > 67) { x[67] = own ? 0.f : x[67]; return x[(67 + 1) % RPT]; } return 0.f;
        case 68: if constexpr (RPT > 68) { x[68] = own ? 0.f : x[68]; return x[(68 + 1) % RPT]; } return 0.f;
        case 69: if constexpr (RPT > 69) { x[69] = own ? 0.f : x[69]; return x[(69 + 1) % RPT]; } return 0.f;
        case 70: if constexpr (RPT > 70) { x[70] = own ? 0.f : x[70]; return x[(70 + 1) % RPT]; } return 0.f;
        case 71: if constexpr (RPT > 71) { x[71] = own ? 0.f : x[71]; return x[(71 + 1) % RPT]; } return 0.f;
        case 72: if constexpr (RPT > 72) { x[72] = own ? 0.f : x[72]; return x[(72 + 1) % RPT]; } return 0.f;
        case 73: if constexpr (RPT > 73) { x[73] = own ? 0.f : x[73]; return x[(73 + 1) % RPT]; } return 0.f;
        case 74: if constexpr (RPT > 74) { x[74] = own ? 0.f : x[74]; return x[(74 + 1) % RPT]; } return 0.f;
        case 75: if constexpr (RPT > 75) { x[75] = own ? 0.f : x[75]; return x[(75 + 1) % RPT]; } return 0.f;
        case 76: if constexpr (RPT > 76) { x[76] = own ? 0.f : x[76]; return x[(76 + 1) % RPT]; } return 0.f;
        case 77: if constexpr (RPT > 77) { x[77] = own ? 0.f : x[77]; return x[(77 + 1) % RPT]; } return 0.f;
        case 78: if constexpr (RPT > 78) { x[78] = own ? 0.f : x[78]; return x[(78 + 1) % RPT]; } return 0.f;
        case 79: if constexpr (RPT > 79) { x[79] = own ? 0.f : x[79]; return x[(79 + 1) % RPT]; } return 0.f;
        default: return 0.f;
    }
}

// Shared-memory index of row r of a column record, padded by 16 bytes every 32 rows
// so that the TPC row blocks of a column read from different banks.
__device__ __forceinline__ int vidx(int r) { return r + ((r >> 5) << 2); }

template <int MAXR>
struct CqRecord {
    float4 head;                       // (residual norm, index bits, sum of norms, exact ||x||^2)
    float col[MAXR + MAXR / 8];        // the candidate column, padded rows (vidx)
};

// Short columns (MAXR <= 64, TPC = 4: 16 rows per thread) fit 64 registers, so two
// CTAs share an SM; that doubles the clusters a batch keeps in flight.
template <int MAXR, int TPC>
__global__ void __launch_bounds__(kCqMaxThreads, (MAXR <= 64 && TPC == 4) ? 2 : 1) k_cpqr_cluster(const CqParams P) {
    constexpr int RPT = MAXR / TPC;
    constexpr int MAXW = kCqMaxThreads / 32;
    constexpr uint32_t REC = sizeof(CqRecord<MAXR>);
    constexpr int NCH = REC / 16;                       // 16-byte chunks of a record
    static_assert(REC % 16 == 0, "record size");
    static_assert(RPT % 4 == 0 && RPT <= 80, "rows per thread");
    __shared__ __align__(128) CqRecord<MAXR> recv[2][kCqMaxCluster];
    __shared__ __align__(128) CqRecord<MAXR> wstg[2][MAXW];   // per-warp staged candidate
    __shared__ unsigned long long cta_key[3];   // the CTA's best key of an exchange (atomic maximum)
    __shared__ float wsum[MAXW];
    __shared__ float wnorm[MAXW];
    __shared__ __align__(8) uint64_t recv_bar[2];
    __shared__ int wait_abort;                  // a thread whose exchange wait timed out sets it

    const uint32_t me = cluster_rank(), C = cluster_nrank();
    const CqTask W = cq_task<MAXR>(P, C);
    if (!W.ok) {
        // every CTA of the cluster reads the same entry and leaves before any cluster barrier
        if (me == 0 && threadIdx.x == 0 && P.order[blockIdx.x / C] >= 0 && P.order[blockIdx.x / C] < P.ntasks)
            set_info(W.info, kInfoBadTable);
        return;
    }
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
    const int cl = t / TPC, qq = t % TPC;
    const int gbase = lane & ~(TPC - 1);     // first lane of this column's thread group
    const unsigned gmask = ((1u << TPC) - 1u) << gbase;
    const int64_t i = static_cast<int64_t>(me) * P.cpb + cl;
    const bool valid = cl < P.cpb && i < W.n;
    const int r = static_cast<int>(W.r);
    const int rb = qq * RPT;                 // first row of this thread's block
    const float sqrt_u = 2.44140625e-04f;    // sqrt of the FP32 unit round-off 2^-24
    const bool need_sum = W.rel_tol > 0.0;
    const float rtol = static_cast<float>(W.rel_tol);   // converted once, off the FP64 pipe's per-step path

    if (t == 0) {
        mbar_init(&recv_bar[0], 1);
        mbar_init(&recv_bar[1], 1);
        cta_key[0] = cta_key[1] = cta_key[2] = 0ull;
        wait_abort = 0;
        fence_barrier_init();
    }
    cluster_sync_all();

    // x: this thread's rows of its column.  Rows of earlier pivot steps are set to zero
    // once their R entry is out, so dot products and norms need no row masks.
    float x[RPT];
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
        float s = 0.f;
        if (valid && rb + u < r)
            for (int ks = 0; ks < W.kslabs; ++ks) s += W.Y[ks * W.slab_stride + i * W.ldy + rb + u];
        x[u] = s;
    }
    float nu = 0.f;
#pragma unroll
    for (int u = 0; u < RPT; ++u) nu = fmaf(x[u], x[u], nu);
#pragma unroll
    for (int o = 1; o < TPC; o <<= 1) nu += __shfl_xor_sync(0xffffffffu, nu, o);
    float nuref = nu;
    float xnext = x[0];       // this thread's candidate for the next step's row (row 0: thread 0)
    bool selected = !valid;
    if (valid && qq == 0) {
        if (!isfinite(nu)) set_info(W.info, kInfoNonFinite);
        W.sel[i] = 0;
    }

    // Exchange q: each warp finds its best candidate, whose threads stage the column and
    // its exact squared norm; after one CTA barrier every warp finds the CTA's best, and
    // warp w writes that record into peers w, w + nw, ... with st.async, completing on
    // the peer's mbarrier in bytes.  Exchange q fills recv[q & 1] and completes phase
    // q >> 1 of recv_bar[q & 1]; a peer can be at most one exchange ahead, so two
    // alternating buffers and barriers never mix phases.
    // warp-level best candidate of this warp's columns, and the warp's sum of norms
    auto warp_best = [&](int q, uint64_t& key, float& part) {
        key = warp_max_key((!selected && qq == 0) ? cand_key(nu, i) : 0ull);
        part = (!selected && qq == 0) ? nu : 0.f;
        if (need_sum || q == 0) part = warp_sum(part);
    };
    // Stage the warp candidates, find the CTA's best and send it to the peers.  The CTA's
    // best key of exchange q is the atomic maximum of the warps' keys in cta_key[q % 3];
    // the slot of exchange q + 1 is cleared before this exchange's barrier (its last
    // reads, of exchange q - 2, were before the previous barrier).
    int kslot = 0;
    auto send_best = [&](int q, uint64_t key, float part) {
        const int slot = q & 1;
        const int knext = kslot == 2 ? 0 : kslot + 1;
        if (key != 0ull && i == key_index(key)) {
            // the TPC threads of the warp's candidate column
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
            for (int u = 0; u < RPT; u += 4) {
                s0 = fmaf(x[u], x[u], s0);
                s1 = fmaf(x[u + 1], x[u + 1], s1);
                s2 = fmaf(x[u + 2], x[u + 2], s2);
                s3 = fmaf(x[u + 3], x[u + 3], s3);
            }
            float s = (s0 + s1) + (s2 + s3);
#pragma unroll
            for (int o = 1; o < TPC; o <<= 1) s += __shfl_xor_sync(gmask, s, o);
#pragma unroll
            for (int u = 0; u < RPT; u += 4)
                *reinterpret_cast<float4*>(&wstg[slot][warp].col[vidx(rb + u)]) =
                    make_float4(x[u], x[u + 1], x[u + 2], x[u + 3]);
            if (qq == 0) wnorm[warp] = s;
        }
        if (lane == 0) {
            if (key != 0ull) atomicMax(&cta_key[kslot], static_cast<unsigned long long>(key));
            wsum[warp] = part;
        }
        if (t == 0) cta_key[knext] = 0ull;
        __syncthreads();
        const uint64_t ck = cta_key[kslot];
        kslot = knext;
        float cs = 0.f;
        if (need_sum || q == 0) cs = warp_sum(lane < nw ? wsum[lane] : 0.f);
        // the warp holding the CTA's best column
        const int wsrc = ck != 0ull ? static_cast<int>((key_index(ck) - static_cast<int64_t>(me) * P.cpb) * TPC / 32) : 0;
        if (t == 0) mbar_arrive_expect_tx(&recv_bar[slot], C * REC);
        const float4 head = make_float4(key_norm(ck), __int_as_float(key_index(ck)), cs, wnorm[wsrc]);
        const float* src = wstg[slot][wsrc].col;
        for (uint32_t d = warp; d < C; d += nw) {
            const uint32_t dst = map_peer(smem_addr(&recv[slot][me]), d);
            const uint32_t bar = map_peer(smem_addr(&recv_bar[slot]), d);
            for (int c = lane; c < NCH; c += 32) {
                const float4 v = c == 0 ? head : *reinterpret_cast<const float4*>(src + 4 * (c - 1));
                st_async_peer(dst + 16u * c, v, bar);
            }
        }
    };
    auto wait_exchange = [&](int q) -> bool {
        return mbar_wait(&recv_bar[q & 1], static_cast<uint32_t>((q >> 1) & 1), &wait_abort, P.limit_ns);
    };

    {
        uint64_t key0;
        float part0;
        warp_best(0, key0, part0);
        send_best(0, key0, part0);
    }
    bool ok = wait_exchange(0);
    int k = 0;
    float total = -1.f;
    for (int j = 0; ok && j < W.kcap; ++j) {
        const int par = j & 1;
        // ---- the pivot: every warp reduces the C records in the same order
        uint64_t hk = 0ull;
        float hs = 0.f;
        if (lane < static_cast<int>(C)) {
            const float4 h = recv[par][lane].head;
            const int hi = __float_as_int(h.y);
            hk = hi >= 0 ? cand_key(h.x, hi) : 0ull;
            hs = h.z;
        }
        const uint64_t best = warp_max_key(hk);
        if (need_sum || j == 0) hs = warp_sum(hs);
        const unsigned hit = __ballot_sync(0xffffffffu, lane < static_cast<int>(C) && hk == best && best != 0ull);
        const int hsrc = hit ? __ffs(hit) - 1 : 0;
        const int p = key_index(best);
        const float hv = best ? key_norm(best) : -1.f;
        if (total < 0.f) total = hs;
        if (need_sum && sqrtf(fmaxf(hs, 0.f)) <= rtol * sqrtf(total)) break;
        if (p < 0 || !(hv > 0.f)) {
            if (me == 0 && t == 0) set_info(W.info, j + 1);
            break;
        }
        const float* pc = recv[par][hsrc].col;
        const float s2 = recv[par][hsrc].head.w;
        const float alpha = pc[vidx(j)];
        const float snorm = sqrtf(s2);
        const float beta = alpha >= 0.f ? -snorm : snorm;
        const float rbeta = __frcp_rn(beta);          // tau / (alpha - beta) = -1 / beta
        const float inv = __frcp_rn(alpha - beta);
        // S = v'.x with v' = (0 above j, alpha - beta at j, pivot column below):
        // pc.x - beta x_j, rows above j being zero in both
        float S0 = 0.f, S1 = 0.f, S2 = 0.f, S3 = 0.f;
#pragma unroll
        for (int u = 0; u < RPT; u += 4) {
            const float4 v4 = *reinterpret_cast<const float4*>(&pc[vidx(rb + u)]);
            S0 = fmaf(v4.x, x[u], S0);
            S1 = fmaf(v4.y, x[u + 1], S1);
            S2 = fmaf(v4.z, x[u + 2], S2);
            S3 = fmaf(v4.w, x[u + 3], S3);
        }
        float S = (S0 + S1) + (S2 + S3);
#pragma unroll
        for (int o = 1; o < TPC; o <<= 1) S += __shfl_xor_sync(0xffffffffu, S, o);
        // X = x_j: thread qj of the group picked it (register uj) at the end of the last step
        const int qj = j / RPT, uj = j - qj * RPT;
        const float X = __shfl_sync(0xffffffffu, xnext, gbase + qj);
        S = fmaf(-beta, X, S);
        if (valid && i == p) {
            selected = true;
            if (qq == 0) {
                W.R[i * W.ldr + j] = f64_of_f32(beta);
                W.J[j] = p;
                W.sel[i] = 1;
            }
        }
        const float tw = -S * rbeta;                        // tau w
        const float sv = selected ? 0.f : tw * inv;         // the pivot column itself stays
        const float rho = X - tw;
        if (!selected && qq == 0) W.R[i * W.ldr + j] = f64_of_f32(rho);
        // norm downdate nu - rho^2 = nu (1 - (rho / sqrt(nu))^2); an exact recompute where
        // cancellation has left at most sqrt(u) of the reference norm
        bool recompute = false;
        if (!selected && nu > 0.f) {
            const float d = fmaxf(fmaf(-rho, rho, nu), 0.f);
            if (d <= sqrt_u * nuref) recompute = true;           // same decision in all TPC threads
            else nu = d;
        }
        uint64_t key;
        float part;
        if (__any_sync(0xffffffffu, recompute)) {
            // x -= (tau w / (alpha - beta)) v'; row j leaves as rho and is then zeroed
#pragma unroll
            for (int u = 0; u < RPT; u += 4) {
                const float4 v4 = *reinterpret_cast<const float4*>(&pc[vidx(rb + u)]);
                x[u] = fmaf(-sv, v4.x, x[u]);
                x[u + 1] = fmaf(-sv, v4.y, x[u + 1]);
                x[u + 2] = fmaf(-sv, v4.z, x[u + 2]);
                x[u + 3] = fmaf(-sv, v4.w, x[u + 3]);
            }
            xnext = zero_and_next<RPT>(x, uj, qq == qj);
            float sq = 0.f;
#pragma unroll
            for (int u = 0; u < RPT; ++u) sq = fmaf(x[u], x[u], sq);
#pragma unroll
            for (int o = 1; o < TPC; o <<= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
            if (recompute) {
                nu = sq;
                nuref = sq;
            }
            warp_best(j + 1, key, part);
        } else {
            // the next candidate search does not depend on x: its shuffles overlap the update
            warp_best(j + 1, key, part);
#pragma unroll
            for (int u = 0; u < RPT; u += 4) {
                const float4 v4 = *reinterpret_cast<const float4*>(&pc[vidx(rb + u)]);
                x[u] = fmaf(-sv, v4.x, x[u]);
                x[u + 1] = fmaf(-sv, v4.y, x[u + 1]);
                x[u + 2] = fmaf(-sv, v4.z, x[u + 2]);
                x[u + 3] = fmaf(-sv, v4.w, x[u + 3]);
            }
            xnext = zero_and_next<RPT>(x, uj, qq == qj);
        }
        send_best(j + 1, key, part);
        ok = wait_exchange(j + 1);
        k = j + 1;
    }
    if (!ok && t == 0) set_info(W.info, kInfoWatchdog);
    // no CTA leaves while a peer may still write into its shared memory
    cluster_sync_all();
    if (me == 0) {
        if (t == 0) *W.k_out = k;
        __shared__ int s_base;
        __shared__ int cnt[MAXW];
        if (t == 0) s_base = k;
        __syncthreads();
        for (int64_t i0 = 0; i0 < W.n; i0 += blockDim.x) {
            const int64_t c = i0 + t;
            const int flag = (c < W.n && !__ldcg(W.sel + c)) ? 1 : 0;
            const unsigned bal = __ballot_sync(0xffffffffu, flag);
            const int wpre = __popc(bal & ((1u << lane) - 1u));
            if (lane == 0) cnt[warp] = __popc(bal);
            __syncthreads();
            int off = 0;
            for (int w = 0; w < warp; ++w) off += cnt[w];
            if (flag) W.J[s_base + off + wpre] = static_cast<int32_t>(c);
            __syncthreads();
            if (t == 0) {
                int tot = 0;
                for (int w = 0; w < nw; ++w) tot += cnt[w];
                s_base += tot;
            }
            __syncthreads();
        }
    }
}

template <int MAXR, int TPC>
static cudaLaunchConfig_t cq_config(int csize, int nclusters, int threads, cudaStream_t s,
                                    cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(csize * nclusters);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// Can a cluster of csize CTAs of this kernel be resident at once?
template <int MAXR, int TPC>
static bool cq_cluster_fits(int csize, int threads) {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        // host-only planning (no device): the GB300 target takes 16-CTA clusters of 512 threads
        cudaGetLastError();
        return csize <= kCqMaxCluster && threads <= kCqMaxThreads;
    }
    auto kern = k_cpqr_cluster<MAXR, TPC>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cq_config<MAXR, TPC>(csize, 1, threads, nullptr, attr);
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return nclusters > 0;
}

template <int MAXR, int TPC>
static cudaError_t launch_cq(const CqParams& P, int csize, int nclusters, int threads, cudaStream_t s) {
    auto kern = k_cpqr_cluster<MAXR, TPC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cq_config<MAXR, TPC>(csize, nclusters, threads, s, attr);
    return cudaLaunchKernelEx(&cfg, kern, P);
}

template <int MAXR>
static bool cq_fits(int tpc, int csize, int threads) {
    if constexpr (MAXR > 128) {
        // two threads per column would hold 80 rows each and spill
        return tpc == 4 && cq_cluster_fits<MAXR, 4>(csize, threads);
    } else {
        return tpc == 4 ? cq_cluster_fits<MAXR, 4>(csize, threads) : cq_cluster_fits<MAXR, 2>(csize, threads);
    }
}

static int cq_maxr(int64_t r) { return r <= 32 ? 32 : (r <= 64 ? 64 : (r <= 96 ? 96 : (r <= 128 ? 128 : 160))); }

static bool cq_fits_any(int maxr, int tpc, int csize, int threads) {
    switch (maxr) {
        case 32: return cq_fits<32>(tpc, csize, threads);
        case 64: return cq_fits<64>(tpc, csize, threads);
        case 96: return cq_fits<96>(tpc, csize, threads);
        case 128: return cq_fits<128>(tpc, csize, threads);
        default: return cq_fits<160>(tpc, csize, threads);
    }
}

bool cpqr_cluster_plan(int64_t r, int64_t n, ClusterCpqrPlan* plan) {
    if (r < 1 || r > kCqMaxRows || n < 1) return false;
    const int maxr = cq_maxr(r);
    int csize = static_cast<int>(std::min<int64_t>(kCqMaxCluster, std::max<int64_t>(1, (n + 63) / 64)));
    for (; csize >= 1; csize = csize > 8 ? 8 : csize - 1) {
        const int64_t cpb = (n + csize - 1) / csize;
        int tpc = 0;
        if (cpb * 4 <= kCqMaxThreads) tpc = 4;
        else if (cpb * 2 <= kCqMaxThreads && maxr <= 128) tpc = 2;
        else return false;
        const int threads = static_cast<int>((cpb * tpc + 31) / 32 * 32);
        if (cq_fits_any(maxr, tpc, csize, threads)) {
            plan->csize = csize;
            plan->cpb = cpb;
            plan->threads = threads;
            plan->maxr = maxr;
            plan->tpc = tpc;
            return true;
        }
        if (csize == 1) break;
    }
    return false;
}

bool cpqr_cluster_shape(int64_t r, int csize, int64_t cpb, int tpc, ClusterCpqrPlan* plan) {
    if (r < 1 || r > kCqMaxRows || csize < 1 || csize > kCqMaxCluster || cpb < 1) return false;
    const int maxr = cq_maxr(r);
    if (cpb * tpc > kCqMaxThreads || (tpc != 2 && tpc != 4)) return false;
    const int threads = static_cast<int>((cpb * tpc + 31) / 32 * 32);
    if (!cq_fits_any(maxr, tpc, csize, threads)) return false;
    plan->csize = csize;
    plan->cpb = cpb;
    plan->threads = threads;
    plan->maxr = maxr;
    plan->tpc = tpc;
    return true;
}

static cudaError_t launch_cq_any(const CqParams& P, const ClusterCpqrPlan& plan, int nclusters, cudaStream_t s) {
    const int cs = plan.csize, th = plan.threads;
    if (plan.tpc == 4) {
        switch (plan.maxr) {
            case 32: return launch_cq<32, 4>(P, cs, nclusters, th, s);
            case 64: return launch_cq<64, 4>(P, cs, nclusters, th, s);
            case 96: return launch_cq<96, 4>(P, cs, nclusters, th, s);
            case 128: return launch_cq<128, 4>(P, cs, nclusters, th, s);
            default: return launch_cq<160, 4>(P, cs, nclusters, th, s);
        }
    }
    switch (plan.maxr) {
        case 32: return launch_cq<32, 2>(P, cs, nclusters, th, s);
        case 64: return launch_cq<64, 2>(P, cs, nclusters, th, s);
        case 96: return launch_cq<96, 2>(P, cs, nclusters, th, s);
        default: return launch_cq<128, 2>(P, cs, nclusters, th, s);
    }
}

cudaError_t launch_cpqr_cluster(const float* Y, int64_t r, int64_t n, int64_t ldy, int kslabs, int64_t slab_stride,
                                int kcap, double rel_tol, int32_t* J, int32_t* k_out, int32_t* info, double* R64,
                                int64_t ldr, uint8_t* sel, const ClusterCpqrPlan& plan, uint64_t limit_ns,
                                cudaStream_t s) {
    CqParams P{};
    P.Y = Y; P.r = r; P.n = n; P.ldy = ldy;
    P.kslabs = kslabs; P.slab_stride = slab_stride;
    P.kcap = kcap; P.rel_tol = rel_tol;
    P.J = J; P.k_out = k_out; P.info = info;
    P.R = R64; P.ldr = ldr; P.sel = sel;
    P.cpb = plan.cpb;
    P.limit_ns = limit_ns;
    return launch_cq_any(P, plan, 1, s);
}

cudaError_t launch_cpqr_cluster_batched(const BatchTask* tasks, const int32_t* order, int ntasks,
                                        const float* partial, double* R_base, uint8_t* sel_base, int32_t* J_base,
                                        int32_t* k_out_base, int32_t* infos, const BatchTotals& tot,
                                        const ClusterCpqrPlan& plan, uint64_t limit_ns, cudaStream_t s) {
    if (ntasks <= 0) return cudaSuccess;
    CqParams P{};
    P.cpb = plan.cpb;
    P.limit_ns = limit_ns;
    P.tasks = tasks; P.order = order; P.partial = partial; P.R_base = R_base; P.sel_base = sel_base;
    P.J_base = J_base; P.k_out_base = k_out_base; P.infos = infos;
    P.ntasks = tot.ntasks; P.partial_total = tot.partial; P.r_total = tot.r; P.j_total = tot.j; P.sel_total = tot.sel;
    return launch_cq_any(P, plan, ntasks, s);
}

}  // namespace gid
