// Truncated column-pivoted Householder QR of a short FP32 matrix on one thread-block
// cluster (Sec. 1.1 / Algorithm 1, its pivoted QR, applied to the sketch Y of the mixed path).
//
// The sketch Y has ell <= 160 rows, so a column fits in the registers of a few
// threads: TPC threads own one column, each a contiguous block of MAXR / TPC
// rows.  The n columns are split over the C CTAs of a cluster (up to 16).
//
// Every pivot step needs one global argmax.  Each CTA stages its best candidate
// (norm, index, sum of norms) and that candidate's current column in its own
// shared memory and bulk-copies the record into every peer's shared memory
// (cp.async.bulk shared::cta -> shared::cluster), completing on the peer's
// mbarrier in bytes.  Each CTA waits (bounded) on its own mbarrier, reduces the
// C records in the same order, and so all CTAs agree on the pivot and hold its
// column locally: one exchange per step, no grid barrier and no memory fences.
//
// Per step each column forms w = v^T x(j:r) with the reflector
// v = x_p / (alpha - beta) (v_j = 1), applies x -= tau w v, records
// R(j, i) = x_j, and downdates its squared norm with the Drmac-Bujanovic
// recompute test.
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
        W.Y = P.Y; W.r = P.r; W.n = P.n; W.ldy = P.ldy; W.slab_stride = 0; W.kslabs = 1;
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

// Bulk copy of `bytes` from this CTA's shared memory into a peer's shared memory,
// counted in bytes on the peer's mbarrier.
__device__ __forceinline__ void bulk_s2peer(uint32_t dst_cluster, uint32_t src_cta, uint32_t bytes,
                                            uint32_t bar_cluster) {
    asm volatile(
        "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst_cluster),
        "r"(src_cta), "r"(bytes), "r"(bar_cluster)
        : "memory");
}

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// (value, index) argmax with ties to the smaller index; -1 index marks "none".
__device__ __forceinline__ void better(float& v, int& i, float ov, int oi) {
    if (oi >= 0 && (i < 0 || ov > v || (ov == v && oi < i))) { v = ov; i = oi; }
}

template <int MAXR>
struct CqRecord {
    float4 head;          // (best norm, index bits, sum of norms, unused)
    float col[MAXR];
};

// Shared-memory index of row r of a per-step vector, padded by 16 bytes every 32
// rows so that the TPC row blocks of a column read from different banks.
__device__ __forceinline__ int vidx(int r) { return r + ((r >> 5) << 2); }

template <int MAXR, int TPC>
__global__ void __launch_bounds__(kCqMaxThreads, 1) k_cpqr_cluster(const CqParams P) {
    constexpr int RPT = MAXR / TPC;
    constexpr int VLEN = MAXR + MAXR / 8;          // padded vector length
    constexpr int MAXW = kCqMaxThreads / 32;
    constexpr uint32_t REC = sizeof(CqRecord<MAXR>);
    static_assert(REC % 16 == 0, "record size");
    static_assert(RPT % 4 == 0, "rows per thread");
    __shared__ __align__(128) CqRecord<MAXR> recv[2][kCqMaxCluster];
    __shared__ __align__(128) CqRecord<MAXR> wstg[2][MAXW];   // per-warp staged candidate
    __shared__ __align__(16) float vp[VLEN];     // v' : 0 above row j, alpha - beta at j, pivot column below
    __shared__ __align__(16) float ej[VLEN];     // unit vector e_j
    __shared__ float wv[MAXW];
    __shared__ int wi[MAXW];
    __shared__ float wsum[MAXW];
    __shared__ float s_sc[4];                    // tau, inv, beta, sum of norms
    __shared__ int s_piv[2];                     // pivot column, stop flag
    __shared__ __align__(8) uint64_t recv_bar[2];

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
    const int64_t i = static_cast<int64_t>(me) * P.cpb + cl;
    const bool valid = cl < P.cpb && i < W.n;
    const int r = static_cast<int>(W.r);
    const int rb = qq * RPT;                 // first row of this thread's block
    const float sqrt_u = 2.44140625e-04f;    // sqrt of the FP32 unit round-off 2^-24

    if (t == 0) {
        mbar_init(&recv_bar[0], 1);
        mbar_init(&recv_bar[1], 1);
        fence_barrier_init();
    }
    cluster_sync_all();

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
    bool selected = !valid;
    if (valid && qq == 0) {
        if (!isfinite(nu)) set_info(W.info, kInfoNonFinite);
        W.sel[i] = 0;
    }

    // Exchange q: each warp stages its best candidate column, warp 0 picks the CTA's best
    // and bulk-copies that record to every peer.  Exchange q fills recv[q & 1] and
    // completes phase q >> 1 of recv_bar[q & 1]; a peer can be at most one exchange ahead,
    // so two alternating buffers and barriers never mix phases, and a staging slot is
    // reused (two exchanges later) only after its copies have landed.
    auto exchange = [&](int q) {
        const int slot = q & 1;
        float bv = -1.f, part = 0.f;
        int bi = -1;
        if (!selected && qq == 0) { bv = nu; bi = static_cast<int>(i); part = nu; }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            better(bv, bi, ov, oi);
            part += __shfl_xor_sync(0xffffffffu, part, o);
        }
        if (valid && i == bi) {
#pragma unroll
            for (int u = 0; u < RPT; u += 4)
                *reinterpret_cast<float4*>(&wstg[slot][warp].col[rb + u]) = make_float4(x[u], x[u + 1], x[u + 2], x[u + 3]);
        }
        if (lane == 0) { wv[warp] = bv; wi[warp] = bi; wsum[warp] = part; }
        fence_proxy_async_smem();
        __syncthreads();
        if (warp == 0) {
            float v0 = lane < nw ? wv[lane] : -1.f;
            int i0 = lane < nw ? wi[lane] : -1;
            int w0 = lane;
            float s0 = lane < nw ? wsum[lane] : 0.f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ov = __shfl_xor_sync(0xffffffffu, v0, o);
                const int oi = __shfl_xor_sync(0xffffffffu, i0, o);
                const int ow = __shfl_xor_sync(0xffffffffu, w0, o);
                if (oi >= 0 && (i0 < 0 || ov > v0 || (ov == v0 && oi < i0))) { v0 = ov; i0 = oi; w0 = ow; }
                s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            }
            const int wsrc = i0 >= 0 ? w0 : 0;
            if (lane == 0) {
                mbar_arrive_expect_tx(&recv_bar[slot], C * REC);
                wstg[slot][wsrc].head = make_float4(v0, __int_as_float(i0), s0, 0.f);
                fence_proxy_async_smem();
            }
            __syncwarp();
            if (lane < static_cast<int>(C)) {
                const uint32_t d = static_cast<uint32_t>(lane);
                bulk_s2peer(map_peer(smem_addr(&recv[slot][me]), d), smem_addr(&wstg[slot][wsrc]), REC,
                            map_peer(smem_addr(&recv_bar[slot]), d));
            }
        }
    };
    auto wait_exchange = [&](int q) -> bool {
        volatile int keep = 0;
        return mbar_wait(&recv_bar[q & 1], static_cast<uint32_t>((q >> 1) & 1), &keep, P.limit_ns);
    };

    exchange(0);
    bool ok = wait_exchange(0);
    int k = 0;
    float total = -1.f;
    for (int j = 0; ok && j < W.kcap; ++j) {
        const int par = j & 1;
        // ---- warp 0: the pivot (same reduction order in every CTA), reflector scalars,
        // and the step vectors v' and e_j
        if (warp == 0) {
            float hv = -1.f, hs = 0.f;
            int hi = -1, hsrc = lane;
            if (lane < static_cast<int>(C)) {
                const float4 h = recv[par][lane].head;
                hv = h.x;
                hi = __float_as_int(h.y);
                hs = h.z;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ov = __shfl_xor_sync(0xffffffffu, hv, o);
                const int oi = __shfl_xor_sync(0xffffffffu, hi, o);
                const int os = __shfl_xor_sync(0xffffffffu, hsrc, o);
                if (oi >= 0 && (hi < 0 || ov > hv || (ov == hv && oi < hi))) { hv = ov; hi = oi; hsrc = os; }
                hs += __shfl_xor_sync(0xffffffffu, hs, o);
            }
            if (total < 0.f) total = hs;
            int stop = 0;
            if (W.rel_tol > 0.0 && sqrtf(fmaxf(hs, 0.f)) <= static_cast<float>(W.rel_tol) * sqrtf(total)) stop = 1;
            if (!stop && (hi < 0 || !(hv > 0.f))) {
                stop = 2;
                if (me == 0 && lane == 0) set_info(W.info, j + 1);
            }
            if (!stop) {
                const float* xw = recv[par][hsrc].col;
                float s2 = 0.f;
                for (int q = j + lane; q < r; q += 32) s2 = fmaf(xw[q], xw[q], s2);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
                const float alpha = xw[j];
                const float snorm = sqrtf(s2);
                const float beta = alpha >= 0.f ? -snorm : snorm;
                const float amb = alpha - beta;
                for (int q = lane; q < MAXR; q += 32) {
                    vp[vidx(q)] = q < j ? 0.f : (q == j ? amb : xw[q]);
                    ej[vidx(q)] = q == j ? 1.f : 0.f;
                }
                if (lane == 0) {
                    s_sc[0] = (beta - alpha) / beta;   // tau
                    s_sc[1] = 1.f / amb;               // inv
                    s_sc[2] = beta;
                }
            }
            if (lane == 0) { s_piv[0] = hi; s_piv[1] = stop; }
        }
        __syncthreads();
        if (s_piv[1]) break;
        const int p = s_piv[0];
        const float tau = s_sc[0], inv = s_sc[1];
        if (valid && i == p) {
            selected = true;
            if (qq == 0) {
                W.R[i * W.ldr + j] = static_cast<double>(s_sc[2]);
                W.J[j] = p;
                W.sel[i] = 1;
            }
        }
        // S = v'.x (= (alpha - beta) w),  X = e_j.x (= x_j): plain FMAs over this thread's rows
        float S0 = 0.f, S1 = 0.f, X = 0.f;
#pragma unroll
        for (int u = 0; u < RPT; u += 4) {
            const float4 v4 = *reinterpret_cast<const float4*>(&vp[vidx(rb + u)]);
            const float4 e4 = *reinterpret_cast<const float4*>(&ej[vidx(rb + u)]);
            S0 = fmaf(v4.x, x[u], S0);
            S1 = fmaf(v4.y, x[u + 1], S1);
            S0 = fmaf(v4.z, x[u + 2], S0);
            S1 = fmaf(v4.w, x[u + 3], S1);
            X = fmaf(e4.x, x[u], X);
            X = fmaf(e4.y, x[u + 1], X);
            X = fmaf(e4.z, x[u + 2], X);
            X = fmaf(e4.w, x[u + 3], X);
        }
        float S = S0 + S1;
#pragma unroll
        for (int o = 1; o < TPC; o <<= 1) {
            S += __shfl_xor_sync(0xffffffffu, S, o);
            X += __shfl_xor_sync(0xffffffffu, X, o);
        }
        const float tw = tau * (inv * S);
        const float sv = tw * inv;
        const float rho = X - tw;
        bool recompute = false;
        if (!selected) {
            // x -= (tau w / (alpha - beta)) v': rows above j unchanged, row j becomes rho
#pragma unroll
            for (int u = 0; u < RPT; u += 4) {
                const float4 v4 = *reinterpret_cast<const float4*>(&vp[vidx(rb + u)]);
                x[u] = fmaf(-sv, v4.x, x[u]);
                x[u + 1] = fmaf(-sv, v4.y, x[u + 1]);
                x[u + 2] = fmaf(-sv, v4.z, x[u + 2]);
                x[u + 3] = fmaf(-sv, v4.w, x[u + 3]);
            }
            if (qq == 0) W.R[i * W.ldr + j] = static_cast<double>(rho);
            if (nu > 0.f) {
                const float t1 = fmaxf(1.f - (rho * rho) / nu, 0.f);
                if (t1 * (nu / nuref) <= sqrt_u) recompute = true;   // same decision in all TPC threads
                else nu = nu * t1;
            }
        }
        if (__any_sync(0xffffffffu, recompute)) {
            float sq = 0.f;
#pragma unroll
            for (int u = 0; u < RPT; ++u) sq = (rb + u > j) ? fmaf(x[u], x[u], sq) : sq;
#pragma unroll
            for (int o = 1; o < TPC; o <<= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
            if (recompute) {
                nu = sq;
                nuref = sq;
            }
        }
        exchange(j + 1);
        ok = wait_exchange(j + 1);
        k = j + 1;
    }
    if (!ok && t == 0) set_info(W.info, kInfoWatchdog);
    // no CTA leaves while a peer may still copy into its shared memory
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

static int cq_maxr(int64_t r) { return r <= 32 ? 32 : (r <= 64 ? 64 : (r <= 128 ? 128 : 160)); }

static bool cq_fits_any(int maxr, int tpc, int csize, int threads) {
    switch (maxr) {
        case 32: return cq_fits<32>(tpc, csize, threads);
        case 64: return cq_fits<64>(tpc, csize, threads);
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
            case 128: return launch_cq<128, 4>(P, cs, nclusters, th, s);
            default: return launch_cq<160, 4>(P, cs, nclusters, th, s);
        }
    }
    switch (plan.maxr) {
        case 32: return launch_cq<32, 2>(P, cs, nclusters, th, s);
        case 64: return launch_cq<64, 2>(P, cs, nclusters, th, s);
        default: return launch_cq<128, 2>(P, cs, nclusters, th, s);
    }
}

cudaError_t launch_cpqr_cluster(const float* Y, int64_t r, int64_t n, int64_t ldy, int kcap, double rel_tol,
                                int32_t* J, int32_t* k_out, int32_t* info, double* R64, int64_t ldr, uint8_t* sel,
                                const ClusterCpqrPlan& plan, uint64_t limit_ns, cudaStream_t s) {
    CqParams P{};
    P.Y = Y; P.r = r; P.n = n; P.ldy = ldy;
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
