// Truncated column-pivoted Householder QR (Sec. 1.1, Algorithm 1, the pivoted QR) on GB300.
//
// Greedy Businger-Golub pivoting: step j picks the unselected column with the
// largest residual norm, builds the Householder reflector that maps its
// residual X(j:r, p) to beta e_1, applies it to the other unselected columns
// and records row j of R.  Column norms are downdated, nu_i -= R(j,i)^2, and
// recomputed when the Drmac-Bujanovic cancellation test fires.
//
// One cooperative grid: CTA b owns a contiguous slice of columns and updates
// them in place (a warp per column).  Each step needs one global argmax, which
// is one bounded grid barrier: every CTA publishes (best norm, index, sum of
// norms) for its slice into a double-buffered candidate table, and after the
// barrier every CTA reduces the same table in the same order, so all CTAs
// agree on the pivot without a second barrier.  The pivot column itself is not
// modified in the step it is chosen, so every CTA reads it straight from the
// working matrix to form the reflector.
#include "common.cuh"
#include "internal.h"

#include <algorithm>

namespace gid {

struct Cand {
    double nu;      // best residual squared norm in the slice (-1 if none)
    double sumnu;   // sum of residual squared norms of unselected columns in the slice
    double total;   // initial sum of squares of the slice (||W||_F^2 part)
    int idx;        // column of the best norm (-1 if none)
    int pad;
};

struct CpqrCtrl {
    uint32_t counter;
    int abort;
    uint32_t pad[62];
};

template <typename T>
struct CpqrParams {
    T* X;
    int64_t r, n, ldx;
    const void* src;
    int src_f64;
    int64_t ldsrc;
    int kcap;
    double rel_tol;
    int32_t* J;
    int32_t* k_out;
    int32_t* info;
    double* R;
    int64_t ldr;
    T* nu;
    T* nuref;
    uint8_t* sel;
    CpqrCtrl* ctrl;
    Cand* cand;       // [2][gridDim.x]
    T* vglobal;       // per-CTA reflector storage when it does not fit in shared memory
    int v_in_smem;
    uint64_t limit_ns;
};

template <typename T> struct SqrtU;
template <> struct SqrtU<double> { static __device__ double v() { return 1.0536712127723509e-08; } };  // 2^-26.5
template <> struct SqrtU<float> { static __device__ float v() { return 2.44140625e-04f; } };           // 2^-12

// Deterministic block sum (fixed tree over warps).  All threads get the result.
template <typename T>
__device__ T block_sum(T v, T* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    T s = 0;
    if (warp == 0) {
        s = lane < nw ? sh[lane] : T(0);
        s = warp_sum(s);
        if (lane == 0) sh[32] = s;
    }
    __syncthreads();
    return sh[32];
}

// argmax of (value, index) with ties to the smaller index; returns to all threads.
__device__ void block_argmax(double v, int idx, double* shv, int* shi, double* outv, int* outi) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ov > v || (ov == v && oi >= 0 && (idx < 0 || oi < idx))) { v = ov; idx = oi; }
    }
    __syncthreads();
    if (lane == 0) { shv[warp] = v; shi[warp] = idx; }
    __syncthreads();
    if (warp == 0) {
        v = lane < nw ? shv[lane] : -1.0;
        idx = lane < nw ? shi[lane] : -1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, v, o);
            const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
            if (ov > v || (ov == v && oi >= 0 && (idx < 0 || oi < idx))) { v = ov; idx = oi; }
        }
        if (lane == 0) { shv[32] = v; shi[32] = idx; }
    }
    __syncthreads();
    *outv = shv[32];
    *outi = shi[32];
}

// Candidate entries written by other CTAs are read from L2 (never from a stale L1 line).
__device__ __forceinline__ Cand load_cand(const Cand* p) {
    Cand c;
    c.nu = __ldcg(&p->nu);
    c.sumnu = __ldcg(&p->sumnu);
    c.total = __ldcg(&p->total);
    c.idx = __ldcg(&p->idx);
    c.pad = 0;
    return c;
}

template <typename T>
__device__ void publish_candidate(const CpqrParams<T>& P, int64_t c0, int64_t c1, int slot, double total,
                                  double* shv, int* shi, T* shs) {
    double best = -1.0;
    int bi = -1;
    T part = 0;
    for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
        if (P.sel[i]) continue;
        const double v = static_cast<double>(P.nu[i]);
        part += P.nu[i];
        if (v > best) { best = v; bi = static_cast<int>(i); }
    }
    double bv;
    int bidx;
    block_argmax(best, bi, shv, shi, &bv, &bidx);
    const T s = block_sum(part, shs);
    if (threadIdx.x == 0) {
        Cand c;
        c.nu = bv;
        c.sumnu = static_cast<double>(s);
        c.total = total;
        c.idx = bidx;
        c.pad = 0;
        P.cand[slot * gridDim.x + blockIdx.x] = c;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_cpqr_grid(const CpqrParams<T> P) {
    extern __shared__ uint8_t smem_dyn[];
    __shared__ double shv[33];
    __shared__ int shi[33];
    __shared__ T shs[33];
    __shared__ int s_ok;
    __shared__ double s_sel[3];   // best nu, sum nu, total
    __shared__ int s_idx;

    const int G = gridDim.x, b = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t c0 = P.n * b / G, c1 = P.n * (b + 1) / G;
    T* v = P.v_in_smem ? reinterpret_cast<T*>(smem_dyn) : P.vglobal + static_cast<int64_t>(b) * P.r;
    const T sqrt_u = SqrtU<T>::v();
    uint32_t epoch = 0;

    // ---- init: working copy, exact squared norms
    T local_total = 0;
    bool bad = false;
    for (int64_t i = c0 + warp; i < c1; i += nw) {
        T* x = P.X + i * P.ldx;
        T s = 0;
        for (int64_t t = lane; t < P.r; t += 32) {
            T a;
            if (P.src) {
                a = P.src_f64 ? static_cast<T>(static_cast<const double*>(P.src)[i * P.ldsrc + t])
                              : static_cast<T>(static_cast<const float*>(P.src)[i * P.ldsrc + t]);
                x[t] = a;
            } else {
                a = x[t];
            }
            s += a * a;
        }
        s = warp_sum(s);
        if (lane == 0) {
            if (!isfinite(static_cast<double>(s))) bad = true;
            P.nu[i] = s;
            P.nuref[i] = s;
            P.sel[i] = 0;
        }
        if (lane == 0) local_total += s;
    }
    if (bad) set_info(P.info, kInfoNonFinite);
    const T tot = block_sum(local_total, shs);
    __syncthreads();
    publish_candidate(P, c0, c1, 0, static_cast<double>(tot), shv, shi, shs);
    bool ok = grid_barrier(&P.ctrl->counter, epoch, &P.ctrl->abort, P.limit_ns, &s_ok);

    int k = 0;
    double total = 0.0;
    for (int j = 0; ok && j < P.kcap; ++j) {
        const int slot = j & 1;
        // ---- global pivot: identical reduction of the candidate table in every CTA
        {
            double bv = -1.0, sn = 0.0, tt = 0.0;
            int bi = -1;
            for (int g = threadIdx.x; g < G; g += blockDim.x) {
                const Cand c = load_cand(P.cand + slot * G + g);
                if (c.nu > bv || (c.nu == bv && c.idx >= 0 && (bi < 0 || c.idx < bi))) { bv = c.nu; bi = c.idx; }
                sn += c.sumnu;
                tt += c.total;
            }
            double gv;
            int gi;
            block_argmax(bv, bi, shv, shi, &gv, &gi);
            const double gsn = block_sum(sn, shv);
            double gtt = 0.0;
            if (j == 0) {
                // the first table also carries the slices' initial sums of squares
                gtt = block_sum(tt, shv);
            }
            if (threadIdx.x == 0) { s_sel[0] = gv; s_sel[1] = gsn; s_sel[2] = gtt; s_idx = gi; }
            __syncthreads();
        }
        if (j == 0) total = s_sel[2];
        const double best = s_sel[0];
        const int p = s_idx;
        if (P.rel_tol > 0.0 && sqrt(fmax(s_sel[1], 0.0)) <= P.rel_tol * sqrt(total)) break;
        if (p < 0 || !(best > 0.0)) {
            if (b == 0 && threadIdx.x == 0) set_info(P.info, j + 1);
            break;
        }
        // ---- reflector from x = X(j:r, p):  beta = -sign(alpha)||x||, v = x / (alpha - beta), v0 = 1
        const T* xp = P.X + static_cast<int64_t>(p) * P.ldx;
        T part = 0;
        for (int64_t t = j + threadIdx.x; t < P.r; t += blockDim.x) {
            const T a = __ldcg(xp + t);
            v[t - j] = a;
            part += a * a;
        }
        const T ss = block_sum(part, shs);   // includes a __syncthreads after the writes
        const T alpha = v[0];
        const T snorm = sqrt(ss);
        const T beta = alpha >= T(0) ? -snorm : snorm;
        const T tau = (beta - alpha) / beta;
        const T denom = alpha - beta;
        __syncthreads();
        for (int64_t t = 1 + threadIdx.x; t < P.r - j; t += blockDim.x) v[t] = v[t] / denom;
        if (threadIdx.x == 0) v[0] = T(1);
        if (p >= c0 && p < c1 && threadIdx.x == 0) {
            P.sel[p] = 1;
            P.J[j] = p;
            P.R[static_cast<int64_t>(p) * P.ldr + j] = static_cast<double>(beta);
        }
        __syncthreads();
        // ---- apply to the unselected columns of this slice (warp per column)
        const int64_t len = P.r - j;
        for (int64_t i = c0 + warp; i < c1; i += nw) {
            if (P.sel[i]) continue;
            T* x = P.X + i * P.ldx + j;
            T w = 0;
            for (int64_t t = lane; t < len; t += 32) w += v[t] * x[t];
            w = warp_sum(w);
            const T tw = tau * w;
            T rho = 0;
            for (int64_t t = lane; t < len; t += 32) {
                const T nx = x[t] - tw * v[t];
                x[t] = nx;
                if (t == 0) rho = nx;
            }
            rho = __shfl_sync(0xffffffffu, rho, 0);
            bool recompute = false;
            T nu_i = P.nu[i];
            if (lane == 0) P.R[i * P.ldr + j] = static_cast<double>(rho);
            if (nu_i > T(0)) {
                T t1 = T(1) - (rho * rho) / nu_i;
                if (t1 < T(0)) t1 = T(0);
                if (t1 * (nu_i / P.nuref[i]) <= sqrt_u) recompute = true;
                else nu_i = nu_i * t1;
            }
            if (recompute) {
                T s = 0;
                for (int64_t t = 1 + lane; t < len; t += 32) s += x[t] * x[t];
                s = warp_sum(s);
                nu_i = s;
                if (lane == 0) P.nuref[i] = s;
            }
            if (lane == 0) P.nu[i] = nu_i;
        }
        __syncthreads();
        publish_candidate(P, c0, c1, slot ^ 1, 0.0, shv, shi, shs);
        ok = grid_barrier(&P.ctrl->counter, epoch, &P.ctrl->abort, P.limit_ns, &s_ok);
        k = j + 1;
    }
    if (!ok) {
        if (threadIdx.x == 0) set_info(P.info, kInfoWatchdog);
        return;
    }
    // ---- CTA 0: rank and the complement J[k:n] in ascending column order
    if (b == 0) {
        if (threadIdx.x == 0) *P.k_out = k;
        __shared__ int s_base;
        if (threadIdx.x == 0) s_base = k;
        __syncthreads();
        for (int64_t i0 = 0; i0 < P.n; i0 += blockDim.x) {
            const int64_t i = i0 + threadIdx.x;
            const int flag = (i < P.n && !__ldcg(P.sel + i)) ? 1 : 0;
            // block exclusive scan of flags (warp ballots)
            const unsigned bal = __ballot_sync(0xffffffffu, flag);
            const int wpre = __popc(bal & ((1u << lane) - 1u));
            if (lane == 0) shi[warp] = __popc(bal);
            __syncthreads();
            int off = 0;
            for (int w = 0; w < warp; ++w) off += shi[w];
            if (flag) P.J[s_base + off + wpre] = static_cast<int32_t>(i);
            __syncthreads();
            if (threadIdx.x == 0) {
                int tot = 0;
                for (int w = 0; w < nw; ++w) tot += shi[w];
                s_base += tot;
            }
            __syncthreads();
        }
    }
}

size_t cpqr_ctrl_bytes(const CpqrPlan& plan, int64_t r, int elem_bytes) {
    size_t b = sizeof(CpqrCtrl) + 2 * static_cast<size_t>(plan.grid) * sizeof(Cand);
    if (plan.smem == 0) b = ((b + 255) & ~size_t(255)) + static_cast<size_t>(plan.grid) * r * elem_bytes;
    return b;
}

bool cpqr_plan(int64_t r, int64_t n, int elem_bytes, CpqrPlan* plan) {
    const DeviceInfo& dev = device_info();
    plan->threads = 256;
    plan->grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(dev.sm_count, n)));
    const size_t vbytes = static_cast<size_t>(r) * elem_bytes;
    plan->smem = vbytes <= 160 * 1024 ? vbytes : 0;
    return true;
}

template <typename T>
static cudaError_t launch_cpqr_t(void* W, int64_t r, int64_t n, int64_t ldw, const void* src, int src_f64,
                                 int64_t ldsrc, int kcap, double rel_tol, int32_t* J, int32_t* k_out,
                                 int32_t* info, double* R64, int64_t ldr, void* nu, void* nuref, uint8_t* sel,
                                 void* ctrl, void* vglobal, const CpqrPlan& plan, uint64_t limit_ns,
                                 cudaStream_t s) {
    CpqrParams<T> P{};
    P.X = static_cast<T*>(W);
    P.r = r; P.n = n; P.ldx = ldw;
    P.src = src; P.src_f64 = src_f64; P.ldsrc = ldsrc;
    P.kcap = kcap; P.rel_tol = rel_tol;
    P.J = J; P.k_out = k_out; P.info = info;
    P.R = R64; P.ldr = ldr;
    P.nu = static_cast<T*>(nu); P.nuref = static_cast<T*>(nuref); P.sel = sel;
    P.ctrl = static_cast<CpqrCtrl*>(ctrl);
    P.cand = reinterpret_cast<Cand*>(static_cast<char*>(ctrl) + sizeof(CpqrCtrl));
    P.vglobal = static_cast<T*>(vglobal);
    P.v_in_smem = plan.smem > 0 ? 1 : 0;
    P.limit_ns = limit_ns;
    cudaError_t e = cudaMemsetAsync(ctrl, 0, sizeof(CpqrCtrl), s);
    if (e != cudaSuccess) return e;
    if (plan.smem > 48 * 1024) {
        e = cudaFuncSetAttribute(k_cpqr_grid<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(plan.smem));
        if (e != cudaSuccess) return e;
    }
    void* args[] = {&P};
    return cudaLaunchCooperativeKernel(reinterpret_cast<void*>(k_cpqr_grid<T>), dim3(plan.grid),
                                       dim3(plan.threads), args, plan.smem, s);
}

cudaError_t launch_cpqr(void* W, int w_f64, int64_t r, int64_t n, int64_t ldw, const void* src, int src_f64,
                        int64_t ldsrc, int kcap, double rel_tol, int32_t* J, int32_t* k_out, int32_t* info,
                        double* R64, int64_t ldr, void* nu, void* nuref, uint8_t* sel, void* ctrl,
                        const CpqrPlan& plan, uint64_t limit_ns, cudaStream_t s) {
    // per-CTA reflector storage follows the candidate table when shared memory is too small
    void* vglobal = nullptr;
    if (plan.smem == 0) {
        const size_t off = (sizeof(CpqrCtrl) + 2 * static_cast<size_t>(plan.grid) * sizeof(Cand) + 255) &
                           ~size_t(255);
        vglobal = static_cast<char*>(ctrl) + off;
    }
    if (w_f64)
        return launch_cpqr_t<double>(W, r, n, ldw, src, src_f64, ldsrc, kcap, rel_tol, J, k_out, info, R64, ldr,
                                     nu, nuref, sel, ctrl, vglobal, plan, limit_ns, s);
    return launch_cpqr_t<float>(W, r, n, ldw, src, src_f64, ldsrc, kcap, rel_tol, J, k_out, info, R64, ldr, nu,
                                nuref, sel, ctrl, vglobal, plan, limit_ns, s);
}

}  // namespace gid
