// Truncated column-pivoted Householder QR (Sec. 1.1, Algorithm 1, the pivoted QR) of a
// matrix whose columns fit the shared memory of a cooperative grid: one warp per column.
//
// CTA b owns the contiguous column slice [n b / G, n (b + 1) / G), held in its shared
// memory for the whole factorisation; warp w of the CTA owns the slice's columns
// w, w + NW, ...  A step needs, besides the pivot column, only the scalars
// alpha = x_p(j) and ||x_p(j:r)||: with beta = -sign(alpha) ||x_p(j:r)|| and
// S_i = x_p(j:r)^T x_i(j:r) - beta x_i(j), the reflector maps column i to
//     R(j,i) = x_i(j) - tw_i,   x_i(t) -= (tw_i / (alpha - beta)) x_p(t)  (t > j),
// tw_i = -S_i / beta.  A column's dot product, update and new squared norm (rows below
// the step, accumulated as the update writes them, so every pivot choice uses exact
// norms) are the work of its warp alone: no CTA-wide reduction.  Per step a warp reduces
// the grid's candidate table itself (no barrier), the CTA takes one barrier to find its
// best remaining column, publishes that column and its norm to a double-buffered global
// slot, and one bounded grid barrier ends the step.
#include "cpqr_grid.cuh"

#include <algorithm>

namespace gid {

constexpr int kResWarps = 8;

// (value, index) warp argmax, ties to the smaller index; lane 0's result goes to every
// lane.  Values must be ordered (no NaN: callers map non-finite norms to -1), so that
// every lane and every warp reducing the same entries takes the same decision: the
// warps of a CTA branch on it independently, and must meet at the same barriers.
__device__ __forceinline__ void warp_argmax(double& v, int& idx) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (oi >= 0 && (idx < 0 || ov > v || (ov == v && oi < idx))) { v = ov; idx = oi; }
    }
    v = __shfl_sync(0xffffffffu, v, 0);
    idx = __shfl_sync(0xffffffffu, idx, 0);
}

// A residual norm as a pivot key: non-finite values (a non-finite input, reported in
// info) order below every real norm.
__device__ __forceinline__ double norm_key(double nu) { return isfinite(nu) ? nu : -1.0; }

template <typename T>
__global__ void __launch_bounds__(kResWarps * 32) k_cpqr_resident(const CpqrParams<T> P) {
    extern __shared__ __align__(16) uint8_t smem_dyn[];
    __shared__ double w_nu[kResWarps], w_sum[kResWarps];
    __shared__ int w_idx[kResWarps];
    __shared__ int s_ok;
    __shared__ int cnt[kResWarps];

    const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int64_t c0 = P.n * b / G, c1 = P.n * (b + 1) / G;
    const int nc = static_cast<int>(c1 - c0);
    const int64_t r = P.r;
    T* nu_s = reinterpret_cast<T*>(smem_dyn);                                       // [cpb]
    uint8_t* sel_s = reinterpret_cast<uint8_t*>(nu_s + P.cpb_max);                 // [cpb]
    T* xs = reinterpret_cast<T*>(sel_s + ((P.cpb_max + 15) & ~int64_t(15)));       // [nc][r]
    uint32_t epoch = 0;

    // ---- init: this warp's columns into shared memory, their exact squared norms
    bool bad = false;
    for (int c = warp; c < nc; c += kResWarps) {
        T* x = xs + static_cast<int64_t>(c) * r;
        const int64_t gc = c0 + c;
        T s = 0;
        for (int64_t t = lane; t < r; t += 32) {
            T a;
            if (P.src) {
                a = P.src_f64 ? static_cast<T>(static_cast<const double*>(P.src)[gc * P.ldsrc + t])
                              : static_cast<T>(static_cast<const float*>(P.src)[gc * P.ldsrc + t]);
            } else {
                a = P.X[gc * P.ldx + t];
            }
            x[t] = a;
            s = fma(a, a, s);
        }
        s = warp_sum(s);
        if (lane == 0) {
            if (!isfinite(static_cast<double>(s))) bad = true;
            nu_s[c] = s;
            sel_s[c] = 0;
            P.sel[gc] = 0;
        }
    }
    if (bad) set_info(P.info, kInfoNonFinite);

    // ---- the CTA's best remaining column for the step on row `row`: each warp's best and
    // sum, one barrier, then warp 0 picks the CTA's best (ties to the smaller column) and
    // publishes it: its rows row..r-1 to pub[slot][b], and the record (exact squared norm
    // of those rows, the entry on `row`, the slice's sum of norms; before the first step
    // that sum is also the slice's total sum of squares)
    auto publish = [&](int slot, int64_t row, bool first) {
        double v = -1.0, part = 0.0;
        int ci = -1;
        for (int c = warp; c < nc; c += kResWarps) {
            if (sel_s[c]) continue;
            const double nu = norm_key(static_cast<double>(nu_s[c]));
            part += nu;
            if (ci < 0 || nu > v) { v = nu; ci = c; }     // c ascends: ties keep the smaller
        }
        if (lane == 0) { w_nu[warp] = v; w_idx[warp] = ci; w_sum[warp] = part; }
        __syncthreads();
        if (warp == 0) {
            double bv = lane < kResWarps ? w_nu[lane] : -1.0;
            int bi = lane < kResWarps ? w_idx[lane] : -1;
            double sum = lane < kResWarps ? w_sum[lane] : 0.0;
            warp_argmax(bv, bi);
            sum = warp_sum(sum);
            T alpha = 0;
            if (bi >= 0 && row < r) {
                const T* x = xs + static_cast<int64_t>(bi) * r;
                T* dst = P.pub + (static_cast<int64_t>(slot) * G + b) * r;
                for (int64_t t = row + lane; t < r; t += 32) dst[t] = x[t];
                alpha = x[row];
            }
            if (lane == 0) {
                Cand cd;
                cd.nu = bv;
                cd.sumnu = sum;
                cd.total = first ? sum : 0.0;
                cd.s2 = bi >= 0 && row < r ? bv : 0.0;    // nu is the exact norm of rows row..r-1
                cd.alpha = static_cast<double>(alpha);
                cd.idx = bi >= 0 ? static_cast<int>(c0 + bi) : -1;
                cd.pad = 0;
                P.cand[slot * G + b] = cd;
            }
        }
    };

    publish(0, 0, true);
    bool ok = grid_barrier(&P.ctrl->counter, epoch, &P.ctrl->abort, P.limit_ns, &s_ok);

    int k = 0;
    double total = 0.0;
    for (int j = 0; ok && j < P.kcap; ++j) {
        const int slot = j & 1;
        // ---- the pivot: every warp reduces the candidate table in the same order
        double bv = -1.0, sn = 0.0, tt = 0.0;
        int bg = -1;
        for (int g = lane; g < G; g += 32) {
            const Cand c = load_cand(P.cand + slot * G + g);
            const double nu = norm_key(c.nu);
            if (c.idx >= 0 && (bg < 0 || nu > bv)) { bv = nu; bg = g; }   // g ascends per lane
            sn += c.sumnu;
            tt += c.total;
        }
        warp_argmax(bv, bg);
        sn = __shfl_sync(0xffffffffu, warp_sum(sn), 0);
        if (j == 0) total = __shfl_sync(0xffffffffu, warp_sum(tt), 0);
        double alpha_d = 0.0, s2 = 0.0;
        int p = -1;
        if (bg >= 0) {
            const Cand w = load_cand(P.cand + slot * G + bg);
            p = w.idx;
            alpha_d = w.alpha;
            s2 = w.s2;
        }
        if (P.rel_tol > 0.0 && sqrt(fmax(sn, 0.0)) <= P.rel_tol * sqrt(total)) break;
        if (p < 0 || !(bv > 0.0) || !(s2 > 0.0)) {
            if (b == 0 && tid == 0) set_info(P.info, j + 1);
            break;
        }
        // ---- reflector scalars; the pivot column as published (not modified in this step)
        const T alpha = static_cast<T>(alpha_d);
        const T snorm = sqrt(static_cast<T>(s2));
        const T beta = alpha >= T(0) ? -snorm : snorm;
        const T rbeta = T(1) / beta;
        const T inv = T(1) / (alpha - beta);
        const T* xp = P.pub + (static_cast<int64_t>(slot) * G + bg) * r;
        const int cp = (p >= c0 && p < c1) ? static_cast<int>(p - c0) : -1;
        if (cp >= 0 && (cp % kResWarps) == warp && lane == 0) {
            sel_s[cp] = 1;
            P.sel[p] = 1;
            P.J[j] = p;
            P.R[static_cast<int64_t>(p) * P.ldr + j] = static_cast<double>(beta);
        }
        // ---- this warp's unselected columns
        for (int c = warp; c < nc; c += kResWarps) {
            if (c == cp || sel_s[c]) continue;
            T* x = xs + static_cast<int64_t>(c) * r;
            T s0 = 0, s1 = 0;
            int64_t t = j + lane;
            for (; t + 32 < r; t += 64) {
                s0 = fma(__ldcg(xp + t), x[t], s0);
                s1 = fma(__ldcg(xp + t + 32), x[t + 32], s1);
            }
            if (t < r) s0 = fma(__ldcg(xp + t), x[t], s0);
            T S = warp_sum(s0 + s1);
            const T X = x[j];
            S = fma(-beta, X, S);
            const T tw = -S * rbeta;
            const T sv = tw * inv;
            if (lane == 0) P.R[(c0 + c) * P.ldr + j] = static_cast<double>(X - tw);
            T q0 = 0, q1 = 0;
            t = j + 1 + lane;
            for (; t + 32 < r; t += 64) {
                const T a0 = fma(-sv, __ldcg(xp + t), x[t]);
                const T a1 = fma(-sv, __ldcg(xp + t + 32), x[t + 32]);
                x[t] = a0;
                x[t + 32] = a1;
                q0 = fma(a0, a0, q0);
                q1 = fma(a1, a1, q1);
            }
            if (t < r) {
                const T a0 = fma(-sv, __ldcg(xp + t), x[t]);
                x[t] = a0;
                q0 = fma(a0, a0, q0);
            }
            const T nu = warp_sum(q0 + q1);
            if (lane == 0) nu_s[c] = nu;
        }
        __syncwarp();
        publish(slot ^ 1, j + 1, false);
        ok = grid_barrier(&P.ctrl->counter, epoch, &P.ctrl->abort, P.limit_ns, &s_ok);
        k = j + 1;
    }
    if (!ok) {
        if (tid == 0) set_info(P.info, kInfoWatchdog);
        return;
    }
    if (b == 0) list_complement(P.J, P.sel, P.n, k, P.k_out, cnt);
}

template <typename T>
cudaError_t launch_cpqr_resident(const CpqrParams<T>& P, int grid, size_t smem, cudaStream_t s) {
    auto kern = k_cpqr_resident<T>;
    if (smem > 48 * 1024) {
        const cudaError_t e =
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    CpqrParams<T> Pc = P;
    void* args[] = {&Pc};
    return cudaLaunchCooperativeKernel(reinterpret_cast<void*>(kern), dim3(grid), dim3(kResWarps * 32), args, smem,
                                       s);
}

template cudaError_t launch_cpqr_resident<double>(const CpqrParams<double>&, int, size_t, cudaStream_t);
template cudaError_t launch_cpqr_resident<float>(const CpqrParams<float>&, int, size_t, cudaStream_t);

}  // namespace gid
