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
// norms) are the work of its warp alone: no CTA-wide reduction.
//
// The grid synchronises through its candidate table alone.  Each CTA publishes its best
// remaining column (the column into a double-buffered global slot, then a record with its
// norm, next-row entry and the slice's sum of norms) and stamps the record with the step
// number last, after a fence (release).  Warp 0 of every CTA polls the stamps of the whole
// table with acquire loads until every record of the step has arrived (bounded by the
// watchdog), reduces it in a fixed order, stages the winner's column in shared memory,
// and one CTA barrier hands the step to the other warps.  No counter barrier: the wait
// for the table is the step's only grid-wide wait.  The table is cleared before the
// launch, so a replayed launch never sees an earlier call's stamps.
#include "cpqr_grid.cuh"

#include <algorithm>

namespace gid {

constexpr int kResWarps = 8;
// Candidate-table entries per lane of the polling warp (a grid of up to 32 x 5 = 160 CTAs).
constexpr int kTableLanes = 5;

__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_s32(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// A residual norm as a pivot key: non-finite values (a non-finite input, reported in
// info) order below every real norm.
__device__ __forceinline__ double norm_key(double nu) { return isfinite(nu) ? nu : -1.0; }

// The same order on the integer pipe: a finite norm's bits plus two (a -0 counts as +0), 1 for
// a non-finite norm or the -1 a record carries for one, 0 for "no candidate"; keys compare as
// unsigned integers, so a step's reductions need no FP64 instruction.
__device__ __forceinline__ uint64_t res_key(float v) {
    const uint32_t a = __float_as_uint(v) & 0x7FFFFFFFu;
    return a >= 0x7F800000u ? 1ull : static_cast<uint64_t>(a) + 2ull;
}
__device__ __forceinline__ uint64_t res_key(double v) {
    const uint64_t u = static_cast<uint64_t>(__double_as_longlong(v));
    const uint64_t a = u & 0x7FFFFFFFFFFFFFFFull;
    if (a >= 0x7FF0000000000000ull || ((u >> 63) != 0ull && a != 0ull)) return 1ull;
    return a + 2ull;
}
// The norm a key stands for, as the record's FP64 value (-1 for keys 0 and 1).
__device__ __forceinline__ double res_key_value(uint64_t key, float) {
    return key >= 2ull ? f64_of_f32(__uint_as_float(static_cast<uint32_t>(key - 2ull))) : -1.0;
}
__device__ __forceinline__ double res_key_value(uint64_t key, double) {
    return key >= 2ull ? __longlong_as_double(static_cast<long long>(key - 2ull)) : -1.0;
}

// Warp argmax of keys with ties to the smaller index; lane 0's result goes to every lane, so
// that every warp reducing the same entries takes the same decision (the warps of a CTA
// branch on it independently and must meet at the same barriers).
__device__ __forceinline__ void warp_argmax_key(uint64_t& key, int& idx) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t ok = __shfl_xor_sync(0xffffffffu, key, o);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (oi >= 0 && (idx < 0 || ok > key || (ok == key && oi < idx))) { key = ok; idx = oi; }
    }
    key = __shfl_sync(0xffffffffu, key, 0);
    idx = __shfl_sync(0xffffffffu, idx, 0);
}

template <typename T>
__global__ void __launch_bounds__(kResWarps * 32) k_cpqr_resident(const CpqrParams<T> P) {
    extern __shared__ __align__(16) uint8_t smem_dyn[];
    __shared__ unsigned long long w_key[kResWarps];
    __shared__ double w_sum[kResWarps];
    __shared__ int w_idx[kResWarps];
    __shared__ int cnt[kResWarps];
    // the step's decision, written by warp 0 before the CTA barrier
    __shared__ double s_alpha, s_s2;
    __shared__ int s_p, s_go;   // s_go: 1 carry on, 0 stop (rank reached or tolerance met), -1 watchdog
    __shared__ int s_src;       // the table entry (CTA) whose published column is the pivot

    const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const bool tol_mode = P.rel_tol > 0.0;     // sums of norms are formed only for the tolerance test
    const int64_t c0 = P.n * b / G, c1 = P.n * (b + 1) / G;
    const int nc = static_cast<int>(c1 - c0);
    const int64_t r = P.r;
    T* nu_s = reinterpret_cast<T*>(smem_dyn);                                       // [cpb]
    uint8_t* sel_s = reinterpret_cast<uint8_t*>(nu_s + P.cpb_max);                 // [cpb]
    T* xs = reinterpret_cast<T*>(sel_s + ((P.cpb_max + 15) & ~int64_t(15)));       // [nc][r]
    T* xps = xs + P.cpb_max * r;                                                    // [r] pivot column

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

    // ---- the CTA's best remaining column for step `step` (row `step`): each warp's best
    // and sum, one barrier, then warp 0 picks the CTA's best (ties to the smaller column),
    // writes its rows step..r-1 to pub[step & 1][b] and the record (exact squared norm of
    // those rows, the entry on row `step`, the slice's sum of norms; for step 0 that sum is
    // also the slice's total), and stamps the record with step + 1 after a fence
    auto publish = [&](int step) {
        const int slot = step & 1;
        uint64_t v = 0ull;
        double part = 0.0;
        int ci = -1;
        for (int c = warp; c < nc; c += kResWarps) {
            if (sel_s[c]) continue;
            const uint64_t key = res_key(nu_s[c]);
            if (tol_mode) part += norm_key(to_f64(nu_s[c]));
            if (ci < 0 || key > v) { v = key; ci = c; }     // c ascends: ties keep the smaller
        }
        if (lane == 0) { w_key[warp] = v; w_idx[warp] = ci; w_sum[warp] = part; }
        __syncthreads();
        // every warp finds the CTA's best the same way; all threads copy its rows
        uint64_t bk = lane < kResWarps ? w_key[lane] : 0ull;
        int bi = lane < kResWarps ? w_idx[lane] : -1;
        warp_argmax_key(bk, bi);
        const double bv = res_key_value(bk, T(0));
        if (bi >= 0 && step < r) {
            const T* x = xs + static_cast<int64_t>(bi) * r;
            T* dst = P.pub + (static_cast<int64_t>(slot) * G + b) * r;
            for (int64_t t = step + tid; t < r; t += kResWarps * 32) dst[t] = x[t];
        }
        // the column's stores, observed through the barrier, before the record's stamp
        __syncthreads();
        if (warp == 0) {
            double sum = 0.0;
            if (tol_mode) sum = warp_sum(lane < kResWarps ? w_sum[lane] : 0.0);
            const T alpha = (bi >= 0 && step < r) ? xs[static_cast<int64_t>(bi) * r + step] : T(0);
            Cand* rec = P.cand + slot * G + b;
            if (lane == 0) {
                rec->nu = bv;
                rec->sumnu = sum;
                rec->total = step == 0 ? sum : 0.0;
                rec->s2 = bi >= 0 && step < r ? bv : 0.0;   // nu is the exact norm of rows step..r-1
                rec->alpha = to_f64(alpha);
                rec->idx = bi >= 0 ? static_cast<int>(c0 + bi) : -1;
                __threadfence();
                st_release_s32(&rec->stamp, step + 1);
            }
        }
    };

    // ---- warp 0: wait (bounded) until every record of step `step` carries its stamp,
    // reduce the table in a fixed order (ties to the smaller CTA, hence column) and, unless
    // `final`, decide the step; the whole CTA then stages the winner's rows step..r-1.
    // s_go: 1 carry on, 0 stop (tolerance met, or zero residual: info = step + 1), -1 watchdog
    double total = 0.0;   // warp 0: ||W||_F^2, from the first table
    auto decide = [&](int step, bool final_wait) {
        const int slot = step & 1;
        // a lane's stamps are read together (relaxed loads, one round trip per poll); once all
        // have arrived, a fence orders the reads of the records and columns after them
        bool ok = true;
        const uint64_t t0 = globaltimer_ns();
        uint32_t it = 0;
        while (true) {
            bool ready = true;
#pragma unroll
            for (int q = 0; q < kTableLanes; ++q) {
                const int g = 32 * q + lane;
                if (g < G) ready &= ld_relaxed_s32(&P.cand[slot * G + g].stamp) == step + 1;
            }
            if (__all_sync(0xffffffffu, ready)) break;
            if ((++it & 15u) == 0) {
                bool stop = false;
                if (lane == 0) {
                    if (ld_volatile_i32(&P.ctrl->abort)) {
                        stop = true;
                    } else if (globaltimer_ns() - t0 > P.limit_ns) {
                        atomicExch(&P.ctrl->abort, 1);
                        stop = true;
                    }
                }
                if (__shfl_sync(0xffffffffu, stop, 0)) {
                    ok = false;
                    break;
                }
            }
        }
        __threadfence();
        __syncwarp();
        if (!ok) {
            if (lane == 0) s_go = -1;
            return;
        }
        if (final_wait) {
            if (lane == 0) s_go = 0;
            return;
        }
        uint64_t bk = 0ull;
        double sn = 0.0, tt = 0.0, wa = 0.0, ws = 0.0;
        int bg = -1, wi = -1;
        Cand e[kTableLanes];
#pragma unroll
        for (int q = 0; q < kTableLanes; ++q) {
            const int g = 32 * q + lane;
            if (g < G) e[q] = load_cand(P.cand + slot * G + g);
            else e[q].idx = -1;
        }
#pragma unroll
        for (int q = 0; q < kTableLanes; ++q) {
            const int g = 32 * q + lane;
            if (g >= G) continue;
            const uint64_t key = res_key(e[q].nu);
            if (e[q].idx >= 0 && (bg < 0 || key > bk)) {   // g ascends per lane
                bk = key; bg = g; wa = e[q].alpha; ws = e[q].s2; wi = e[q].idx;
            }
            if (tol_mode) {
                sn += e[q].sumnu;
                tt += e[q].total;
            }
        }
        warp_argmax_key(bk, bg);
        if (tol_mode) {
            sn = __shfl_sync(0xffffffffu, warp_sum(sn), 0);
            if (step == 0) total = __shfl_sync(0xffffffffu, warp_sum(tt), 0);
        }
        const double bv = res_key_value(bk, 0.0);
        const int src_lane = bg >= 0 ? (bg & 31) : 0;
        const double alpha = __shfl_sync(0xffffffffu, wa, src_lane);
        const double s2 = __shfl_sync(0xffffffffu, ws, src_lane);
        const int p = bg >= 0 ? __shfl_sync(0xffffffffu, wi, src_lane) : -1;
        int go = 1;
        if (tol_mode && sqrt(fmax(sn, 0.0)) <= P.rel_tol * sqrt(total)) {
            go = 0;
        } else if (p < 0 || !positive_bits(bv) || !positive_bits(s2)) {
            go = 0;
            if (b == 0 && lane == 0) set_info(P.info, step + 1);
        }
        if (lane == 0) {
            s_go = go;
            s_src = bg;
            s_p = p;
            s_alpha = alpha;
            s_s2 = s2;
        }
    };

    publish(0);
    int k = 0, go = 1;
    for (int j = 0; j < P.kcap; ++j) {
        if (warp == 0) decide(j, false);
        __syncthreads();
        go = s_go;
        if (go <= 0) break;
        {
            // the pivot column's rows j..r-1 from the table, every thread a few of them
            const T* src = P.pub + (static_cast<int64_t>(j & 1) * G + s_src) * r;
            for (int64_t t = j + tid; t < r; t += kResWarps * 32) xps[t] = __ldcg(src + t);
            __syncthreads();
        }
        // ---- reflector scalars; the pivot column staged in xps (not modified in this step)
        const int p = s_p;
        const T alpha = narrow_exact(s_alpha, T(0));
        const T snorm = sqrt(narrow_exact(s_s2, T(0)));
        const T beta = alpha >= T(0) ? -snorm : snorm;
        const T rbeta = T(1) / beta;
        const T inv = T(1) / (alpha - beta);
        const T* xp = xps;
        const int cp = (p >= c0 && p < c1) ? static_cast<int>(p - c0) : -1;
        if (cp >= 0 && (cp % kResWarps) == warp && lane == 0) {
            sel_s[cp] = 1;
            P.sel[p] = 1;
            P.J[j] = p;
            P.R[static_cast<int64_t>(p) * P.ldr + j] = to_f64(beta);
        }
        // ---- this warp's unselected columns
        for (int c = warp; c < nc; c += kResWarps) {
            if (c == cp || sel_s[c]) continue;
            T* x = xs + static_cast<int64_t>(c) * r;
            T s0 = 0, s1 = 0;
            int64_t t = j + lane;
            for (; t + 32 < r; t += 64) {
                s0 = fma(xp[t], x[t], s0);
                s1 = fma(xp[t + 32], x[t + 32], s1);
            }
            if (t < r) s0 = fma(xp[t], x[t], s0);
            T S = warp_sum(s0 + s1);
            const T X = x[j];
            S = fma(-beta, X, S);
            const T tw = -S * rbeta;
            const T sv = tw * inv;
            if (lane == 0) P.R[(c0 + c) * P.ldr + j] = to_f64(X - tw);
            T q0 = 0, q1 = 0;
            t = j + 1 + lane;
            for (; t + 32 < r; t += 64) {
                const T a0 = fma(-sv, xp[t], x[t]);
                const T a1 = fma(-sv, xp[t + 32], x[t + 32]);
                x[t] = a0;
                x[t + 32] = a1;
                q0 = fma(a0, a0, q0);
                q1 = fma(a1, a1, q1);
            }
            if (t < r) {
                const T a0 = fma(-sv, xp[t], x[t]);
                x[t] = a0;
                q0 = fma(a0, a0, q0);
            }
            const T nu = warp_sum(q0 + q1);
            if (lane == 0) nu_s[c] = nu;
        }
        __syncwarp();
        publish(j + 1);
        k = j + 1;
    }
    if (go < 0) {
        if (tid == 0) set_info(P.info, kInfoWatchdog);
        return;
    }
    if (b == 0) {
        // after the last step, CTA 0 waits for the final table too: every pivot's flag
        // (written before its owner's next record) is then visible to the listing
        if (go == 1) {
            if (warp == 0) decide(k, true);
            __syncthreads();
            if (s_go < 0) {
                if (tid == 0) set_info(P.info, kInfoWatchdog);
                return;
            }
        }
        list_complement(P.J, P.sel, P.n, k, P.k_out, cnt);
    }
}

template <typename T>
cudaError_t launch_cpqr_resident(const CpqrParams<T>& P, int grid, size_t smem, cudaStream_t s) {
    if (grid > 32 * kTableLanes) return cudaErrorInvalidValue;
    auto kern = k_cpqr_resident<T>;
    if (smem > 48 * 1024) {
        const cudaError_t e =
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    // clear the stamps of both table slots: a record of this launch is recognised by them
    cudaError_t e = cudaMemsetAsync(P.cand, 0, 2 * static_cast<size_t>(grid) * sizeof(Cand), s);
    if (e != cudaSuccess) return e;
    CpqrParams<T> Pc = P;
    void* args[] = {&Pc};
    return cudaLaunchCooperativeKernel(reinterpret_cast<void*>(kern), dim3(grid), dim3(kResWarps * 32), args, smem,
                                       s);
}

template cudaError_t launch_cpqr_resident<double>(const CpqrParams<double>&, int, size_t, cudaStream_t);
template cudaError_t launch_cpqr_resident<float>(const CpqrParams<float>&, int, size_t, cudaStream_t);

}  // namespace gid
