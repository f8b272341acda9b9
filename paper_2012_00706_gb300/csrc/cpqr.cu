// Truncated column-pivoted Householder QR (Sec. 1.1, Algorithm 1, the pivoted QR) of a
// tall or wide matrix on one cooperative grid.
//
// Greedy Businger-Golub pivoting: step j picks the unselected column with the
// largest residual norm, builds the Householder reflector that maps its residual
// x_p(j:r) to beta e_1 (beta = -sign(alpha) ||x_p(j:r)||, alpha = x_p(j)), applies it
// to the other unselected columns and records row j of R.  Column norms are
// downdated, nu_i <- nu_i - R(j,i)^2, and recomputed exactly when the
// Drmac-Bujanovic cancellation test fires.
//
// With v = (1, x_p(j+1:r) / (alpha - beta)) and tau = (beta - alpha) / beta the
// reflector applied to column i is x_i -= tau (v^T x_i) v.  Writing
// S_i = x_p(j:r)^T x_i(j:r) - beta x_i(j), it is
//     tw_i = tau v^T x_i = -S_i / beta,   R(j,i) = x_i(j) - tw_i,
//     x_i(t) -= (tw_i / (alpha - beta)) x_p(t)   for t > j,
// so the pivot column itself, unscaled, is all a step needs besides two scalars.
//
// CTA b owns the contiguous column slice [n b / G, n (b + 1) / G) of the working copy
// in global memory and updates it in place, in one of two modes fixed per launch.  Column
// mode (a warp per column): dot product, scalars and update of a column by one warp with
// no CTA barrier.  Row mode (fewer columns than warps, all threads splitting the rows with
// several loads in flight per thread): each column stays one update behind, and one pass
// per step applies the previous step's update and forms this step's dot products S_i, with
// the pivot column brought up to date on the fly.  The CTA then publishes its best
// remaining candidate (norm, index, sum of norms, and the candidate's exact squared norm
// and next-row entry, the reflector scalars of the next step); after one bounded grid
// barrier every CTA reduces the same candidate table in the same order, on integer keys
// of the norms' bits, and agrees on the next pivot.  Matrices whose columns fit the
// grid's shared memory go to the resident kernel instead (cpqr_resident.cu).
#include "cpqr_grid.cuh"

#include <algorithm>

namespace gid {

constexpr int kGridThreads = 512;
constexpr int kGridWarps = kGridThreads / 32;
constexpr int kSuper = 256;                  // columns whose dot products share one CTA barrier
// columns of one pass over the rows, and rows per thread unrolled: 32 loads in flight
template <typename T> struct ColGroup;
template <> struct ColGroup<double> { static constexpr int cols = 8, unroll = 4; };
template <> struct ColGroup<float> { static constexpr int cols = 16, unroll = 2; };
constexpr size_t kResidentSmem = 200 * 1024; // shared memory for resident columns

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

// argmax of pivot keys (norm_bits_key) with ties to the smaller index and, when with_sum,
// a sum, in one pass (three barriers); returns to all threads.  The keys compare on the
// integer pipe, so a step's reductions need no FP64 instruction unless sums are asked for.
__device__ void block_argmax_key(uint64_t key, int idx, bool with_sum, double part, uint64_t* shk, int* shi,
                                 double* shp, uint64_t* outk, int* outi, double* outp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (!key) idx = -1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t ok = __shfl_xor_sync(0xffffffffu, key, o);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (with_sum) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (ok > key || (ok == key && oi >= 0 && (idx < 0 || oi < idx))) { key = ok; idx = oi; }
    }
    __syncthreads();
    if (lane == 0) { shk[warp] = key; shi[warp] = idx; shp[warp] = part; }
    __syncthreads();
    if (warp == 0) {
        key = lane < nw ? shk[lane] : 0ull;
        idx = lane < nw ? shi[lane] : -1;
        part = lane < nw ? shp[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const uint64_t ok = __shfl_xor_sync(0xffffffffu, key, o);
            const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
            if (with_sum) part += __shfl_xor_sync(0xffffffffu, part, o);
            if (ok > key || (ok == key && oi >= 0 && (idx < 0 || oi < idx))) { key = ok; idx = oi; }
        }
        if (lane == 0) { shk[32] = key; shi[32] = idx; shp[32] = part; }
    }
    __syncthreads();
    *outk = shk[32];
    *outi = shi[32];
    *outp = shp[32];
}

// Per-CTA state in shared memory (static part).
template <typename T>
struct GridShared {
    double shv[33];
    int shi[33];
    T shs[33];
    double shp[33];
    int ok;
    int p, pg;
    double alpha, s2, sumnu, total, sv_p;
};

// Dynamic shared memory of a CTA: residual norms, reference norms and (column mode) exact
// squared norms below the step's row of its (at most cpb) columns, the per-warp partial sums and reflector scalars of one super-group of
// min(cpb, kSuper) columns, the staged pivot column (rstage rows, column mode), the
// super-group's recompute flags, and the columns' selection flags.
__host__ __device__ inline int64_t grid_super(int64_t cpb) { return cpb < kSuper ? cpb : kSuper; }
// The staged pivot column comes first (16-byte aligned for vector reads), rounded up to 16 bytes.
__host__ __device__ inline int64_t grid_rstage_padded(int64_t rstage, int elem_bytes) {
    const int64_t per = 16 / elem_bytes;
    return (rstage + per - 1) / per * per;
}
template <typename T>
__host__ __device__ inline size_t grid_smem_bytes(int64_t cpb, int64_t rstage) {
    const size_t sup = static_cast<size_t>(grid_super(cpb));
    return (3 * static_cast<size_t>(cpb) + (kGridWarps + 1) * sup +
            static_cast<size_t>(grid_rstage_padded(rstage, sizeof(T)))) * sizeof(T) +
           sup * sizeof(int) + ((static_cast<size_t>(cpb) + 15) & ~size_t(15));
}

// 16-byte vectors of the column mode's vector path.
template <typename T> struct Vec16;
template <> struct Vec16<float> {
    using V = float4;
    static constexpr int E = 4;
    static __device__ __forceinline__ float dot(const float4 a, const float4 b, float s) {
        return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, fmaf(a.x, b.x, s))));
    }
    static __device__ __forceinline__ float4 axpy(float m, const float4 p, const float4 x) {
        return make_float4(fmaf(m, p.x, x.x), fmaf(m, p.y, x.y), fmaf(m, p.z, x.z), fmaf(m, p.w, x.w));
    }
    static __device__ __forceinline__ float sq(const float4 a, float s) { return dot(a, a, s); }
    static __device__ __forceinline__ void zero_first(float4& a) { a.x = 0.f; }
    static __device__ __forceinline__ float4 ldcg(const float* p) { return __ldcg(reinterpret_cast<const float4*>(p)); }
};
template <> struct Vec16<double> {
    using V = double2;
    static constexpr int E = 2;
    static __device__ __forceinline__ double dot(const double2 a, const double2 b, double s) {
        return fma(a.y, b.y, fma(a.x, b.x, s));
    }
    static __device__ __forceinline__ double2 axpy(double m, const double2 p, const double2 x) {
        return make_double2(fma(m, p.x, x.x), fma(m, p.y, x.y));
    }
    static __device__ __forceinline__ double sq(const double2 a, double s) { return dot(a, a, s); }
    static __device__ __forceinline__ void zero_first(double2& a) { a.x = 0.0; }
    static __device__ __forceinline__ double2 ldcg(const double* p) {
        return __ldcg(reinterpret_cast<const double2*>(p));
    }
};

// Column mode (a warp per column, no CTA barrier inside a step) when every warp has a
// column; the pivot column is staged in shared memory when it takes at most 64 KB.
constexpr size_t kStageBytes = 64 * 1024;
inline bool grid_colmode(int64_t cpb) { return cpb >= kGridWarps; }
inline int64_t grid_rstage(int64_t cpb, int64_t r, int elem_bytes) {
    return grid_colmode(cpb) && static_cast<size_t>(r) * elem_bytes <= kStageBytes ? r : 0;
}

// The pivoted QR of one matrix by the G CTAs b = 0..G-1 (a whole grid, or one group of a
// grouped launch).
template <typename T, bool COLMODE>
__device__ __forceinline__ void cpqr_grid_body(const CpqrParams<T>& P, const int G, const int b, GridShared<T>& G_,
                                               uint8_t* smem_dyn) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int64_t c0 = P.n * b / G, c1 = P.n * (b + 1) / G;
    const int nc = static_cast<int>(c1 - c0);
    const int64_t r = P.r;
    const T sqrt_u = SqrtU<T>::v();
    const int sup = static_cast<int>(grid_super(P.cpb_max));
    const bool tol_mode = P.rel_tol > 0.0;     // sums of norms are formed only for the tolerance test
    uint64_t* const shk = reinterpret_cast<uint64_t*>(G_.shv);
    if ((P.colmode != 0) != COLMODE || (!COLMODE && !P.pub)) {
        // the parameters name the other mode, or row mode lacks its pivot-column slots (every
        // CTA of the matrix sees the same parameters and leaves before the first grid barrier)
        if (b == 0 && tid == 0) set_info(P.info, kInfoBadTable);
        return;
    }
    T* xps_s = reinterpret_cast<T*>(smem_dyn);  // [rstage] staged pivot column (column mode)
    T* nu_s = xps_s + grid_rstage_padded(P.rstage, sizeof(T));
    T* nuref_s = nu_s + P.cpb_max;
    T* s2_s = nuref_s + P.cpb_max;              // column mode: exact ||x(j+1:r)||^2 after step j
    T* red_s = s2_s + P.cpb_max;                // [kGridWarps][sup]
    T* sv_s = red_s + kGridWarps * sup;
    int* rec_s = reinterpret_cast<int*>(sv_s + sup);
    uint8_t* sel_s = reinterpret_cast<uint8_t*>(rec_s + sup);
    uint32_t epoch = 0;

    // column c (local index) of the slice in the global working copy (the parameters may
    // sit in shared memory, where stores through X could alias them: keep them local)
    T* const Xs = P.X + c0 * P.ldx;
    const int64_t ldx = P.ldx;
    auto col = [&](int c) -> T* { return Xs + c * ldx; };

    // ---- init: copy the slice into the working copy (or take it there), exact squared norms
    T local_total = 0;
    bool bad = false;
    for (int c = 0; c < nc; ++c) {
        T* x = col(c);
        T s = 0;
#pragma unroll 8
        for (int64_t t = tid; t < r; t += nt) {
            T a;
            if (P.src) {
                a = P.src_f64 ? static_cast<T>(static_cast<const double*>(P.src)[(c0 + c) * P.ldsrc + t])
                              : static_cast<T>(static_cast<const float*>(P.src)[(c0 + c) * P.ldsrc + t]);
                x[t] = a;
            } else {
                a = x[t];
            }
            s += a * a;
        }
        s = block_sum(s, G_.shs);
        if (tid == 0) {
            if (!isfinite(static_cast<double>(s))) bad = true;
            nu_s[c] = s;
            nuref_s[c] = s;
            s2_s[c] = s;
            sel_s[c] = 0;
            P.sel[c0 + c] = 0;
            local_total += s;
        }
    }
    if (bad) set_info(P.info, kInfoNonFinite);

    // Row mode keeps each column one update behind: step j's update is applied by step j + 1's
    // pass.  The pivot column of step j brought up to date at row t is
    // fma(-sv_p, xprev[t], xq[t]) (xq: its stored copy, xprev: step j - 1's pivot column,
    // kept in pub by its owner); candidates read after step j add their own pending update.
    const T* pf_xq = nullptr;
    const T* pf_xprev = nullptr;
    T pf_msvp = 0;
    bool pf_pend = false;
    auto pivot_at = [&](int64_t t) -> T {
        const T q = __ldcg(pf_xq + t);
        return pf_pend ? fma(pf_msvp, __ldcg(pf_xprev + t), q) : q;
    };

    // ---- publish this slice's best candidate for the step with row `row` (exact squared
    // norm of its rows row..r-1, its entry on row `row`; `lagging`: row mode after a step,
    // whose update the candidate's values take on the fly)
    auto publish = [&](int slot, int row, double total, bool lagging) {
        uint64_t bestk = 0ull;
        int bi = -1;
        T part = 0;
        for (int c = tid; c < nc; c += nt) {
            if (sel_s[c]) continue;
            const T v = nu_s[c];
            if (tol_mode) part += v;
            const uint64_t key = norm_bits_key(v);
            if (key > bestk) { bestk = key; bi = c; }      // c ascends: ties keep the smaller
        }
        uint64_t bk;
        double sumd;
        int bl;
        block_argmax_key(bestk, bi, tol_mode, tol_mode ? to_f64(part) : 0.0, shk, G_.shi, G_.shp, &bk, &bl, &sumd);
        const double bv = key_norm_f64(bk, T(0));
        T s2 = 0;
        T alpha = 0;
        if (COLMODE && bl >= 0 && row < r) {
            // column mode: the exact norm below the row, left by the column's warp
            s2 = s2_s[bl];
            alpha = col(bl)[row];
        } else if (bl >= 0 && row < r && lagging) {
            // as below, on the values after the pending update
            const T* x = col(bl);
            const T msv = -sv_s[bl];
            auto cur = [&](int64_t t) { return fma(msv, pivot_at(t), x[t]); };
            T sa[8] = {};
            int64_t t = row + tid;
            for (; t + 7 * nt < r; t += 8 * nt) {
                T a[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) a[u] = cur(t + u * nt);
#pragma unroll
                for (int u = 0; u < 8; ++u) sa[u] = fma(a[u], a[u], sa[u]);
            }
            for (; t < r; t += nt) {
                const T a = cur(t);
                sa[0] = fma(a, a, sa[0]);
            }
            const T s = ((sa[0] + sa[1]) + (sa[2] + sa[3])) + ((sa[4] + sa[5]) + (sa[6] + sa[7]));
            s2 = block_sum(s, G_.shs);
            alpha = cur(row);
        } else if (bl >= 0 && row < r) {
            // the candidate's exact squared norm: eight independent sums keep eight loads in
            // flight per thread (this pass is on every step's critical path)
            const T* x = col(bl);
            T sa[8] = {};
            int64_t t = row + tid;
            for (; t + 7 * nt < r; t += 8 * nt) {
                T a[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) a[u] = x[t + u * nt];
#pragma unroll
                for (int u = 0; u < 8; ++u) sa[u] = fma(a[u], a[u], sa[u]);
            }
            for (; t < r; t += nt) sa[0] = fma(x[t], x[t], sa[0]);
            const T s = ((sa[0] + sa[1]) + (sa[2] + sa[3])) + ((sa[4] + sa[5]) + (sa[6] + sa[7]));
            s2 = block_sum(s, G_.shs);
            alpha = x[row];
        }
        if (tid == 0) {
            Cand cd;
            cd.nu = bv;
            cd.sumnu = tol_mode ? to_f64(static_cast<T>(sumd)) : 0.0;
            cd.total = total;
            cd.s2 = to_f64(s2);
            cd.alpha = to_f64(alpha);
            cd.sv = (lagging && bl >= 0) ? to_f64(sv_s[bl]) : 0.0;
            cd.idx = bl >= 0 ? static_cast<int>(c0 + bl) : -1;
            cd.stamp = 0;
            P.cand[slot * G + b] = cd;
        }
    };

    {
        const T tot = block_sum(tid == 0 ? local_total : T(0), G_.shs);
        publish(0, 0, static_cast<double>(tot), false);
    }
    bool ok = grid_barrier(&P.ctrl->counter, epoch, &P.ctrl->abort, P.limit_ns, &G_.ok,
                           static_cast<uint32_t>(G));

    int k = 0;
    double total = 0.0;
    for (int j = 0; ok && j < P.kcap; ++j) {
        const int slot = j & 1;
        // ---- global pivot: identical reduction of the candidate table in every CTA
        {
            uint64_t bk = 0ull;
            double sn = 0.0, tt = 0.0;
            int bg = -1;
            for (int g = tid; g < G; g += nt) {
                const Cand c = load_cand(P.cand + slot * G + g);
                const uint64_t key = c.idx >= 0 ? norm_bits_key(c.nu) : 0ull;
                if (key > bk) { bk = key; bg = g; }          // g ascends: ties keep the smaller CTA
                if (tol_mode) {
                    sn += c.sumnu;
                    tt += c.total;
                }
            }
            uint64_t gk;
            double gsn;
            int gg;
            block_argmax_key(bk, bg, tol_mode, sn, shk, G_.shi, G_.shp, &gk, &gg, &gsn);
            double gv = -1.0;
            const double gtt = (j == 0 && tol_mode) ? block_sum(tt, G_.shv) : 0.0;
            if (tid == 0) {
                G_.pg = gg;
                G_.p = -1;
                if (gg >= 0) {
                    const Cand w = load_cand(P.cand + slot * G + gg);
                    G_.p = w.idx;
                    G_.alpha = w.alpha;
                    G_.s2 = w.s2;
                    G_.sv_p = w.sv;
                    gv = w.nu;
                }
                G_.shv[32] = gv;
                G_.sumnu = gsn;
                if (j == 0) G_.total = gtt;
            }
            __syncthreads();
        }
        if (j == 0) total = G_.total;
        const int p = G_.p;
        const double best = G_.shv[32];
        if (tol_mode && sqrt(fmax(G_.sumnu, 0.0)) <= P.rel_tol * sqrt(total)) break;
        if (p < 0 || !positive_bits(best) || !positive_bits(G_.s2)) {
            if (b == 0 && tid == 0) set_info(P.info, j + 1);
            break;
        }
        // ---- reflector scalars (the pivot column is not modified in this step)
        const T alpha = narrow_exact(G_.alpha, T(0));
        const T snorm = sqrt(narrow_exact(G_.s2, T(0)));
        const T beta = alpha >= T(0) ? -snorm : snorm;
        const T rb = T(1) / beta;
        const T inv = T(1) / (alpha - beta);
        const T* xp = P.X + p * P.ldx;
        if (p >= c0 && p < c1 && tid == 0) {
            sel_s[p - c0] = 1;
            P.sel[p] = 1;
            P.J[j] = p;
            P.R[static_cast<int64_t>(p) * P.ldr + j] = to_f64(beta);
        }
        __syncthreads();
        if constexpr (COLMODE) {
            // ---- column mode: warp w takes columns w, w + 16, ...; per column the dot
            // product (one warp reduction), the reflector scalars, the update and, where the
            // downdate is refused, the exact squared norm, with no CTA barrier in between
            // xp(t): the staged copy, or L2 (the column was written by another CTA)
            auto run_cols = [&](auto xpv) {
                for (int c = warp; c < nc; c += kGridWarps) {
                    if (sel_s[c]) continue;
                    T* x = col(c);
                    T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
                    int64_t t = j + lane;
                    for (; t + 96 < r; t += 128) {
                        s0 = fma(xpv(t), x[t], s0);
                        s1 = fma(xpv(t + 32), x[t + 32], s1);
                        s2 = fma(xpv(t + 64), x[t + 64], s2);
                        s3 = fma(xpv(t + 96), x[t + 96], s3);
                    }
                    for (; t < r; t += 32) s0 = fma(xpv(t), x[t], s0);
                    T sdot = warp_sum((s0 + s1) + (s2 + s3));
                    const T X = x[j];
                    sdot = fma(-beta, X, sdot);
                    const T tw = -sdot * rb;
                    const T sv = tw * inv;
                    const T rho = X - tw;
                    const T nu = nu_s[c];
                    bool rec = false;
                    T d = nu;
                    if (nu > T(0)) {
                        d = fmax(nu - rho * rho, T(0));
                        rec = d <= sqrt_u * nuref_s[c];
                    }
                    __syncwarp();
                    if (lane == 0) {
                        P.R[(c0 + c) * P.ldr + j] = to_f64(rho);
                        if (nu > T(0) && !rec) nu_s[c] = d;
                    }
                    const T msv = -sv;
                    T q0 = 0, q1 = 0;
                    t = j + 1 + lane;
                    for (; t + 32 < r; t += 64) {
                        const T n0 = fma(msv, xpv(t), x[t]);
                        const T n1 = fma(msv, xpv(t + 32), x[t + 32]);
                        x[t] = n0;
                        x[t + 32] = n1;
                        q0 = fma(n0, n0, q0);
                        q1 = fma(n1, n1, q1);
                    }
                    for (; t < r; t += 32) {
                        const T n0 = fma(msv, xpv(t), x[t]);
                        x[t] = n0;
                        q0 = fma(n0, n0, q0);
                    }
                    // the exact squared norm below row j, for this step's record and, where
                    // the downdate was refused, as the new norm
                    const T sq = warp_sum(q0 + q1);
                    if (lane == 0) {
                        s2_s[c] = sq;
                        if (rec) {
                            nu_s[c] = sq;
                            nuref_s[c] = sq;
                        }
                    }
                }
            };
            // the same column work with 16-byte vectors (columns 16-byte aligned): a scalar head
            // up to the first aligned row, vectors, a scalar tail; several vectors in flight
            using VT = Vec16<T>;
            using V = typename VT::V;
            constexpr int E = VT::E;
            auto run_cols_vec = [&](auto xpv, auto xpw) {
                const int64_t hd = min(r, (static_cast<int64_t>(j) + E - 1) / E * E);
                const int64_t rd = hd + (r - hd) / E * E;
                const int64_t hu = min(r, (static_cast<int64_t>(j) + E) / E * E);     // after row j
                const int64_t ru = hu + (r - hu) / E * E;
                for (int c = warp; c < nc; c += kGridWarps) {
                    if (sel_s[c]) continue;
                    T* x = col(c);
                    T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
                    if (j + lane < hd) s0 = xpv(j + lane) * x[j + lane];
                    if (rd + lane < r) s1 = xpv(rd + lane) * x[rd + lane];
                    {
                        const V* xv = reinterpret_cast<const V*>(x + hd);
                        const int64_t nv = (rd - hd) / E;
                        int64_t v = lane;
                        for (; v + 224 < nv; v += 256) {
                            V a[8], q[8];
#pragma unroll
                            for (int u = 0; u < 8; ++u) {
                                a[u] = xv[v + 32 * u];
                                q[u] = xpw(hd + (v + 32 * u) * E);
                            }
                            s0 = VT::dot(a[0], q[0], s0);
                            s1 = VT::dot(a[1], q[1], s1);
                            s2 = VT::dot(a[2], q[2], s2);
                            s3 = VT::dot(a[3], q[3], s3);
                            s0 = VT::dot(a[4], q[4], s0);
                            s1 = VT::dot(a[5], q[5], s1);
                            s2 = VT::dot(a[6], q[6], s2);
                            s3 = VT::dot(a[7], q[7], s3);
                        }
                        for (; v < nv; v += 32) s0 = VT::dot(xv[v], xpw(hd + v * E), s0);
                    }
                    T sdot = warp_sum((s0 + s1) + (s2 + s3));
                    const T X = x[j];
                    sdot = fma(-beta, X, sdot);
                    const T tw = -sdot * rb;
                    const T sv = tw * inv;
                    const T rho = X - tw;
                    const T nu = nu_s[c];
                    bool rec = false;
                    T d = nu;
                    if (nu > T(0)) {
                        d = fmax(nu - rho * rho, T(0));
                        rec = d <= sqrt_u * nuref_s[c];
                    }
                    __syncwarp();
                    if (lane == 0) {
                        P.R[(c0 + c) * P.ldr + j] = to_f64(rho);
                        if (nu > T(0) && !rec) nu_s[c] = d;
                    }
                    const T msv = -sv;
                    T q0 = 0, q1 = 0;
                    if (j + 1 + lane < hu) {
                        const int64_t t = j + 1 + lane;
                        const T n0 = fma(msv, xpv(t), x[t]);
                        x[t] = n0;
                        q0 = n0 * n0;
                    }
                    if (ru + lane < r) {
                        const int64_t t = ru + lane;
                        const T n0 = fma(msv, xpv(t), x[t]);
                        x[t] = n0;
                        q1 = n0 * n0;
                    }
                    {
                        V* xv = reinterpret_cast<V*>(x + hu);
                        const int64_t nv = (ru - hu) / E;
                        int64_t v = lane;
                        for (; v + 96 < nv; v += 128) {
                            V a[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u) a[u] = VT::axpy(msv, xpw(hu + (v + 32 * u) * E), xv[v + 32 * u]);
#pragma unroll
                            for (int u = 0; u < 4; ++u) xv[v + 32 * u] = a[u];
                            q0 = VT::sq(a[0], q0);
                            q1 = VT::sq(a[1], q1);
                            q0 = VT::sq(a[2], q0);
                            q1 = VT::sq(a[3], q1);
                        }
                        for (; v < nv; v += 32) {
                            const V a = VT::axpy(msv, xpw(hu + v * E), xv[v]);
                            xv[v] = a;
                            q0 = VT::sq(a, q0);
                        }
                    }
                    // the exact squared norm below row j, for this step's record and, where
                    // the downdate was refused, as the new norm
                    const T sq = warp_sum(q0 + q1);
                    if (lane == 0) {
                        s2_s[c] = sq;
                        if (rec) {
                            nu_s[c] = sq;
                            nuref_s[c] = sq;
                        }
                    }
                }
            };
            // short FP32 columns (at most 16 vectors per lane): the column is read once into
            // registers during the dot product and updated from there, one read and one write
            // per step
            constexpr int NVR = 16;
            auto run_cols_reg = [&](auto xpv, auto xpw) {
                const int64_t hd = min(r, (static_cast<int64_t>(j) + E - 1) / E * E);
                const int64_t rd = hd + (r - hd) / E * E;
                const int64_t nv = (rd - hd) / E;
                for (int c = warp; c < nc; c += kGridWarps) {
                    if (sel_s[c]) continue;
                    T* x = col(c);
                    V* xv = reinterpret_cast<V*>(x + hd);
                    V xr[NVR];
                    T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
#pragma unroll
                    for (int u = 0; u < NVR; ++u) {
                        const int64_t v = lane + 32 * u;
                        if (v < nv) xr[u] = xv[v];
                    }
#pragma unroll
                    for (int u = 0; u < NVR; ++u) {
                        const int64_t v = lane + 32 * u;
                        if (v < nv) {
                            const V q = xpw(hd + v * E);
                            if ((u & 3) == 0) s0 = VT::dot(xr[u], q, s0);
                            else if ((u & 3) == 1) s1 = VT::dot(xr[u], q, s1);
                            else if ((u & 3) == 2) s2 = VT::dot(xr[u], q, s2);
                            else s3 = VT::dot(xr[u], q, s3);
                        }
                    }
                    // the scalar head rows [j, hd) and tail rows [rd, r)
                    const int64_t th = j + lane, tt = rd + lane;
                    const bool in_h = th < hd, in_t = tt < r;
                    const T xh = in_h ? x[th] : T(0), xt = in_t ? x[tt] : T(0);
                    if (in_h) s0 = fma(xpv(th), xh, s0);
                    if (in_t) s1 = fma(xpv(tt), xt, s1);
                    T sdot = warp_sum((s0 + s1) + (s2 + s3));
                    const T X = x[j];
                    sdot = fma(-beta, X, sdot);
                    const T tw = -sdot * rb;
                    const T sv = tw * inv;
                    const T rho = X - tw;
                    const T nu = nu_s[c];
                    bool rec = false;
                    T d = nu;
                    if (nu > T(0)) {
                        d = fmax(nu - rho * rho, T(0));
                        rec = d <= sqrt_u * nuref_s[c];
                    }
                    __syncwarp();
                    if (lane == 0) {
                        P.R[(c0 + c) * P.ldr + j] = to_f64(rho);
                        if (nu > T(0) && !rec) nu_s[c] = d;
                    }
                    const T msv = -sv;
                    T q0 = 0, q1 = 0;
                    // rows above j + 1 leave the computation: row j is set to zero (its R entry is
                    // out), so that the recomputed norm covers rows j + 1 .. r - 1 only
                    if (in_h) {
                        const T n0 = th == j ? T(0) : fma(msv, xpv(th), xh);
                        x[th] = n0;
                        q0 = n0 * n0;
                    }
                    if (in_t) {
                        const T n0 = fma(msv, xpv(tt), xt);
                        x[tt] = n0;
                        q1 = n0 * n0;
                    }
#pragma unroll
                    for (int u = 0; u < NVR; ++u) {
                        const int64_t v = lane + 32 * u;
                        if (v < nv) {
                            V a = VT::axpy(msv, xpw(hd + v * E), xr[u]);
                            if (u == 0 && lane == 0 && hd == j) VT::zero_first(a);
                            xv[v] = a;
                            q0 = VT::sq(a, q0);
                        }
                    }
                    // the exact squared norm below row j, for this step's record and, where
                    // the downdate was refused, as the new norm
                    const T sq = warp_sum(q0 + q1);
                    if (lane == 0) {
                        s2_s[c] = sq;
                        if (rec) {
                            nu_s[c] = sq;
                            nuref_s[c] = sq;
                        }
                    }
                }
            };
            const bool vec = (ldx * static_cast<int64_t>(sizeof(T))) % 16 == 0 &&
                             (reinterpret_cast<uintptr_t>(Xs) & 15u) == 0;
            if (P.rstage > 0) {
                for (int64_t t = j + tid; t < r; t += nt) xps_s[t] = __ldcg(xp + t);
                __syncthreads();
                bool reg = false;
                if constexpr (sizeof(T) == 4) reg = vec && r - j <= static_cast<int64_t>(32) * NVR * E;
                if (reg) {
                    if constexpr (sizeof(T) == 4)
                        run_cols_reg([&](int64_t t) { return xps_s[t]; },
                                     [&](int64_t t) { return *reinterpret_cast<const V*>(xps_s + t); });
                } else if (vec)
                    run_cols_vec([&](int64_t t) { return xps_s[t]; },
                                 [&](int64_t t) { return *reinterpret_cast<const V*>(xps_s + t); });
                else
                    run_cols([&](int64_t t) { return xps_s[t]; });
            } else {
                if (vec && (reinterpret_cast<uintptr_t>(xp) & 15u) == 0)
                    run_cols_vec([&](int64_t t) { return __ldcg(xp + t); }, [&](int64_t t) { return VT::ldcg(xp + t); });
                else
                    run_cols([&](int64_t t) { return __ldcg(xp + t); });
            }
            __syncthreads();
        } else {
        // ---- row mode (fewer columns than warps: all threads split the rows).  One pass over
        // rows j..r-1 applies step j - 1's update to the slice's unselected columns (their
        // coefficients in sv_s, step j - 1's pivot column from pub) and forms this step's dot
        // products S_c = x_p(j:r)^T x_c(j:r) with the pivot column brought up to date on the
        // fly; the pivot's owner keeps that column in pub for step j + 1.  One barrier, the
        // reflector scalars (this step's update coefficients replace the applied ones), and the
        // exact norms where the downdate was refused.  Step j's update waits for step j + 1's
        // pass: a column is read and written once per step.
        constexpr int CG = ColGroup<T>::cols;
        constexpr int UR = ColGroup<T>::unroll;
        const bool pend = j > 0;
        pf_xq = xp;
        pf_xprev = P.pub + static_cast<int64_t>((j + 1) & 1) * r;     // step j - 1's slot
        pf_msvp = pend ? -narrow_exact(G_.sv_p, T(0)) : T(0);
        pf_pend = pend;
        T* const xcur = P.pub + static_cast<int64_t>(j & 1) * r;
        const bool own_p = p >= c0 && p < c1;
        for (int g0 = 0; g0 < nc; g0 += CG) {
            const int gn = min(CG, nc - g0);
            bool act[CG];
            T* xc[CG];
            T msv[CG], S[CG];
#pragma unroll
            for (int q = 0; q < CG; ++q) {
                act[q] = q < gn && !sel_s[g0 + q];
                xc[q] = col(min(g0 + q, nc - 1));
                msv[q] = (act[q] && pend) ? -sv_s[g0 + q] : T(0);
                S[q] = 0;
            }
            const bool keep = own_p && g0 == 0;
            bool any = keep;
#pragma unroll
            for (int q = 0; q < CG; ++q) any |= act[q];
            if (!any) continue;     // every column of the group is selected: nothing reads its sums
#pragma unroll UR
            for (int64_t t = j + tid; t < r; t += nt) {
                const T pp = pend ? __ldcg(pf_xprev + t) : T(0);
                const T q0 = __ldcg(xp + t);
                const T pv = pend ? fma(pf_msvp, pp, q0) : q0;
                if (keep) xcur[t] = pv;
#pragma unroll
                for (int q = 0; q < CG; ++q) {
                    if (act[q]) {
                        T v = xc[q][t];
                        if (pend) {
                            v = fma(msv[q], pp, v);
                            xc[q][t] = v;
                        }
                        S[q] = fma(pv, v, S[q]);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < CG; ++q) {
                const T v = warp_sum(S[q]);
                if (lane == 0 && q < gn) red_s[warp * sup + g0 + q] = v;
            }
        }
        __syncthreads();
        for (int c = tid; c < nc; c += nt) {
            T sv = 0;
            int rec = 0;
            if (!sel_s[c]) {
                T s = 0;
                for (int w = 0; w < kGridWarps; ++w) s += red_s[w * sup + c];
                const T X = col(c)[j];
                s = fma(-beta, X, s);
                const T tw = -s * rb;
                sv = tw * inv;
                const T rho = X - tw;
                P.R[(c0 + c) * P.ldr + j] = to_f64(rho);
                // downdate; an exact recompute where cancellation has eaten sqrt(u)
                const T nu = nu_s[c];
                if (nu > T(0)) {
                    const T d = fmax(nu - rho * rho, T(0));
                    if (d <= sqrt_u * nuref_s[c]) rec = 1;
                    else nu_s[c] = d;
                }
            }
            sv_s[c] = sv;
            rec_s[c] = rec;
        }
        __syncthreads();
        // the refused downdates: exact squared norms of x_c(j+1:r) after this step's update
        // (rare; the values are taken on the fly like the candidate's below)
        bool any_rec = false;
        for (int c = 0; c < nc; ++c) any_rec |= rec_s[c] != 0;
        if (any_rec) {
            for (int g0 = 0; g0 < nc; g0 += CG) {
                const int gn = min(CG, nc - g0);
                bool act[CG];
                const T* xc[CG];
                T msv[CG], sq[CG];
                bool grp = false;
#pragma unroll
                for (int q = 0; q < CG; ++q) {
                    act[q] = q < gn && rec_s[g0 + q] != 0;
                    xc[q] = col(min(g0 + q, nc - 1));
                    msv[q] = act[q] ? -sv_s[g0 + q] : T(0);
                    grp |= act[q];
                    sq[q] = 0;
                }
                if (!grp) continue;
#pragma unroll UR
                for (int64_t t = j + 1 + tid; t < r; t += nt) {
                    const T pv = pivot_at(t);
#pragma unroll
                    for (int q = 0; q < CG; ++q) {
                        if (act[q]) {
                            const T nx = fma(msv[q], pv, xc[q][t]);
                            sq[q] = fma(nx, nx, sq[q]);
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < CG; ++q) {
                    const T v = warp_sum(sq[q]);
                    if (lane == 0 && q < gn) red_s[warp * sup + g0 + q] = v;
                }
            }
            __syncthreads();
            for (int c = tid; c < nc; c += nt) {
                if (!rec_s[c]) continue;
                T s = 0;
                for (int w = 0; w < kGridWarps; ++w) s += red_s[w * sup + c];
                nu_s[c] = s;
                nuref_s[c] = s;
            }
            __syncthreads();
        }
        }
        publish(slot ^ 1, j + 1, 0.0, !COLMODE);
        ok = grid_barrier(&P.ctrl->counter, epoch, &P.ctrl->abort, P.limit_ns, &G_.ok,
                           static_cast<uint32_t>(G));
        k = j + 1;
    }
    if (!ok) {
        if (tid == 0) set_info(P.info, kInfoWatchdog);
        return;
    }
    if (b == 0) list_complement(P.J, P.sel, P.n, k, P.k_out, G_.shi);
}

// COLMODE: the slice's mode (a warp per column, or the rows split over all threads),
// fixed per launch so that each mode's registers are allocated on their own.
template <typename T, bool COLMODE>
__global__ void __launch_bounds__(kGridThreads) k_cpqr_grid(const CpqrParams<T> P) {
    extern __shared__ __align__(16) uint8_t smem_dyn[];
    __shared__ GridShared<T> G_;
    cpqr_grid_body<T, COLMODE>(P, static_cast<int>(gridDim.x), static_cast<int>(blockIdx.x), G_, smem_dyn);
}

// Grouped launch: CTAs [g gsize, (g + 1) gsize) factor the matrix of groups[g] on their own,
// with the group's own candidate table and barrier counter.  The launch is cooperative, so
// every group is resident at once and its barrier waits only on its own CTAs.  Every
// group's parameters name the launch's mode.
template <typename T, bool COLMODE>
__global__ void __launch_bounds__(kGridThreads) k_cpqr_grid_grouped(const CpqrParams<T>* __restrict__ groups,
                                                                   int gsize, int32_t* J_base, int32_t* k_out_base,
                                                                   int32_t* info_base) {
    extern __shared__ __align__(16) uint8_t smem_dyn[];
    __shared__ GridShared<T> G_;
    __shared__ CpqrParams<T> sP;
    if (threadIdx.x == 0) {
        sP = groups[blockIdx.x / gsize];
        sP.J = J_base + sP.out_j;
        sP.k_out = k_out_base + sP.out_i;
        sP.info = info_base + sP.out_i;
    }
    __syncthreads();
    cpqr_grid_body<T, COLMODE>(sP, gsize, static_cast<int>(blockIdx.x % gsize), G_, smem_dyn);
}

template <typename T>
cudaError_t launch_cpqr_grouped(const CpqrParams<T>* groups, int ngroups, int gsize, int colmode, size_t smem,
                                int32_t* J_base, int32_t* k_out_base, int32_t* info_base, cudaStream_t s) {
    void* kern = colmode ? reinterpret_cast<void*>(k_cpqr_grid_grouped<T, true>)
                         : reinterpret_cast<void*>(k_cpqr_grid_grouped<T, false>);
    if (smem > 48 * 1024) {
        const cudaError_t e =
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    void* args[] = {const_cast<CpqrParams<T>**>(&groups), &gsize, &J_base, &k_out_base, &info_base};
    return cudaLaunchCooperativeKernel(kern, dim3(static_cast<unsigned>(ngroups * gsize)), dim3(kGridThreads), args,
                                       smem, s);
}
template cudaError_t launch_cpqr_grouped<float>(const CpqrParams<float>*, int, int, int, size_t, int32_t*, int32_t*,
                                                int32_t*, cudaStream_t);
template cudaError_t launch_cpqr_grouped<double>(const CpqrParams<double>*, int, int, int, size_t, int32_t*, int32_t*,
                                                 int32_t*, cudaStream_t);

size_t cpqr_grouped_smem(int64_t cpb, int64_t rstage, int f64) {
    return f64 ? grid_smem_bytes<double>(cpb, rstage) : grid_smem_bytes<float>(cpb, rstage);
}

int cpqr_grouped_colmode(int64_t cpb) { return grid_colmode(cpb) ? 1 : 0; }
int64_t cpqr_grouped_rstage(int64_t cpb, int64_t r, int elem_bytes) { return grid_rstage(cpb, r, elem_bytes); }

// Control region: the barrier word, the two candidate tables, then (at a 256-byte offset)
// the resident kernel's published columns [2][grid][r] or the streaming kernel's two
// pivot-column slots [2][r].
size_t cpqr_ctrl_bytes(const CpqrPlan& plan, int64_t r, int elem_bytes) {
    size_t b = cpqr_pub_offset(plan.grid);
    b += (plan.resident ? 2 * static_cast<size_t>(plan.grid) : size_t(2)) * r * elem_bytes;
    return b;
}

size_t cpqr_pub_offset(int grid) {
    return (sizeof(CpqrCtrl) + 2 * static_cast<size_t>(grid) * sizeof(Cand) + 255) & ~size_t(255);
}

bool cpqr_plan(int64_t r, int64_t n, int elem_bytes, CpqrPlan* plan) {
    const DeviceInfo& dev = device_info();
    plan->threads = kGridThreads;
    plan->grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(dev.sm_count, n)));
    const int64_t cpb = (n + plan->grid - 1) / plan->grid;
    // shared memory beyond the static part (about 2 KB) and a margin
    const size_t budget = std::min<size_t>(kResidentSmem, static_cast<size_t>(dev.max_smem_optin) - 8 * 1024);
    const bool f64 = elem_bytes == 8;
    const int64_t rst = grid_rstage(cpb, r, elem_bytes);
    const size_t lean = f64 ? grid_smem_bytes<double>(cpb, rst) : grid_smem_bytes<float>(cpb, rst);
    const size_t full = f64 ? resident_smem_bytes<double>(cpb, r) : resident_smem_bytes<float>(cpb, r);
    // resident (warp per column, cpqr_resident.cu) when the slice's columns fit the shared
    // memory, streamed through the working copy otherwise
    plan->resident = full <= budget ? 1 : 0;
    if (!plan->resident && lean > budget) return false;
    plan->smem = plan->resident ? full : lean;
    return true;
}

template <typename T>
static cudaError_t launch_cpqr_t(void* W, int64_t r, int64_t n, int64_t ldw, const void* src, int src_f64,
                                 int64_t ldsrc, int kcap, double rel_tol, int32_t* J, int32_t* k_out,
                                 int32_t* info, double* R64, int64_t ldr, uint8_t* sel, void* ctrl,
                                 const CpqrPlan& plan, uint64_t limit_ns, cudaStream_t s) {
    CpqrParams<T> P{};
    P.X = static_cast<T*>(W);
    P.r = r; P.n = n; P.ldx = ldw;
    P.src = src; P.src_f64 = src_f64; P.ldsrc = ldsrc;
    P.kcap = kcap; P.rel_tol = rel_tol;
    P.J = J; P.k_out = k_out; P.info = info;
    P.R = R64; P.ldr = ldr;
    P.sel = sel;
    P.ctrl = static_cast<CpqrCtrl*>(ctrl);
    P.cand = reinterpret_cast<Cand*>(static_cast<char*>(ctrl) + sizeof(CpqrCtrl));
    P.resident = plan.resident;
    P.pub = reinterpret_cast<T*>(static_cast<char*>(ctrl) + cpqr_pub_offset(plan.grid));
    P.cpb_max = (n + plan.grid - 1) / plan.grid;
    P.colmode = grid_colmode(P.cpb_max) ? 1 : 0;
    P.rstage = grid_rstage(P.cpb_max, r, static_cast<int>(sizeof(T)));
    P.limit_ns = limit_ns;
    cudaError_t e = cudaMemsetAsync(ctrl, 0, sizeof(CpqrCtrl), s);
    if (e != cudaSuccess) return e;
    if (P.resident) return launch_cpqr_resident<T>(P, plan.grid, plan.smem, s);
    void* kern = P.colmode ? reinterpret_cast<void*>(k_cpqr_grid<T, true>) : reinterpret_cast<void*>(k_cpqr_grid<T, false>);
    if (plan.smem > 48 * 1024) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(plan.smem));
        if (e != cudaSuccess) return e;
    }
    void* args[] = {&P};
    return cudaLaunchCooperativeKernel(kern, dim3(plan.grid), dim3(plan.threads), args, plan.smem, s);
}

cudaError_t launch_cpqr(void* W, int w_f64, int64_t r, int64_t n, int64_t ldw, const void* src, int src_f64,
                        int64_t ldsrc, int kcap, double rel_tol, int32_t* J, int32_t* k_out, int32_t* info,
                        double* R64, int64_t ldr, void* nu, void* nuref, uint8_t* sel, void* ctrl,
                        const CpqrPlan& plan, uint64_t limit_ns, cudaStream_t s) {
    (void)nu;
    (void)nuref;
    if (w_f64)
        return launch_cpqr_t<double>(W, r, n, ldw, src, src_f64, ldsrc, kcap, rel_tol, J, k_out, info, R64, ldr,
                                     sel, ctrl, plan, limit_ns, s);
    return launch_cpqr_t<float>(W, r, n, ldw, src, src_f64, ldsrc, kcap, rel_tol, J, k_out, info, R64, ldr, sel,
                                ctrl, plan, limit_ns, s);
}

}  // namespace gid
