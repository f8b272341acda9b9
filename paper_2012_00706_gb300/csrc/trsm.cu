// Coefficient matrix and error estimate of the column ID on GB300.
//
// T = R11^-1 R12 (Algorithm 1, the coefficient solve; R11 upper triangular and nonsingular, so
// the pseudo-inverse of the paper's Remark is its inverse), delivered in FP64,
// followed by `refine_steps` steps of iterative refinement
// T += R11^-1 (R12 - R11 T) with the residual formed in FP64.  The plain path
// solves in FP64; the mixed path, whose R comes from the FP32 pivoted QR, solves
// in FP32 and refines with the FP64 residual (mixed-precision iterative
// refinement).  The pivoted QR leaves R in FP64 storage (exact for FP32 R).
//
// k <= 256: one warp per column of T, the column in registers (lane l holds
// rows l, l+32, ...), R11 in shared memory where it fits; otherwise one thread per column.
//
// An FP32 solve refined once cuts the error by about kappa(R11) u32 per step, so
// the mixed path estimates kappa(R11) from the ratio of R11's largest and smallest
// diagonal magnitudes (a lower bound of the condition number) and, when
// kappa u32 exceeds 1e-2, solves and refines in FP64 instead (one ID), or takes
// more refinement steps (batched IDs).
#include "common.cuh"
#include "internal.h"

#include <algorithm>
#include <type_traits>

namespace gid {

constexpr int kSolveThreads = 64;

template <bool kSmem>
__global__ void __launch_bounds__(kSolveThreads)
k_solve_T(const double* __restrict__ R, int64_t ldr, const int32_t* __restrict__ J,
          const int32_t* __restrict__ k_ptr, int kcap, int64_t n, double* __restrict__ T, int64_t ldt,
          double* __restrict__ scratch, int refine_steps) {
    extern __shared__ double r11s[];
    const int k = *k_ptr;
    if (k <= 0) return;
    // R11(a, b) = R(a, J[b]) for a <= b
    if (kSmem) {
        for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) {
            const int a = idx % k, bb = idx / k;
            r11s[bb * k + a] = (a <= bb) ? R[static_cast<int64_t>(J[bb]) * ldr + a] : 0.0;
        }
        __syncthreads();
    }
    auto r11 = [&](int a, int bb) -> double {
        return kSmem ? r11s[bb * k + a] : __ldg(R + static_cast<int64_t>(J[bb]) * ldr + a);
    };
    for (int64_t c = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; c < n - k;
         c += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const double* r12 = R + static_cast<int64_t>(J[k + c]) * ldr;
        double* t = T + c * ldt;
        for (int a = k - 1; a >= 0; --a) {
            double s = r12[a];
            for (int bb = a + 1; bb < k; ++bb) s = fma(-r11(a, bb), t[bb], s);
            t[a] = s / r11(a, a);
        }
        double* d = scratch + c * kcap;
        for (int it = 0; it < refine_steps; ++it) {
            for (int a = 0; a < k; ++a) {
                double s = r12[a];
                for (int bb = a; bb < k; ++bb) s = fma(-r11(a, bb), t[bb], s);
                d[a] = s;
            }
            for (int a = k - 1; a >= 0; --a) {
                double s = d[a];
                for (int bb = a + 1; bb < k; ++bb) s = fma(-r11(a, bb), d[bb], s);
                d[a] = s / r11(a, a);
            }
            for (int a = 0; a < k; ++a) t[a] += d[a];
        }
    }
}

// The thread-per-column solve's correction vectors (kcap per column), or the product
// solve's FP32 R11 inverse, packed R11 and flag (2 kq^2 + 1 floats, kq = kcap rounded up to 4).
size_t solve_T_scratch_doubles(int kcap, int64_t n) {
    const size_t kq = static_cast<size_t>((kcap + 3) & ~3);
    return std::max(static_cast<size_t>(kcap) * static_cast<size_t>(n), kq * kq + 1);
}

// ---- warp-per-column solve for k <= 32*KQ: lane l holds rows l, l+32, ... of its column.
//
// Back-substitution is done column-oriented: for a = k-1 .. 0 the owner lane of
// row a forms t_a = t_a / R(a,a) (times the stored reciprocal) and broadcasts it,
// then every lane updates its rows b < a by t_b -= R(b,a) t_a (independent FMAs).
// TS is the precision of the two solves: double for the plain path; float for
// the mixed path, whose R is FP32, with the refinement residual
// R12 - R11 T formed in FP64 (mixed-precision iterative refinement).
constexpr int kWarpSolveWarps = 8;
// Largest rank of the warp-per-column solve: 32 rows per register block, 8 blocks.
constexpr int kWarpSolveMaxQ = 8;

// The steps a run by 32-row block qa (a compile-time register index), bottom block
// first: rows of the blocks above are all updated, rows of block qa only above a, and
// the blocks below, already final, are not touched.
// Where the solves read column a of R11 (rows 0..a): a k x k column-major copy in shared
// memory, or (the FP64 fallback of the mixed path) R itself in global memory through J.
template <typename TS>
struct SmemCols {
    const TS* base;
    int k;
    __device__ const TS* col(int a) const { return base + static_cast<int64_t>(a) * k; }
};
struct GlobalCols {
    const double* R;
    int64_t ldr;
    const int32_t* J;
    __device__ const double* col(int a) const { return R + static_cast<int64_t>(__ldg(J + a)) * ldr; }
};

template <typename TS, int KQ, typename Cols>
__device__ __forceinline__ void warp_backsub(TS (&t)[KQ], const Cols& cols, const TS* __restrict__ rinv,
                                             int k, int lane) {
#pragma unroll
    for (int qa = KQ - 1; qa >= 0; --qa) {
        for (int a = min(32 * qa + 31, k - 1); a >= 32 * qa; --a) {
            const int i = a - 32 * qa;
            const TS ta = __shfl_sync(0xffffffffu, t[qa] * rinv[a], i);
            const TS* col = cols.col(a) + lane;
#pragma unroll
            for (int q = 0; q < qa; ++q) t[q] = fma(-col[32 * q], ta, t[q]);
            if (lane < i) t[qa] = fma(-col[32 * qa], ta, t[qa]);
            else if (lane == i) t[qa] = ta;
        }
    }
}

// Refinement residual R12 - R11 T of the mixed path on the FP32 pipe.  R11, R12 and
// the first solve are FP32 values, so every product R(b,a) t_a splits exactly into
// two floats (p = fl(R t), e = fma(R, t, -p)); the sums are kept as unevaluated float
// pairs (TwoSum), which carries about 48 significant bits, well beyond the FP32
// round-off the refinement corrects.  t is passed as a float pair (hi, lo); lo is zero
// in the first refinement step.  Lane b accumulates rows b, b + 32, ... over a >= b.
template <int KQ>
__device__ __forceinline__ void residual_pairs(const double (&rhs)[KQ], const float (&th)[KQ], const float (&tl)[KQ],
                                               bool use_lo, const float* __restrict__ r11s, int k, int lane,
                                               double (&res)[KQ]) {
    float sh[KQ], sl[KQ];
#pragma unroll
    for (int q = 0; q < KQ; ++q) {
        sh[q] = static_cast<float>(rhs[q]);
        sl[q] = 0.f;
    }
    // a runs by 32-row block qa (compile-time register index): rows of the blocks above
    // take every step, rows of block qa those with b <= a
    auto update = [&](float& h, float& l, float rv, float ah, float al) {
        // explicit round-to-nearest operations: no contraction into FMAs
        const float p = __fmul_rn(rv, ah);
        const float e = fmaf(rv, ah, -p);
        const float s = __fadd_rn(h, p);                     // TwoSum(h, p)
        const float bp = __fsub_rn(s, h);
        const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(p, bp));
        h = s;
        l = __fadd_rn(l, __fadd_rn(err, e));
        if (use_lo) l = fmaf(rv, al, l);                     // R t_lo is below the pair's resolution
    };
#pragma unroll
    for (int qa = 0; qa < KQ; ++qa) {
        const int a_end = min(32 * qa + 32, k);
        for (int a = 32 * qa; a < a_end; ++a) {
            const int i = a - 32 * qa;
            const float ah = __shfl_sync(0xffffffffu, th[qa], i);
            const float al = use_lo ? __shfl_sync(0xffffffffu, tl[qa], i) : 0.f;
            const float* col = r11s + static_cast<int64_t>(a) * k + lane;
#pragma unroll
            for (int q = 0; q < qa; ++q) update(sh[q], sl[q], -col[32 * q], ah, al);
            if (lane <= i) update(sh[qa], sl[qa], -col[32 * qa], ah, al);
        }
    }
#pragma unroll
    for (int q = 0; q < KQ; ++q) res[q] = static_cast<double>(sh[q]) + static_cast<double>(sl[q]);
}

// Stage R11 = R(0:k, J[0:k]) (k x k, column-major, upper triangle: the solves never read
// below the diagonal) and the reciprocals of its diagonal.  Warp w takes columns
// a = w, w + nw, ...: its lanes first load those columns' pivot indices together, then
// each column's rows go to consecutive lanes, so the R loads are coalesced and none
// waits on another.
template <typename TS>
__device__ __forceinline__ void stage_r11(const double* __restrict__ R, int64_t ldr, const int32_t* __restrict__ J,
                                          int k, TS* r11s, TS* rinv) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int a0 = warp; a0 < k; a0 += 32 * nw) {
        const int ncol = min(32, (k - a0 + nw - 1) / nw);
        const int jl = lane < ncol ? __ldg(J + a0 + nw * lane) : 0;
#pragma unroll 4
        for (int c = 0; c < ncol; ++c) {
            const int a = a0 + nw * c;
            const double* col = R + static_cast<int64_t>(__shfl_sync(0xffffffffu, jl, c)) * ldr;
            TS* dst = r11s + static_cast<int64_t>(a) * k;
            for (int b = lane; b <= a; b += 32) dst[b] = static_cast<TS>(col[b]);
            if (lane == 0) rinv[a] = static_cast<TS>(1.0) / static_cast<TS>(col[a]);
        }
    }
}

// kappa u32 > 1e-2, i.e. max |R_jj| > kIllRatio min |R_jj| over the diagonal of R11.
constexpr double kIllRatio = 1e-2 * 16777216.0;
// Refinement steps of the batched FP32 solve when R11 is that ill-conditioned.
constexpr int kIllRefineSteps = 6;

// max |R(a, J[a])| > kIllRatio min |R(a, J[a])| over a < k, the same answer in every
// thread of the block (and in every block: all read the same R).
__device__ __forceinline__ bool r11_ill_conditioned(const double* __restrict__ R, int64_t ldr,
                                                    const int32_t* __restrict__ J, int k) {
    __shared__ double s_mx[32], s_mn[32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    double mx = 0.0, mn = INFINITY;
    for (int a = threadIdx.x; a < k; a += blockDim.x) {
        const double d = fabs(__ldg(R + static_cast<int64_t>(__ldg(J + a)) * ldr + a));
        mx = fmax(mx, d);
        mn = fmin(mn, d);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    }
    __syncthreads();
    if (lane == 0) { s_mx[warp] = mx; s_mn[warp] = mn; }
    __syncthreads();
    mx = 0.0;
    mn = INFINITY;
    for (int w = 0; w < nw; ++w) { mx = fmax(mx, s_mx[w]); mn = fmin(mn, s_mn[w]); }
    return mx > kIllRatio * mn;
}

// The columns of T this warp owns.  TS = float: R11 in shared memory (FP32 values), float-pair
// refinement residual; TS = double: R11 read through `cols`, FP64 residual.
template <typename TS, int KQ, typename Cols>
__device__ __forceinline__ void solve_columns(const double* __restrict__ R, int64_t ldr, const int32_t* __restrict__ J,
                                              int k, int64_t n, double* __restrict__ T, int64_t ldt, int refine_steps,
                                              const Cols& cols, const TS* rinv) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    for (int64_t c = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); c < n - k;
         c += nwarps) {
        const double* r12 = R + static_cast<int64_t>(J[k + c]) * ldr;
        double rhs[KQ];
        TS t[KQ];
#pragma unroll
        for (int q = 0; q < KQ; ++q) {
            const int b = lane + 32 * q;
            rhs[q] = b < k ? r12[b] : 0.0;
            t[q] = static_cast<TS>(rhs[q]);
        }
        warp_backsub<TS, KQ>(t, cols, rinv, k, lane);
        double tt[KQ];
#pragma unroll
        for (int q = 0; q < KQ; ++q) tt[q] = static_cast<double>(t[q]);
        for (int it = 0; it < refine_steps; ++it) {
            double res[KQ];
            if constexpr (std::is_same<TS, float>::value) {
                // R is FP32 (mixed path): exact products, float-pair sums
                float th[KQ], tl[KQ];
#pragma unroll
                for (int q = 0; q < KQ; ++q) {
                    th[q] = static_cast<float>(tt[q]);
                    tl[q] = static_cast<float>(tt[q] - static_cast<double>(th[q]));
                }
                residual_pairs<KQ>(rhs, th, tl, it > 0, cols.base, k, lane, res);
            } else {
                // residual R12 - R11 T in FP64 (row-oriented: lane b sums over a >= b)
#pragma unroll
                for (int q = 0; q < KQ; ++q) res[q] = rhs[q];
#pragma unroll
                for (int qa = 0; qa < KQ; ++qa) {
                    const int a_end = min(32 * qa + 32, k);
                    for (int a = 32 * qa; a < a_end; ++a) {
                        const int i = a - 32 * qa;
                        const double ta = __shfl_sync(0xffffffffu, tt[qa], i);
                        const double* col = cols.col(a) + lane;
#pragma unroll
                        for (int q = 0; q < qa; ++q) res[q] = fma(-col[32 * q], ta, res[q]);
                        if (lane <= i) res[qa] = fma(-col[32 * qa], ta, res[qa]);
                    }
                }
            }
            TS d[KQ];
#pragma unroll
            for (int q = 0; q < KQ; ++q) d[q] = static_cast<TS>(res[q]);
            warp_backsub<TS, KQ>(d, cols, rinv, k, lane);
#pragma unroll
            for (int q = 0; q < KQ; ++q) tt[q] += static_cast<double>(d[q]);
        }
        double* out = T + c * ldt;
#pragma unroll
        for (int q = 0; q < KQ; ++q) {
            const int b = lane + 32 * q;
            if (b < k) out[b] = tt[q];
        }
    }
}

// The FP64 solves of k_solve_T_warp's fallbacks, kept out of line so that their registers
// do not weigh on the common path's allocation.
template <int KQ>
__device__ __noinline__ void solve_fp64_fallback(const double* __restrict__ R, int64_t ldr,
                                                 const int32_t* __restrict__ J, int k, int64_t n,
                                                 double* __restrict__ T, int64_t ldt, int refine_steps,
                                                 int64_t smem_bytes, uint8_t* sm) {
    if ((static_cast<int64_t>(k) * k + k) * 8 <= smem_bytes) {
        double* r11s = reinterpret_cast<double*>(sm);
        double* rinv = r11s + static_cast<int64_t>(k) * k;
        stage_r11<double>(R, ldr, J, k, r11s, rinv);
        __syncthreads();
        solve_columns<double, KQ>(R, ldr, J, k, n, T, ldt, refine_steps, SmemCols<double>{r11s, k}, rinv);
    } else {
        double* rinv = reinterpret_cast<double*>(sm);
        for (int a = threadIdx.x; a < k; a += blockDim.x) rinv[a] = 1.0 / R[static_cast<int64_t>(J[a]) * ldr + a];
        __syncthreads();
        solve_columns<double, KQ>(R, ldr, J, k, n, T, ldt, refine_steps, GlobalCols{R, ldr, J}, rinv);
    }
}

// TS = double: the plain path, R11 staged in FP64.  TS = float: the mixed path, whose R is
// FP32 (R11 staged in FP32, float-pair refinement residual), unless R11 is ill-conditioned
// (r11_ill_conditioned): then the FP64 solve and residual, on the same FP64-stored R.  The
// FP64 solves stage R11 in shared memory when `smem_bytes` holds an FP64 copy; otherwise
// (a rank too large for the copy, or the mixed path's ill-conditioned fallback) they read
// R11 from R itself through J, with the FP64 reciprocals of its diagonal in shared memory.
template <typename TS, int KQ>
__global__ void __launch_bounds__(kWarpSolveWarps * 32)
k_solve_T_warp(const double* __restrict__ R, int64_t ldr, const int32_t* __restrict__ J,
               const int32_t* __restrict__ k_ptr, int64_t n, double* __restrict__ T, int64_t ldt,
               int refine_steps, int64_t smem_bytes) {
    extern __shared__ __align__(16) uint8_t sm[];
    const int k = *k_ptr;
    if (k <= 0) return;
    const bool ts_fits = (static_cast<int64_t>(k) * k + k) * static_cast<int64_t>(sizeof(TS)) <= smem_bytes;
    bool fp64 = !ts_fits;
    if constexpr (std::is_same<TS, float>::value) fp64 = fp64 || r11_ill_conditioned(R, ldr, J, k);
    if (fp64) {
        solve_fp64_fallback<KQ>(R, ldr, J, k, n, T, ldt, refine_steps, smem_bytes, sm);
        return;
    }
    TS* r11s = reinterpret_cast<TS*>(sm);
    TS* rinv = r11s + static_cast<int64_t>(k) * k;
    stage_r11<TS>(R, ldr, J, k, r11s, rinv);
    __syncthreads();
    solve_columns<TS, KQ>(R, ldr, J, k, n, T, ldt, refine_steps, SmemCols<TS>{r11s, k}, rinv);
}

template <typename TS, int KQ>
static cudaError_t launch_warp_solve(const double* R64, int64_t ldr, const int32_t* J, const int32_t* k_ptr, int kcap,
                                     int64_t n, double* T, int64_t ldt, int refine_steps, cudaStream_t s) {
    // R11 and its diagonal reciprocals in the solve precision when they fit (the FP64
    // fallbacks need only k doubles of it)
    const size_t budget = static_cast<size_t>(device_info().max_smem_optin) - 4096;
    const size_t need = (static_cast<size_t>(kcap) * kcap + kcap) * sizeof(TS);
    const size_t smem = std::max(need <= budget ? need : size_t(0), kcap * sizeof(double)) + 16;
    auto kern = k_solve_T_warp<TS, KQ>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    // one warp per column where possible: the solves are chains of k dependent steps, so
    // more resident warps (several CTAs per SM; R11 is small) hide their latency
    const int64_t cols = std::max<int64_t>(1, n - 1);
    const int64_t want = (cols + kWarpSolveWarps - 1) / kWarpSolveWarps;
    const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(want, 8LL * device_info().sm_count)));
    kern<<<grid, kWarpSolveWarps * 32, smem, s>>>(R64, ldr, J, k_ptr, n, T, ldt, refine_steps,
                                                  static_cast<int64_t>(smem - 16));
    return cudaGetLastError();
}

template <typename TS>
static cudaError_t launch_warp_solve_kq(int kq, const double* R64, int64_t ldr, const int32_t* J, const int32_t* k_ptr,
                                        int kcap, int64_t n, double* T, int64_t ldt, int refine_steps,
                                        cudaStream_t s) {
    switch (kq) {
        case 1: return launch_warp_solve<TS, 1>(R64, ldr, J, k_ptr, kcap, n, T, ldt, refine_steps, s);
        case 2: return launch_warp_solve<TS, 2>(R64, ldr, J, k_ptr, kcap, n, T, ldt, refine_steps, s);
        case 3: return launch_warp_solve<TS, 3>(R64, ldr, J, k_ptr, kcap, n, T, ldt, refine_steps, s);
        case 4: return launch_warp_solve<TS, 4>(R64, ldr, J, k_ptr, kcap, n, T, ldt, refine_steps, s);
        case 5: return launch_warp_solve<TS, 5>(R64, ldr, J, k_ptr, kcap, n, T, ldt, refine_steps, s);
        case 6: return launch_warp_solve<TS, 6>(R64, ldr, J, k_ptr, kcap, n, T, ldt, refine_steps, s);
        case 7: return launch_warp_solve<TS, 7>(R64, ldr, J, k_ptr, kcap, n, T, ldt, refine_steps, s);
        default: return launch_warp_solve<TS, 8>(R64, ldr, J, k_ptr, kcap, n, T, ldt, refine_steps, s);
    }
}

// The warp-per-column solve of columns [c0, c_end) of T of one matrix of the batch (T with
// leading dimension ldr): R11 staged in FP32, FP32 solves, `steps` refinement steps with the
// float-pair residual.
template <int KQ>
__device__ __forceinline__ void batched_warp_columns(const double* __restrict__ R, int ldr,
                                                     const int32_t* __restrict__ J, int k, int64_t c0, int64_t c_end,
                                                     double* __restrict__ T, int steps, uint8_t* sm) {
    float* r11s = reinterpret_cast<float*>(sm);                         // k x k, column-major
    float* rinv = r11s + static_cast<int64_t>(k) * k;
    stage_r11<float>(R, ldr, J, k, r11s, rinv);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int64_t c = c0 + (threadIdx.x >> 5); c < c_end; c += blockDim.x >> 5) {
        const double* r12 = R + static_cast<int64_t>(J[k + c]) * ldr;
        double rhs[KQ];
        float t[KQ];
#pragma unroll
        for (int q = 0; q < KQ; ++q) {
            const int b = lane + 32 * q;
            rhs[q] = b < k ? r12[b] : 0.0;
            t[q] = static_cast<float>(rhs[q]);
        }
        warp_backsub<float, KQ>(t, SmemCols<float>{r11s, k}, rinv, k, lane);
        double tt[KQ];
#pragma unroll
        for (int q = 0; q < KQ; ++q) tt[q] = static_cast<double>(t[q]);
        for (int it = 0; it < steps; ++it) {
            double res[KQ];
            float th[KQ], tl[KQ];
#pragma unroll
            for (int q = 0; q < KQ; ++q) {
                th[q] = static_cast<float>(tt[q]);
                tl[q] = static_cast<float>(tt[q] - static_cast<double>(th[q]));
            }
            residual_pairs<KQ>(rhs, th, tl, it > 0, r11s, k, lane, res);
            float d[KQ];
#pragma unroll
            for (int q = 0; q < KQ; ++q) d[q] = static_cast<float>(res[q]);
            warp_backsub<float, KQ>(d, SmemCols<float>{r11s, k}, rinv, k, lane);
#pragma unroll
            for (int q = 0; q < KQ; ++q) tt[q] += static_cast<double>(d[q]);
        }
        double* out = T + c * ldr;
#pragma unroll
        for (int q = 0; q < KQ; ++q) {
            const int b = lane + 32 * q;
            if (b < k) out[b] = tt[q];
        }
    }
}

// ---- batched solve: CTA b solves columns [c0, c0 + ncols) of T of task units[b].task,
// with the warp-per-column scheme above (FP32 solves, FP64 refinement residual).
constexpr int kBatchSolveMaxWarps = 16;

template <int KQ>
__global__ void __launch_bounds__(kBatchSolveMaxWarps * 32)
k_solve_T_batched(const BatchTask* __restrict__ tasks, const SolveUnit* __restrict__ units,
                  const double* __restrict__ R_base, const int32_t* __restrict__ J_base,
                  const int32_t* __restrict__ k_out, int32_t* infos, double* __restrict__ T_base,
                  BatchTotals tot, int kmax, int refine_steps) {
    extern __shared__ __align__(16) uint8_t sm[];
    __shared__ int s_bad;
    const SolveUnit su = units[blockIdx.x];
    if (su.task < 0 || su.task >= tot.ntasks) return;
    const BatchTask& bt = tasks[su.task];
    const int k = k_out[su.task];
    const int64_t c_end = min(min(static_cast<int64_t>(su.c0) + su.ncols, bt.n - k), bt.tcols);
    if (k <= 0 || su.c0 < 0 || su.c0 >= c_end) return;
    const double* R = R_base + bt.r_off;
    const int32_t* J = J_base + bt.j_off;
    const int ldr = bt.kcap;
    // every index below stays inside this task's regions: check the entry and the
    // pivot list before using them
    if (threadIdx.x == 0)
        s_bad = !(k <= bt.kcap && k <= kmax && bt.r_off >= 0 && bt.r_off + static_cast<int64_t>(bt.kcap) * bt.n <= tot.r &&
                  bt.j_off >= 0 && bt.j_off + bt.n <= tot.j && bt.t_off >= 0 &&
                  bt.t_off + static_cast<int64_t>(bt.kcap) * bt.tcols <= tot.t);
    __syncthreads();
    if (s_bad) {
        if (threadIdx.x == 0) set_info(infos + su.task, kInfoBadTable);
        return;
    }
    for (int64_t a = threadIdx.x; a < bt.n; a += blockDim.x)
        if (J[a] < 0 || J[a] >= bt.n) s_bad = 1;
    __syncthreads();
    if (s_bad) {
        if (threadIdx.x == 0) set_info(infos + su.task, kInfoBadTable);
        return;
    }
    // an ill-conditioned R11 takes more refinement steps (each cuts the error by kappa u32)
    const int steps = (refine_steps > 0 && r11_ill_conditioned(R, ldr, J, k))
                          ? max(refine_steps, kIllRefineSteps) : refine_steps;
    batched_warp_columns<KQ>(R, ldr, J, k, su.c0, c_end, T_base + bt.t_off, steps, sm);
}

template <int KQ>
static cudaError_t launch_batched_solve(const BatchTask* tasks, const SolveUnit* units, int nunits, int kmax,
                                        int warps, const double* R_base, const int32_t* J_base,
                                        const int32_t* k_out, int32_t* infos, double* T_base,
                                        const BatchTotals& tot, int refine_steps, cudaStream_t s) {
    const size_t smem = static_cast<size_t>(kmax) * kmax * sizeof(float) + kmax * sizeof(float) + 16;
    auto kern = k_solve_T_batched<KQ>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    kern<<<nunits, warps * 32, smem, s>>>(tasks, units, R_base, J_base, k_out, infos, T_base, tot, kmax,
                                          refine_steps);
    return cudaGetLastError();
}

cudaError_t launch_solve_T_batched(const BatchTask* tasks, const SolveUnit* units, int nunits, int kmax, int warps,
                                   const double* R_base, const int32_t* J_base, const int32_t* k_out,
                                   int32_t* infos, double* T_base, const BatchTotals& tot, int refine_steps,
                                   cudaStream_t s) {
    if (nunits <= 0) return cudaSuccess;
    if (kmax < 1 || kmax > 128 || warps < 1 || warps > kBatchSolveMaxWarps) return cudaErrorInvalidValue;
    switch ((kmax + 31) / 32) {
        case 1: return launch_batched_solve<1>(tasks, units, nunits, kmax, warps, R_base, J_base, k_out, infos,
                                               T_base, tot, refine_steps, s);
        case 2: return launch_batched_solve<2>(tasks, units, nunits, kmax, warps, R_base, J_base, k_out, infos,
                                               T_base, tot, refine_steps, s);
        case 3: return launch_batched_solve<3>(tasks, units, nunits, kmax, warps, R_base, J_base, k_out, infos,
                                               T_base, tot, refine_steps, s);
        default: return launch_batched_solve<4>(tasks, units, nunits, kmax, warps, R_base, J_base, k_out, infos,
                                                T_base, tot, refine_steps, s);
    }
}

// ---- FP32 coefficient solve as products (R from an FP32 pivoted QR, k <= 128, one
// refinement step).  k_r11_inverse stages R11 once per CTA (every load in flight), forms
// X = R11^-1 by warp substitutions (X(:,j) solves the leading (j+1) x (j+1) system for
// e_j), and leaves in the scratch X, a packed FP32 copy of R11 and the ill-conditioning
// flag.  k_solve_T_gemm then takes kGemmCols columns of T per CTA: T0 = X R12, the residual
// E = R12 - R11 T0 with exact products summed as float pairs (as residual_pairs), and
// T = T0 + X E, delivered in FP64.  The refinement is the same one step as the warp
// solve's; the substitutions, a dependent chain per column of T there, run once per column
// of R11 here, and the rest are register-tiled products (a 4 x 2 block per thread) that skip
// the zero triangles of X and R11.  An ill-conditioned R11 (r11_ill_conditioned) takes the
// FP64 solves of the warp kernel instead.
//
// Scratch (floats, kq = kcap rounded up to 4): X [kq x kq], R11 [kq x kq], flag; both
// matrices are column-major with the device rank's kp = k rounded up to 4 as leading
// dimension, zero below the diagonal and past k.
// Tile width of T (512 threads: 32 row groups x 16 column pairs).  In the in-flight stream
// 32-column tiles beat 16-column ones (half the CTAs, each hiding its latency with twice
// the warps) at 4 us more solve latency.
constexpr int kGemmCols = 32;
constexpr int kGemmMaxK = 128;

__host__ __device__ inline int gemm_kp(int k) { return (k + 3) & ~3; }

// An FP32 value stored in an FP64 word, converted by its bits when it is a normal float
// (the values R holds on this path), by the FP64 pipe otherwise.
__device__ __forceinline__ float f32_of_exact(double x) {
    const uint32_t hi = static_cast<uint32_t>(__double2hiint(x));
    const uint32_t lo = static_cast<uint32_t>(__double2loint(x));
    const uint32_t e = (hi >> 20) & 0x7FFu;
    if (e >= 897u && e <= 1150u && (lo & 0x1FFFFFFFu) == 0u)
        return __uint_as_float((hi & 0x80000000u) | ((e - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
    return __double2float_rn(x);
}

// The inverse of R11 for columns j = jb * 8 + warp of X (this CTA's block jb): stage R11 once
// (every load in flight), test its conditioning (block 0), and leave X(:, j) and the packed
// R11(:, j) in the scratch (layout above).  R11(a, b) = R(a, J[b]).  Returns false (nothing
// written) when a pivot index is out of range [0, n).
template <int KQ>
__device__ __forceinline__ bool r11_inverse_body(const double* __restrict__ R, int64_t ldr,
                                                 const int32_t* __restrict__ J, int64_t n, int k, int jb,
                                                 float* __restrict__ scr, int kq_cap, uint8_t* sm) {
    __shared__ int js[32 * KQ];
    __shared__ int s_bad;
    const int kp = gemm_kp(k);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* r11s = reinterpret_cast<float*>(sm);                 // k x k, column-major
    float* rinv = r11s + static_cast<int64_t>(k) * k;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const int v = __ldg(J + i);
        js[i] = v;
        if (v < 0 || v >= n) s_bad = 1;
    }
    __syncthreads();
    if (s_bad) return false;
    // R11 by rounds of 4 columns per warp, the 4 KQ loads of a lane issued together
    for (int a0 = warp; a0 < k; a0 += 4 * kWarpSolveWarps) {
        double v[4][KQ];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int a = a0 + u * kWarpSolveWarps;
            const double* col = R + static_cast<int64_t>(js[min(a, k - 1)]) * ldr;
#pragma unroll
            for (int q = 0; q < KQ; ++q) {
                const int b = lane + 32 * q;
                v[u][q] = (a < k && b <= a) ? col[b] : 0.0;
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int a = a0 + u * kWarpSolveWarps;
            if (a >= k) continue;
#pragma unroll
            for (int q = 0; q < KQ; ++q) {
                const int b = lane + 32 * q;
                if (b <= a) r11s[a * k + b] = f32_of_exact(v[u][q]);
                if (b == a) rinv[a] = 1.f / f32_of_exact(v[u][q]);
            }
        }
    }
    float* X = scr;
    float* R11p = scr + static_cast<int64_t>(kq_cap) * kq_cap;
    __syncthreads();
    if (jb == 0) {
        // the test of r11_ill_conditioned on the staged diagonal (the same FP32 values)
        __shared__ float s_mx[kWarpSolveWarps], s_mn[kWarpSolveWarps];
        float mx = 0.f, mn = INFINITY;
        for (int a = threadIdx.x; a < k; a += blockDim.x) {
            const float d = fabsf(r11s[a * k + a]);
            mx = fmaxf(mx, d);
            mn = fminf(mn, d);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        }
        if (lane == 0) {
            s_mx[warp] = mx;
            s_mn[warp] = mn;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) {
                mx = fmaxf(mx, s_mx[w]);
                mn = fminf(mn, s_mn[w]);
            }
            const bool ill = static_cast<double>(mx) > kIllRatio * static_cast<double>(mn);
            reinterpret_cast<int*>(R11p + static_cast<int64_t>(kq_cap) * kq_cap)[0] = ill ? 1 : 0;
        }
    }
    const int j = jb * kWarpSolveWarps + warp;
    if (j >= kp) return true;
    // the packed copy of R11 for the product kernel: each warp writes the column it inverts
    for (int b = lane; b < kp; b += 32) R11p[j * kp + b] = (j < k && b <= j) ? r11s[j * k + b] : 0.f;
    float t[KQ];
#pragma unroll
    for (int q = 0; q < KQ; ++q) t[q] = (lane + 32 * q == j) ? 1.f : 0.f;
    // X(:, j) involves R11(0:j, 0:j) only: a chain of j + 1 steps
    if (j < k) warp_backsub<float, KQ>(t, SmemCols<float>{r11s, k}, rinv, j + 1, lane);
    float* xc = X + static_cast<int64_t>(j) * kp;
#pragma unroll
    for (int q = 0; q < KQ; ++q) {
        const int b = lane + 32 * q;
        if (b < kp) xc[b] = (j < k && b <= j) ? t[q] : 0.f;
    }
    return true;
}

template <int KQ>
__global__ void __launch_bounds__(kWarpSolveWarps * 32)
k_r11_inverse(const double* __restrict__ R, int64_t ldr, const int32_t* __restrict__ J,
              const int32_t* __restrict__ k_ptr, int64_t n, float* __restrict__ scr, int kq_cap) {
    extern __shared__ __align__(16) uint8_t sm[];
    const int k = *k_ptr;
    if (k <= 0 || static_cast<int>(blockIdx.x) * kWarpSolveWarps >= gemm_kp(k)) return;
    r11_inverse_body<KQ>(R, ldr, J, n, k, blockIdx.x, scr, kq_cap, sm);
}

// Shared memory of the product tiles for a scratch capacity kq and tiles of `cols` columns: X
// and R11 (kq x kq each), the R12 / residual tile and the T0 tile (kq rows of cols + 2 floats:
// the padding spreads the column-wise stores of the R12 staging over the banks), in floats.
__host__ __device__ inline int gemm_ld(int cols) { return cols + 2; }
__host__ __device__ inline size_t gemm_tile_floats(int kq, int cols) {
    return 2 * static_cast<size_t>(kq) * kq + 2 * static_cast<size_t>(kq) * gemm_ld(cols);
}

// Columns [c0, c0 + ncols) of T (ncols <= COLS) from the staged X and R11 (kp x kp in Xs,
// Rs): stage R12 (column c of the tile is R(:, jcol[c])), T0 = X R12, E = R12 - R11 T0 (exact
// products, float-pair sums), T = T0 + X E written as T[(c0 + c) ldt + row].  All 16 COLS
// threads of the CTA call it (32 row groups x COLS / 2 column pairs); it ends with a barrier.
template <int KQ, int COLS>
__device__ __forceinline__ void gemm_tile(const double* __restrict__ R, int64_t ldr, const int* jcol, int k, int kp,
                                          int ncols, const float* Xs, const float* Rs, float* Bt, float* Tt,
                                          double* __restrict__ T, int64_t c0, int64_t ldt) {
    constexpr int LD = COLS + 2, NCG = COLS / 2, NW = COLS / 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // R12 tile: warp w takes columns w and w + NW, its lanes the rows
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int c = warp + u * NW;
        const double* col = R + static_cast<int64_t>(jcol[c]) * ldr;
        double v[KQ];
#pragma unroll
        for (int q = 0; q < KQ; ++q) {
            const int b = lane + 32 * q;
            v[q] = (b < k && c < ncols) ? col[b] : 0.0;
        }
#pragma unroll
        for (int q = 0; q < KQ; ++q) {
            const int b = lane + 32 * q;
            if (b < kp) Bt[b * LD + c] = f32_of_exact(v[q]);
        }
    }
    __syncthreads();
    const int tx = threadIdx.x % NCG, ty = threadIdx.x / NCG;   // columns 2 tx, 2 tx + 1; rows 4 ty .. 4 ty + 3
    const int r0 = 4 * ty, cc = 2 * tx;
    const bool live = r0 < kp;
    float t0[4][2] = {};
    if (live) {
        // T0 = X R12: X(r, b) = 0 for b < r
#pragma unroll 4
        for (int b = r0; b < kp; ++b) {
            const float4 xv = *reinterpret_cast<const float4*>(Xs + b * kp + r0);
            const float2 bv = *reinterpret_cast<const float2*>(Bt + b * LD + cc);
            const float xa[4] = {xv.x, xv.y, xv.z, xv.w}, ba[2] = {bv.x, bv.y};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int jj = 0; jj < 2; ++jj) t0[i][jj] = fmaf(xa[i], ba[jj], t0[i][jj]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
            *reinterpret_cast<float2*>(Tt + (r0 + i) * LD + cc) = make_float2(t0[i][0], t0[i][1]);
    }
    __syncthreads();
    float e[4][2] = {};
    if (live) {
        // E = R12 - R11 T0: exact products (p, fma error), float-pair sums (TwoSum)
        float hi[4][2], lo[4][2];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 bv = *reinterpret_cast<const float2*>(Bt + (r0 + i) * LD + cc);
            hi[i][0] = bv.x;
            hi[i][1] = bv.y;
            lo[i][0] = lo[i][1] = 0.f;
        }
#pragma unroll 2
        for (int b = r0; b < kp; ++b) {
            const float4 rv = *reinterpret_cast<const float4*>(Rs + b * kp + r0);
            const float2 tv = *reinterpret_cast<const float2*>(Tt + b * LD + cc);
            const float ra[4] = {-rv.x, -rv.y, -rv.z, -rv.w}, ta[2] = {tv.x, tv.y};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int jj = 0; jj < 2; ++jj) {
                    const float pr = __fmul_rn(ra[i], ta[jj]);
                    const float er = fmaf(ra[i], ta[jj], -pr);
                    const float sum = __fadd_rn(hi[i][jj], pr);
                    const float bp = __fsub_rn(sum, hi[i][jj]);
                    const float err = __fadd_rn(__fsub_rn(hi[i][jj], __fsub_rn(sum, bp)), __fsub_rn(pr, bp));
                    hi[i][jj] = sum;
                    lo[i][jj] = __fadd_rn(lo[i][jj], __fadd_rn(err, er));
                }
        }
        // the pair's sum rounded once to FP32
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int jj = 0; jj < 2; ++jj) e[i][jj] = __fadd_rn(hi[i][jj], lo[i][jj]);
    }
    __syncthreads();    // every read of R12 is done before E takes its place
    if (live) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            *reinterpret_cast<float2*>(Bt + (r0 + i) * LD + cc) = make_float2(e[i][0], e[i][1]);
    }
    __syncthreads();
    if (live) {
        // T = T0 + X E
        float d[4][2] = {};
#pragma unroll 4
        for (int b = r0; b < kp; ++b) {
            const float4 xv = *reinterpret_cast<const float4*>(Xs + b * kp + r0);
            const float2 ev = *reinterpret_cast<const float2*>(Bt + b * LD + cc);
            const float xa[4] = {xv.x, xv.y, xv.z, xv.w}, ea[2] = {ev.x, ev.y};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int jj = 0; jj < 2; ++jj) d[i][jj] = fmaf(xa[i], ea[jj], d[i][jj]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int row = r0 + i;
            if (row >= k) continue;
#pragma unroll
            for (int jj = 0; jj < 2; ++jj) {
                const int c = cc + jj;
                if (c < ncols)
                    T[(c0 + c) * ldt + row] = static_cast<double>(t0[i][jj]) + static_cast<double>(d[i][jj]);
            }
        }
    }
    __syncthreads();    // the tiles are free for the next call
}

// X and R11 from the scratch into shared memory (kp x kp each, float4 copies).
__device__ __forceinline__ void stage_x_r11(const float* __restrict__ scr, int kq_cap, int kp, float* Xs, float* Rs) {
    const float4* xg4 = reinterpret_cast<const float4*>(scr);
    const float4* rg4 = reinterpret_cast<const float4*>(scr + static_cast<int64_t>(kq_cap) * kq_cap);
    float4* xs4 = reinterpret_cast<float4*>(Xs);
    float4* rs4 = reinterpret_cast<float4*>(Rs);
    const int n4 = kp * kp / 4;
#pragma unroll 8
    for (int i = threadIdx.x; i < n4; i += blockDim.x) {
        const float4 x = __ldg(xg4 + i), r = __ldg(rg4 + i);
        xs4[i] = x;
        rs4[i] = r;
    }
}

template <int KQ, int COLS>
__global__ void __launch_bounds__(16 * COLS)
k_solve_T_gemm(const double* __restrict__ R, int64_t ldr, const int32_t* __restrict__ J,
               const int32_t* __restrict__ k_ptr, int64_t n, const float* __restrict__ scr, int kq_cap,
               double* __restrict__ T, int64_t ldt, int refine_steps, int64_t smem_bytes) {
    extern __shared__ __align__(16) uint8_t sm[];
    __shared__ int jc[COLS];
    const int k = *k_ptr;
    if (k <= 0) return;
    if (__ldg(reinterpret_cast<const int*>(scr + 2 * static_cast<int64_t>(kq_cap) * kq_cap))) {
        // every CTA takes part: the fallback's warps cover all columns of T by a grid stride
        solve_fp64_fallback<KQ>(R, ldr, J, k, n, T, ldt, refine_steps, smem_bytes, sm);
        return;
    }
    const int64_t nc = n - k;
    const int64_t c0 = static_cast<int64_t>(blockIdx.x) * COLS;
    if (c0 >= nc) return;
    const int ncols = static_cast<int>(min(static_cast<int64_t>(COLS), nc - c0));
    const int kp = gemm_kp(k);
    float* Xs = reinterpret_cast<float*>(sm);        // kp x kp, column-major
    float* Rs = Xs + kp * kp;                        // R11, kp x kp column-major
    float* Bt = Rs + kp * kp;                        // [kp][gemm_ld]: R12, then the residual E
    float* Tt = Bt + kp * gemm_ld(COLS);             // [kp][gemm_ld]: T0
    if (threadIdx.x < COLS) jc[threadIdx.x] = threadIdx.x < ncols ? __ldg(J + k + c0 + threadIdx.x) : 0;
    stage_x_r11(scr, kq_cap, kp, Xs, Rs);
    __syncthreads();
    gemm_tile<KQ, COLS>(R, ldr, jc, k, kp, ncols, Xs, Rs, Bt, Tt, T, c0, ldt);
}

template <int KQ, int COLS>
static cudaError_t launch_gemm_tiles(const double* R64, int64_t ldr, const int32_t* J, const int32_t* k_ptr, int kcap,
                                     int64_t n, double* T, int64_t ldt, float* scr, cudaStream_t s) {
    const int kq = gemm_kp(kcap);
    // the tiles' shared memory, or the FP64 fallback's copy of R11 if that is larger
    const size_t tiles = gemm_tile_floats(kq, COLS) * sizeof(float);
    const size_t fb = (static_cast<size_t>(kcap) * kcap + kcap) * sizeof(double);
    const size_t smem = std::max(tiles, fb) + 16;
    auto kern = k_solve_T_gemm<KQ, COLS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int64_t cols = std::max<int64_t>(1, n - 1);
    const unsigned grid = static_cast<unsigned>((cols + COLS - 1) / COLS);
    kern<<<grid, 16 * COLS, smem, s>>>(R64, ldr, J, k_ptr, n, scr, kq, T, ldt, 1, static_cast<int64_t>(smem - 16));
    return cudaGetLastError();
}

template <int KQ>
static cudaError_t launch_gemm_solve(const double* R64, int64_t ldr, const int32_t* J, const int32_t* k_ptr, int kcap,
                                     int64_t n, double* T, int64_t ldt, float* scr, cudaStream_t s) {
    const int kq = gemm_kp(kcap);
    const size_t inv_smem = (static_cast<size_t>(kcap) * kcap + kcap) * sizeof(float) + 16;
    auto kinv = k_r11_inverse<KQ>;
    cudaError_t e = cudaFuncSetAttribute(kinv, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(inv_smem));
    if (e != cudaSuccess) return e;
    kinv<<<(kq + kWarpSolveWarps - 1) / kWarpSolveWarps, kWarpSolveWarps * 32, inv_smem, s>>>(R64, ldr, J, k_ptr, n,
                                                                                                scr, kq);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_gemm_tiles<KQ, kGemmCols>(R64, ldr, J, k_ptr, kcap, n, T, ldt, scr, s);
}

// ---- the batch's solve as products: k_r11_inverse_batched forms every matrix's X, packed
// R11 and flag in its slice of the inverse region (BatchTask::inv_off, the layout above with
// kq = kcap rounded up to 4), CTA (matrix, 8-column block of X); k_solve_T_batched_gemm then
// runs the unit's columns by tiles of kGemmCols, or the warp-per-column solve with extra
// refinement steps for an ill-conditioned R11.
__host__ __device__ inline int64_t batch_inv_floats(int kcap) {
    const int64_t kq = gemm_kp(kcap);
    return 2 * kq * kq + 4;
}

// A table entry whose regions all lie inside the workspace and the outputs.
__device__ __forceinline__ bool batch_entry_ok(const BatchTask& bt, int k, int kmax, const BatchTotals& tot) {
    return k <= bt.kcap && k <= kmax && bt.r_off >= 0 && bt.r_off + static_cast<int64_t>(bt.kcap) * bt.n <= tot.r &&
           bt.j_off >= 0 && bt.j_off + bt.n <= tot.j && bt.t_off >= 0 &&
           bt.t_off + static_cast<int64_t>(bt.kcap) * bt.tcols <= tot.t && bt.inv_off >= 0 &&
           bt.inv_off + batch_inv_floats(bt.kcap) <= tot.inv;
}

template <int KQ>
__global__ void __launch_bounds__(kWarpSolveWarps * 32)
k_r11_inverse_batched(const BatchTask* __restrict__ tasks, const double* __restrict__ R_base,
                      const int32_t* __restrict__ J_base, const int32_t* __restrict__ k_out, BatchTotals tot,
                      float* __restrict__ inv_base) {
    extern __shared__ __align__(16) uint8_t sm[];
    const int task = blockIdx.x;
    if (task >= tot.ntasks) return;
    const BatchTask& bt = tasks[task];
    const int k = k_out[task];
    if (k <= 0 || static_cast<int>(blockIdx.y) * kWarpSolveWarps >= gemm_kp(k)) return;
    if (!batch_entry_ok(bt, k, 32 * KQ, tot)) return;     // the product kernel reports it
    r11_inverse_body<KQ>(R_base + bt.r_off, bt.kcap, J_base + bt.j_off, bt.n, k, blockIdx.y,
                         inv_base + bt.inv_off, gemm_kp(bt.kcap), sm);
}

template <int KQ>
__global__ void __launch_bounds__(16 * kGemmCols)
k_solve_T_batched_gemm(const BatchTask* __restrict__ tasks, const SolveUnit* __restrict__ units,
                       const double* __restrict__ R_base, const int32_t* __restrict__ J_base,
                       const int32_t* __restrict__ k_out, int32_t* infos, double* __restrict__ T_base,
                       BatchTotals tot, int kmax, int refine_steps, const float* __restrict__ inv_base) {
    extern __shared__ __align__(16) uint8_t sm[];
    __shared__ int s_bad;
    __shared__ int jc[kGemmCols];
    const SolveUnit su = units[blockIdx.x];
    if (su.task < 0 || su.task >= tot.ntasks) return;
    const BatchTask& bt = tasks[su.task];
    const int k = k_out[su.task];
    const int64_t c_end = min(min(static_cast<int64_t>(su.c0) + su.ncols, bt.n - k), bt.tcols);
    if (k <= 0 || su.c0 < 0 || su.c0 >= c_end) return;
    const double* R = R_base + bt.r_off;
    const int32_t* J = J_base + bt.j_off;
    const int ldr = bt.kcap;
    // every index below stays inside this task's regions: check the entry and the pivot list
    if (threadIdx.x == 0) s_bad = !batch_entry_ok(bt, k, kmax, tot);
    __syncthreads();
    if (s_bad) {
        if (threadIdx.x == 0) set_info(infos + su.task, kInfoBadTable);
        return;
    }
    for (int64_t a = threadIdx.x; a < bt.n; a += blockDim.x)
        if (J[a] < 0 || J[a] >= bt.n) s_bad = 1;
    __syncthreads();
    if (s_bad) {
        if (threadIdx.x == 0) set_info(infos + su.task, kInfoBadTable);
        return;
    }
    const float* scr = inv_base + bt.inv_off;
    const int kq = gemm_kp(bt.kcap);
    double* T = T_base + bt.t_off;
    if (__ldg(reinterpret_cast<const int*>(scr + 2 * static_cast<int64_t>(kq) * kq))) {
        // an ill-conditioned R11 takes more refinement steps (each cuts the error by kappa u32)
        batched_warp_columns<KQ>(R, ldr, J, k, su.c0, c_end, T, max(refine_steps, kIllRefineSteps), sm);
        return;
    }
    const int kp = gemm_kp(k);
    float* Xs = reinterpret_cast<float*>(sm);
    float* Rs = Xs + kp * kp;
    float* Bt = Rs + kp * kp;
    float* Tt = Bt + kp * gemm_ld(kGemmCols);
    stage_x_r11(scr, kq, kp, Xs, Rs);
    for (int64_t t0 = su.c0; t0 < c_end; t0 += kGemmCols) {
        const int ncols = static_cast<int>(min(static_cast<int64_t>(kGemmCols), c_end - t0));
        if (threadIdx.x < kGemmCols) jc[threadIdx.x] = threadIdx.x < ncols ? J[k + t0 + threadIdx.x] : 0;
        __syncthreads();
        gemm_tile<KQ, kGemmCols>(R, ldr, jc, k, kp, ncols, Xs, Rs, Bt, Tt, T, t0, ldr);
    }
}

template <int KQ>
static cudaError_t launch_batched_product(const BatchTask* tasks, int ntasks, const SolveUnit* units, int nunits,
                                          int kmax, const double* R_base, const int32_t* J_base, const int32_t* k_out,
                                          int32_t* infos, double* T_base, const BatchTotals& tot, int refine_steps,
                                          float* inv, bool with_inverse, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    if (with_inverse) {
        const size_t inv_smem = (static_cast<size_t>(32 * KQ) * 32 * KQ + 32 * KQ) * sizeof(float) + 16;
        auto kinv = k_r11_inverse_batched<KQ>;
        e = cudaFuncSetAttribute(kinv, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(inv_smem));
        if (e != cudaSuccess) return e;
        const dim3 grid(static_cast<unsigned>(ntasks), static_cast<unsigned>((gemm_kp(kmax) + kWarpSolveWarps - 1) /
                                                                             kWarpSolveWarps));
        kinv<<<grid, kWarpSolveWarps * 32, inv_smem, s>>>(tasks, R_base, J_base, k_out, tot, inv);
        e = cudaGetLastError();
        if (e != cudaSuccess || nunits <= 0) return e;
    }
    const size_t smem = gemm_tile_floats(gemm_kp(kmax), kGemmCols) * sizeof(float) + 16;
    auto kern = k_solve_T_batched_gemm<KQ>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    kern<<<nunits, 16 * kGemmCols, smem, s>>>(tasks, units, R_base, J_base, k_out, infos, T_base, tot, kmax,
                                            refine_steps, inv);
    return cudaGetLastError();
}

cudaError_t launch_r11_inverse_batched(const BatchTask* tasks, int ntasks, int kmax, const double* R_base,
                                       const int32_t* J_base, const int32_t* k_out, const BatchTotals& tot, float* inv,
                                       cudaStream_t s) {
    if (ntasks <= 0) return cudaSuccess;
    if (kmax < 1 || kmax > kGemmMaxK) return cudaErrorInvalidValue;
    switch ((kmax + 31) / 32) {
        case 1: return launch_batched_product<1>(tasks, ntasks, nullptr, 0, kmax, R_base, J_base, k_out, nullptr,
                                                 nullptr, tot, 1, inv, true, s);
        case 2: return launch_batched_product<2>(tasks, ntasks, nullptr, 0, kmax, R_base, J_base, k_out, nullptr,
                                                 nullptr, tot, 1, inv, true, s);
        case 3: return launch_batched_product<3>(tasks, ntasks, nullptr, 0, kmax, R_base, J_base, k_out, nullptr,
                                                 nullptr, tot, 1, inv, true, s);
        default: return launch_batched_product<4>(tasks, ntasks, nullptr, 0, kmax, R_base, J_base, k_out, nullptr,
                                                  nullptr, tot, 1, inv, true, s);
    }
}

cudaError_t launch_solve_T_batched_product(const BatchTask* tasks, const SolveUnit* units, int nunits, int kmax,
                                           const double* R_base, const int32_t* J_base, const int32_t* k_out,
                                           int32_t* infos, double* T_base, const BatchTotals& tot, int refine_steps,
                                           const float* inv, cudaStream_t s) {
    if (nunits <= 0) return cudaSuccess;
    if (kmax < 1 || kmax > kGemmMaxK) return cudaErrorInvalidValue;
    float* iv = const_cast<float*>(inv);
    switch ((kmax + 31) / 32) {
        case 1: return launch_batched_product<1>(tasks, 0, units, nunits, kmax, R_base, J_base, k_out, infos, T_base,
                                                 tot, refine_steps, iv, false, s);
        case 2: return launch_batched_product<2>(tasks, 0, units, nunits, kmax, R_base, J_base, k_out, infos, T_base,
                                                 tot, refine_steps, iv, false, s);
        case 3: return launch_batched_product<3>(tasks, 0, units, nunits, kmax, R_base, J_base, k_out, infos, T_base,
                                                 tot, refine_steps, iv, false, s);
        default: return launch_batched_product<4>(tasks, 0, units, nunits, kmax, R_base, J_base, k_out, infos, T_base,
                                                  tot, refine_steps, iv, false, s);
    }
}

size_t batch_inverse_floats(int kcap) { return static_cast<size_t>(batch_inv_floats(kcap)); }

cudaError_t launch_solve_T(const double* R64, int64_t ldr, const int32_t* J, const int32_t* k_ptr, int kcap,
                           int64_t n, double* T, int64_t ldt, double* scratch, int refine_steps, int low_solve,
                           cudaStream_t s) {
    if (low_solve && refine_steps == 1 && kcap <= kGemmMaxK) {
        float* X = reinterpret_cast<float*>(scratch);
        switch ((kcap + 31) / 32) {
            case 1: return launch_gemm_solve<1>(R64, ldr, J, k_ptr, kcap, n, T, ldt, X, s);
            case 2: return launch_gemm_solve<2>(R64, ldr, J, k_ptr, kcap, n, T, ldt, X, s);
            case 3: return launch_gemm_solve<3>(R64, ldr, J, k_ptr, kcap, n, T, ldt, X, s);
            default: return launch_gemm_solve<4>(R64, ldr, J, k_ptr, kcap, n, T, ldt, X, s);
        }
    }
    if (kcap <= 32 * kWarpSolveMaxQ) {
        const int kq = (kcap + 31) / 32;
        if (low_solve) return launch_warp_solve_kq<float>(kq, R64, ldr, J, k_ptr, kcap, n, T, ldt, refine_steps, s);
        return launch_warp_solve_kq<double>(kq, R64, ldr, J, k_ptr, kcap, n, T, ldt, refine_steps, s);
    }
    // k > 256: thread per column, FP64 throughout, R11 read through L1/L2
    const int64_t cols = std::max<int64_t>(1, n - 1);
    const unsigned grid = static_cast<unsigned>((cols + kSolveThreads - 1) / kSolveThreads);
    k_solve_T<false><<<grid, kSolveThreads, 0, s>>>(R64, ldr, J, k_ptr, kcap, n, T, ldt, scratch, refine_steps);
    return cudaGetLastError();
}

// ------------------------------------------------------------ error estimate

// acc2[0] += sum over complement columns c of ||A(:,J[k+c]) - A(:,J[0:k]) T(:,c)||^2 by
// 64 x 64 residual tiles (256 threads, 4 x 4 entries each, k in chunks of 16 staged in
// shared memory, FP64): A(:,J[0:k]) is read once per 64 complement columns.  The grid
// covers n - 1 complement columns; k is read on the device, tiles past n - k leave.
constexpr int kResTile = 64;
constexpr int kResK = 16;

template <typename TA>
__global__ void __launch_bounds__(256)
k_residual_tiles(const TA* __restrict__ A, int64_t m, int64_t n, int64_t lda, const int32_t* __restrict__ J,
                 const int32_t* __restrict__ k_ptr, const double* __restrict__ T, int64_t ldt, double* acc2) {
    __shared__ double As[kResK][kResTile + 1];
    __shared__ double Ts[kResK][kResTile + 1];
    __shared__ double red[8];
    const int k = *k_ptr;
    const int64_t nc = n - k;
    const int64_t r0 = static_cast<int64_t>(blockIdx.x) * kResTile;
    const int64_t q0 = static_cast<int64_t>(blockIdx.y) * kResTile;
    if (k <= 0 || q0 >= nc) return;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const int64_t c = q0 + tx * 4 + v;
        const TA* col = c < nc ? A + static_cast<int64_t>(J[k + c]) * lda : nullptr;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t row = r0 + ty * 4 + u;
            acc[u][v] = (col && row < m) ? static_cast<double>(col[row]) : 0.0;
        }
    }
    for (int b0 = 0; b0 < k; b0 += kResK) {
        for (int idx = threadIdx.x; idx < kResK * kResTile; idx += 256) {
            const int bb = idx / kResTile, i = idx % kResTile;
            const int b = b0 + bb;
            const int64_t row = r0 + i, c = q0 + i;
            As[bb][i] = (b < k && row < m) ? static_cast<double>(A[static_cast<int64_t>(J[b]) * lda + row]) : 0.0;
            Ts[bb][i] = (b < k && c < nc) ? T[c * ldt + b] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int bb = 0; bb < kResK; ++bb) {
            double a[4], t[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) { a[u] = As[bb][ty * 4 + u]; t[u] = Ts[bb][tx * 4 + u]; }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(-a[u], t[v], acc[u][v]);
        }
        __syncthreads();
    }
    double sq = 0.0;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) sq = fma(acc[u][v], acc[u][v], sq);
    sq = warp_sum(sq);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < 8; ++w) tot += red[w];
        atomicAdd(acc2, tot);
    }
}

// FP32 A: the same residual with exact FP32 products.  T is split once into FP32 parts
// (Th + Tl = T to about 2^-48, k_split_T); every product a Th splits exactly into two floats
// (p = fl(a Th), e = fma(a, Th, -p)), the sums are kept as unevaluated float pairs (TwoSum)
// and a Tl goes into the low part.  The pair carries about 48 bits: the residual, even where
// it is 1e-6 of the data, keeps about nine digits, and the FP32 pipe runs it at some sixty
// times the FP64 pipe's rate.  The squares of the residual entries are summed in FP64.
__global__ void k_split_T(const double* __restrict__ T, int64_t ldt, const int32_t* __restrict__ k_ptr, int64_t n,
                          int ld, float* __restrict__ Th, float* __restrict__ Tl) {
    const int k = *k_ptr;
    const int64_t nc = n - k;
    for (int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; idx < nc * k;
         idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t c = idx / k, b = idx - c * k;
        const double t = T[c * ldt + b];
        const float h = static_cast<float>(t);
        Th[c * ld + b] = h;
        Tl[c * ld + b] = static_cast<float>(t - static_cast<double>(h));
    }
}

__global__ void __launch_bounds__(256)
k_residual_tiles_pair(const float* __restrict__ A, int64_t m, int64_t n, int64_t lda, const int32_t* __restrict__ J,
                      const int32_t* __restrict__ k_ptr, const float* __restrict__ Th, const float* __restrict__ Tl,
                      int ld, double* acc2) {
    __shared__ float As[kResK][kResTile + 1];
    __shared__ float Hs[kResK][kResTile + 1];
    __shared__ float Ls[kResK][kResTile + 1];
    __shared__ double red[8];
    const int k = *k_ptr;
    const int64_t nc = n - k;
    const int64_t r0 = static_cast<int64_t>(blockIdx.x) * kResTile;
    const int64_t q0 = static_cast<int64_t>(blockIdx.y) * kResTile;
    if (k <= 0 || q0 >= nc) return;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float hi[4][4], lo[4][4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const int64_t c = q0 + tx * 4 + v;
        const float* col = c < nc ? A + static_cast<int64_t>(J[k + c]) * lda : nullptr;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t row = r0 + ty * 4 + u;
            hi[u][v] = (col && row < m) ? col[row] : 0.f;
            lo[u][v] = 0.f;
        }
    }
    for (int b0 = 0; b0 < k; b0 += kResK) {
        for (int idx = threadIdx.x; idx < kResK * kResTile; idx += 256) {
            const int bb = idx / kResTile, i = idx % kResTile;
            const int b = b0 + bb;
            const int64_t row = r0 + i, c = q0 + i;
            As[bb][i] = (b < k && row < m) ? A[static_cast<int64_t>(J[b]) * lda + row] : 0.f;
            Hs[bb][i] = (b < k && c < nc) ? Th[c * ld + b] : 0.f;
            Ls[bb][i] = (b < k && c < nc) ? Tl[c * ld + b] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int bb = 0; bb < kResK; ++bb) {
            float na[4], th[4], tl[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                na[u] = -As[bb][ty * 4 + u];
                th[u] = Hs[bb][tx * 4 + u];
                tl[u] = Ls[bb][tx * 4 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const float p = __fmul_rn(na[u], th[v]);
                    const float e = fmaf(na[u], th[v], -p);
                    const float sum = __fadd_rn(hi[u][v], p);
                    const float bp = __fsub_rn(sum, hi[u][v]);
                    const float err = __fadd_rn(__fsub_rn(hi[u][v], __fsub_rn(sum, bp)), __fsub_rn(p, bp));
                    hi[u][v] = sum;
                    lo[u][v] = fmaf(na[u], tl[v], __fadd_rn(lo[u][v], __fadd_rn(err, e)));
                }
        }
        __syncthreads();
    }
    double sq = 0.0;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const double r = static_cast<double>(hi[u][v]) + static_cast<double>(lo[u][v]);
            sq = fma(r, r, sq);
        }
    sq = warp_sum(sq);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < 8; ++w) tot += red[w];
        atomicAdd(acc2, tot);
    }
}

// acc2[1] += ||A||_F^2 (grid-stride over the columns, warp per column).
template <typename TA>
__global__ void k_sumsq(const TA* __restrict__ A, int64_t m, int64_t n, int64_t lda, double* acc2) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    double s = 0.0;
    for (int64_t j = w0; j < n; j += nw) {
        const TA* col = A + j * lda;
        for (int64_t i = lane; i < m; i += 32) {
            const double x = static_cast<double>(col[i]);
            s = fma(x, x, s);
        }
    }
    s = warp_sum(s);
    if (lane == 0) atomicAdd(acc2 + 1, s);
}

__global__ void k_residual_finish(const double* acc2, double* err_out) {
    *err_out = acc2[1] > 0.0 ? sqrt(acc2[0] / acc2[1]) : 0.0;
}

cudaError_t launch_residual_fro(const void* A, int a_f64, int64_t m, int64_t n, int64_t lda, const int32_t* J,
                                const int32_t* k_ptr, const double* T, int64_t ldt, int kcap, double* acc2,
                                double* err_out, float* tsplit, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(acc2, 0, 2 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    const int64_t ncmax = std::max<int64_t>(1, n - 1);
    const dim3 g(static_cast<unsigned>((m + kResTile - 1) / kResTile),
                 static_cast<unsigned>((ncmax + kResTile - 1) / kResTile));
    const unsigned gs = static_cast<unsigned>(std::min<int64_t>((n * 32 + 255) / 256, 8LL * device_info().sm_count));
    if (a_f64) {
        k_residual_tiles<double><<<g, 256, 0, s>>>(static_cast<const double*>(A), m, n, lda, J, k_ptr, T, ldt, acc2);
        k_sumsq<double><<<gs, 256, 0, s>>>(static_cast<const double*>(A), m, n, lda, acc2);
    } else {
        // T split into FP32 parts (kcap x (n - 1) each, ld kcap), then the float-pair tiles
        float* Th = tsplit;
        float* Tl = tsplit + static_cast<int64_t>(kcap) * ncmax;
        const unsigned gsp = static_cast<unsigned>(std::min<int64_t>((ncmax * kcap + 255) / 256, 8LL * device_info().sm_count));
        k_split_T<<<gsp, 256, 0, s>>>(T, ldt, k_ptr, n, kcap, Th, Tl);
        k_residual_tiles_pair<<<g, 256, 0, s>>>(static_cast<const float*>(A), m, n, lda, J, k_ptr, Th, Tl, kcap,
                                                 acc2);
        k_sumsq<float><<<gs, 256, 0, s>>>(static_cast<const float*>(A), m, n, lda, acc2);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_residual_finish<<<1, 1, 0, s>>>(acc2, err_out);
    return cudaGetLastError();
}

// ------------------------------------------------------------ reconstruction

// Ahat(:, J[k + c]) = A(:, J[0:k]) T(:, c): a 64 x 64 output tile per CTA (256 threads,
// 4 x 4 outputs each), k in chunks of 16 staged in shared memory, FP64 accumulation.
constexpr int kRecTile = 64;
constexpr int kRecK = 16;

template <typename TA>
__global__ void __launch_bounds__(256)
k_reconstruct_one(const TA* __restrict__ A, int64_t m, int64_t lda, const int32_t* __restrict__ J, int k,
                  const double* __restrict__ T, int64_t ldt, int64_t nc, TA* __restrict__ Ahat, int64_t ldh) {
    __shared__ double As[kRecK][kRecTile + 1];
    __shared__ double Ts[kRecK][kRecTile + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t r0 = static_cast<int64_t>(blockIdx.x) * kRecTile;
    const int64_t q0 = static_cast<int64_t>(blockIdx.y) * kRecTile;
    double acc[4][4] = {};
    for (int b0 = 0; b0 < k; b0 += kRecK) {
        for (int idx = threadIdx.x; idx < kRecK * kRecTile; idx += 256) {
            const int bb = idx / kRecTile, i = idx % kRecTile;
            const int b = b0 + bb;
            const int64_t row = r0 + i, c = q0 + i;
            As[bb][i] = (b < k && row < m) ? static_cast<double>(A[static_cast<int64_t>(J[b]) * lda + row]) : 0.0;
            Ts[bb][i] = (b < k && c < nc) ? T[c * ldt + b] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int bb = 0; bb < kRecK; ++bb) {
            double a[4], t[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) { a[u] = As[bb][ty * 4 + u]; t[u] = Ts[bb][tx * 4 + u]; }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], t[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const int64_t c = q0 + tx * 4 + v;
        if (c >= nc) continue;
        TA* dst = Ahat + static_cast<int64_t>(J[k + c]) * ldh;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t row = r0 + ty * 4 + u;
            if (row < m) dst[row] = static_cast<TA>(acc[u][v]);
        }
    }
}

// Ahat(:, J[b]) = A(:, J[b]) for the skeleton columns b < k.
template <typename TA>
__global__ void k_copy_skeleton(const TA* __restrict__ A, int64_t m, int64_t lda, const int32_t* __restrict__ J,
                                int k, TA* __restrict__ Ahat, int64_t ldh) {
    for (int b = blockIdx.y; b < k; b += gridDim.y) {
        const int64_t col = J[b];
        for (int64_t row = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; row < m;
             row += static_cast<int64_t>(gridDim.x) * blockDim.x)
            Ahat[col * ldh + row] = A[col * lda + row];
    }
}

cudaError_t launch_reconstruct_one(const void* A, int a_f64, int64_t m, int64_t n, int64_t lda, const int32_t* J,
                                   int k, const double* T, int64_t ldt, void* Ahat, int64_t ldh, cudaStream_t s) {
    const int64_t nc = n - k;
    const dim3 gs(static_cast<unsigned>(std::min<int64_t>((m + 255) / 256, 64)),
                  static_cast<unsigned>(std::min(k, 65535)));
    if (a_f64)
        k_copy_skeleton<double><<<gs, 256, 0, s>>>(static_cast<const double*>(A), m, lda, J, k,
                                                   static_cast<double*>(Ahat), ldh);
    else
        k_copy_skeleton<float><<<gs, 256, 0, s>>>(static_cast<const float*>(A), m, lda, J, k,
                                                  static_cast<float*>(Ahat), ldh);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || nc <= 0) return e;
    const dim3 g(static_cast<unsigned>((m + kRecTile - 1) / kRecTile), static_cast<unsigned>((nc + kRecTile - 1) / kRecTile));
    if (a_f64)
        k_reconstruct_one<double><<<g, 256, 0, s>>>(static_cast<const double*>(A), m, lda, J, k, T, ldt, nc,
                                                    static_cast<double*>(Ahat), ldh);
    else
        k_reconstruct_one<float><<<g, 256, 0, s>>>(static_cast<const float*>(A), m, lda, J, k, T, ldt, nc,
                                                   static_cast<float*>(Ahat), ldh);
    return cudaGetLastError();
}

}  // namespace gid
