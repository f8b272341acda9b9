// Coefficient matrix and error estimate of the column ID on GB300.
//
// T = R11^-1 R12 (Algorithm 1 line 4; R11 upper triangular and nonsingular, so
// its pseudo-inverse of the paper's Remark is its inverse), in FP64 by
// back-substitution, followed by `refine_steps` steps of iterative refinement
// T += R11^-1 (R12 - R11 T) with the residual formed in FP64.  The pivoted QR
// leaves R in FP64 storage (exactly, whatever precision it ran in), so the
// solve is independent of the factorisation's precision.
//
// R11 sits in shared memory (read as warp-wide broadcasts); one thread owns
// one column of T.  The work is FP64-ALU bound: about k^2 (n-k) flops per
// solve pass.
#include "common.cuh"
#include "internal.h"

#include <algorithm>

namespace gid {

constexpr int kSolveThreads = 64;
constexpr int kSmemR11MaxK = 150;

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

size_t solve_T_scratch_doubles(int kcap, int64_t n) { return static_cast<size_t>(kcap) * static_cast<size_t>(n); }

cudaError_t launch_solve_T(const double* R64, int64_t ldr, const int32_t* J, const int32_t* k_ptr, int kcap,
                           int64_t n, double* T, int64_t ldt, double* scratch, int refine_steps,
                           cudaStream_t s) {
    const int64_t cols = std::max<int64_t>(1, n - 1);
    const unsigned grid = static_cast<unsigned>((cols + kSolveThreads - 1) / kSolveThreads);
    if (kcap <= kSmemR11MaxK) {
        const size_t smem = static_cast<size_t>(kcap) * kcap * sizeof(double);
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k_solve_T<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 static_cast<int>(smem));
            if (e != cudaSuccess) return e;
        }
        k_solve_T<true><<<grid, kSolveThreads, smem, s>>>(R64, ldr, J, k_ptr, kcap, n, T, ldt, scratch,
                                                          refine_steps);
    } else {
        k_solve_T<false><<<grid, kSolveThreads, 0, s>>>(R64, ldr, J, k_ptr, kcap, n, T, ldt, scratch,
                                                        refine_steps);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------ error estimate

// acc2[0] += sum over complement columns c of ||A(:,Jc[c]) - A(:,J[0:k]) T(:,c)||^2,
// acc2[1] += ||A||_F^2.  One warp per column, FP64.
template <typename TA>
__global__ void k_residual_fro(const TA* __restrict__ A, int64_t m, int64_t n, int64_t lda,
                               const int32_t* __restrict__ J, const int32_t* __restrict__ k_ptr,
                               const double* __restrict__ T, int64_t ldt, double* acc2) {
    const int k = *k_ptr;
    const int lane = threadIdx.x & 31;
    const int64_t w = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    if (w >= n) return;
    double res = 0.0, tot = 0.0;
    const int64_t col = J[w];
    const TA* a = A + col * lda;
    for (int64_t i = lane; i < m; i += 32) {
        const double x = static_cast<double>(a[i]);
        tot += x * x;
        if (w >= k) {
            const double* t = T + (w - k) * ldt;
            double r = x;
            for (int b = 0; b < k; ++b) r = fma(-static_cast<double>(A[static_cast<int64_t>(J[b]) * lda + i]), t[b], r);
            res += r * r;
        }
    }
    res = warp_sum(res);
    tot = warp_sum(tot);
    if (lane == 0) {
        atomicAdd(acc2, res);
        atomicAdd(acc2 + 1, tot);
    }
}

__global__ void k_residual_finish(const double* acc2, double* err_out) {
    *err_out = acc2[1] > 0.0 ? sqrt(acc2[0] / acc2[1]) : 0.0;
}

cudaError_t launch_residual_fro(const void* A, int a_f64, int64_t m, int64_t n, int64_t lda, const int32_t* J,
                                const int32_t* k_ptr, const double* T, int64_t ldt, double* acc2,
                                double* err_out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(acc2, 0, 2 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    const unsigned grid = static_cast<unsigned>((n * 32 + 255) / 256);
    if (a_f64)
        k_residual_fro<double><<<grid, 256, 0, s>>>(static_cast<const double*>(A), m, n, lda, J, k_ptr, T, ldt, acc2);
    else
        k_residual_fro<float><<<grid, 256, 0, s>>>(static_cast<const float*>(A), m, n, lda, J, k_ptr, T, ldt, acc2);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_residual_finish<<<1, 1, 0, s>>>(acc2, err_out);
    return cudaGetLastError();
}

}  // namespace gid
