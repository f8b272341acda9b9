// Adjoint of the column ID with the pivots held fixed, and the reconstruction
// A_hat = A(:, J[0:k]) P (Algorithm 1, the reconstruction), on GB300 in FP32.
//
// With X = A(:, J[0:k]), C = A(:, J[k:n]) and the least-squares coefficients
// T = X^+ C (for a column-pivoted QR of A this is exactly R11^-1 R12), the
// reconstruction is A_hat = [X, X T] in the column order of J.  Given
// G = dL/dA_hat (split into G_s = G(:, J[0:k]), G_c = G(:, J[k:n])) and
// Tb = dL/dT, the gradient w.r.t. A is (least-squares derivatives of Golub and
// Pereyra, written with the thin QR X = Q R):
//
//   B1 = Q^T G_c + R^-T Tb                    (k x (n-k))
//   B2 = R^-1 B1
//   Z  = G_c T^T + C B2^T                     (m x k)
//   K2 = Q^T Z + R^-T (Tb T^T)                (k x k)
//   dA(:, J[0:k]) = G_s + Z - Q K2,   dA(:, J[k:n]) = Q B1.
//
// The heavy terms are gather-GEMMs (columns selected through J) done by one
// batched, register-tiled FP32 kernel; the thin QR is classical Gram-Schmidt
// applied twice, one CTA per matrix; the substitutions with R and R^T run a warp per column.
#include "common.cuh"
#include "internal.h"

#include <algorithm>

namespace gid {

// ------------------------------------------------------------------ gather GEMM

// Operand element (i, j) = base[b * bstride + i * rs + col(j) * cs], col(j) = map[b * mstride + j] or j.
struct GOp {
    const float* base;
    int64_t bstride, rs, cs;
    const int32_t* map;
    int64_t mstride;
    int64_t moff;        // offset added to the map index (e.g. k for the complement J[k:n])
};

struct GOut {
    float* base;
    int64_t bstride, rs, cs;
    const int32_t* map;
    int64_t mstride, moff;
};

struct GemmArgs {
    GOp a, b;            // D (M x N) = alpha * A (M x K) * B (K x N) + beta * D
    GOut d;
    int64_t M, N, K;
    float alpha, beta;
};

// Register-tiled FP32 gather GEMM, D (M x N) = alpha A (M x K) B (K x N) + beta D, batched over
// blockIdx.z.  The tile is TM x TN with 256 threads (16 x 16, MR x NR outputs each) and TK-deep
// chunks; the next chunk is fetched into registers while the current one is multiplied, and
// the gathered indices (A's K-index map, B's and D's N-index maps) are read once per tile into
// shared memory.  Consecutive threads walk the unit-stride dimension of each operand.
constexpr int kGK = 32;

template <int TM, int TN>
__global__ void __launch_bounds__(256) k_gemm_gather(const GemmArgs g) {
    constexpr int MR = TM / 16, NR = TN / 16;
    constexpr int LA = TM * kGK / 256, LB = TN * kGK / 256;   // elements per thread per chunk
    __shared__ __align__(16) float As[kGK][TM + 4];
    __shared__ __align__(16) float Bs[kGK][TN + 4];
    __shared__ int64_t amap[kGK];         // A column offsets (col(k) * cs) of the current chunk
    __shared__ int64_t bmap[TN], dmap[TN];
    const int64_t b = blockIdx.z;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t i0 = static_cast<int64_t>(blockIdx.y) * TM, j0 = static_cast<int64_t>(blockIdx.x) * TN;
    const float* abase = g.a.base + b * g.a.bstride;
    const float* bbase = g.b.base + b * g.b.bstride;
    for (int t = threadIdx.x; t < TN; t += 256) {
        const int64_t j = min(j0 + t, g.N - 1);
        bmap[t] = (g.b.map ? static_cast<int64_t>(g.b.map[b * g.b.mstride + g.b.moff + j]) : j) * g.b.cs;
        dmap[t] = (g.d.map ? static_cast<int64_t>(g.d.map[b * g.d.mstride + g.d.moff + j]) : j) * g.d.cs;
    }
    // element e of this thread's share of a chunk: (row, k) of A and (k, column) of B
    auto a_rc = [&](int e, int& ii, int& kk) {
        const int idx = threadIdx.x + 256 * e;
        if (g.a.rs == 1) { ii = idx % TM; kk = idx / TM; } else { kk = idx % kGK; ii = idx / kGK; }
    };
    auto b_rc = [&](int e, int& kk, int& jj) {
        const int idx = threadIdx.x + 256 * e;
        if (g.b.rs == 1) { kk = idx % kGK; jj = idx / kGK; } else { jj = idx % TN; kk = idx / TN; }
    };
    float ra[LA], rb[LB];
    auto fetch = [&](int64_t k0) {
        // amap for this chunk: written by the first kGK threads, read after a barrier
        __syncthreads();
        if (threadIdx.x < kGK) {
            const int64_t kg = min(k0 + threadIdx.x, g.K - 1);
            amap[threadIdx.x] =
                (g.a.map ? static_cast<int64_t>(g.a.map[b * g.a.mstride + g.a.moff + kg]) : kg) * g.a.cs;
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < LA; ++e) {
            int ii, kk;
            a_rc(e, ii, kk);
            const int64_t gi = i0 + ii, gk = k0 + kk;
            ra[e] = (gi < g.M && gk < g.K) ? abase[gi * g.a.rs + amap[kk]] : 0.f;
        }
#pragma unroll
        for (int e = 0; e < LB; ++e) {
            int kk, jj;
            b_rc(e, kk, jj);
            const int64_t gj = j0 + jj, gk = k0 + kk;
            rb[e] = (gj < g.N && gk < g.K) ? bbase[gk * g.b.rs + bmap[jj]] : 0.f;
        }
    };
    float acc[MR][NR] = {};
    fetch(0);
    for (int64_t k0 = 0; k0 < g.K; k0 += kGK) {
        __syncthreads();     // the previous chunk's reads of As / Bs are done
#pragma unroll
        for (int e = 0; e < LA; ++e) {
            int ii, kk;
            a_rc(e, ii, kk);
            As[kk][ii] = ra[e];
        }
#pragma unroll
        for (int e = 0; e < LB; ++e) {
            int kk, jj;
            b_rc(e, kk, jj);
            Bs[kk][jj] = rb[e];
        }
        if (k0 + kGK < g.K) fetch(k0 + kGK);   // in flight during the products below
        else __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < kGK; ++kk) {
            float av[MR], bv[NR];
#pragma unroll
            for (int p = 0; p < MR; ++p) av[p] = As[kk][ty * MR + p];
#pragma unroll
            for (int q = 0; q < NR; ++q) bv[q] = Bs[kk][tx * NR + q];
#pragma unroll
            for (int p = 0; p < MR; ++p)
#pragma unroll
                for (int q = 0; q < NR; ++q) acc[p][q] = fmaf(av[p], bv[q], acc[p][q]);
        }
    }
    float* dbase = g.d.base + b * g.d.bstride;
#pragma unroll
    for (int p = 0; p < MR; ++p) {
        const int64_t gi = i0 + ty * MR + p;
        if (gi >= g.M) continue;
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            const int jj = tx * NR + q;
            if (j0 + jj >= g.N) continue;
            float* dst = dbase + gi * g.d.rs + dmap[jj];
            *dst = g.beta == 0.f ? g.alpha * acc[p][q] : fmaf(g.alpha, acc[p][q], g.beta * *dst);
        }
    }
}

static cudaError_t gemm(const GemmArgs& g, int64_t batch, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    const unsigned z = static_cast<unsigned>(batch);
    // tile shapes for the ranks of the adjoint's products (one side often k <= 32)
    if (g.M <= 32) {
        dim3 grid(static_cast<unsigned>((g.N + 127) / 128), static_cast<unsigned>((g.M + 31) / 32), z);
        k_gemm_gather<32, 128><<<grid, 256, 0, s>>>(g);
    } else if (g.N <= 32) {
        dim3 grid(static_cast<unsigned>((g.N + 31) / 32), static_cast<unsigned>((g.M + 127) / 128), z);
        k_gemm_gather<128, 32><<<grid, 256, 0, s>>>(g);
    } else {
        dim3 grid(static_cast<unsigned>((g.N + 63) / 64), static_cast<unsigned>((g.M + 63) / 64), z);
        k_gemm_gather<64, 64><<<grid, 256, 0, s>>>(g);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ thin QR (CGS2)

// Q R = A(:, J[0:k]) by classical Gram-Schmidt applied twice, one CTA per matrix.
// Q: m x k (ld m), R: k x k upper (ld k), FP32.
__global__ void __launch_bounds__(512) k_cgs2(const float* __restrict__ A, int64_t lda, int64_t strideA, int64_t m,
                                              const int32_t* __restrict__ J, int64_t strideJ, int k,
                                              float* __restrict__ Q, float* __restrict__ R) {
    extern __shared__ float sh[];
    float* h = sh;              // k projections
    float* red = sh + 128;      // warp partials
    const int64_t b = blockIdx.x;
    const float* a = A + b * strideA;
    const int32_t* jj = J + b * strideJ;
    float* q = Q + b * m * k;
    float* r = R + b * k * k;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
    for (int idx = t; idx < k * k; idx += blockDim.x) r[idx] = 0.f;
    for (int j = 0; j < k; ++j) {
        float* qj = q + static_cast<int64_t>(j) * m;
        const float* aj = a + static_cast<int64_t>(jj[j]) * lda;
        for (int64_t i = t; i < m; i += blockDim.x) qj[i] = aj[i];
        __syncthreads();
        for (int pass = 0; pass < 2; ++pass) {
            // h = Q(:, 0:j)^T q_j : warp w computes entries w, w + nw, ...
            for (int c = warp; c < j; c += nw) {
                const float* qc = q + static_cast<int64_t>(c) * m;
                float s = 0.f;
                for (int64_t i = lane; i < m; i += 32) s = fmaf(qc[i], qj[i], s);
                s = warp_sum(s);
                if (lane == 0) h[c] = s;
            }
            __syncthreads();
            for (int64_t i = t; i < m; i += blockDim.x) {
                float v = qj[i];
                for (int c = 0; c < j; ++c) v = fmaf(-h[c], q[static_cast<int64_t>(c) * m + i], v);
                qj[i] = v;
            }
            if (t < j) r[static_cast<int64_t>(j) * k + t] += h[t];
            __syncthreads();
        }
        float s = 0.f;
        for (int64_t i = t; i < m; i += blockDim.x) s = fmaf(qj[i], qj[i], s);
        s = warp_sum(s);
        if (lane == 0) red[warp] = s;
        __syncthreads();
        if (t == 0) {
            float tot = 0.f;
            for (int w = 0; w < nw; ++w) tot += red[w];
            red[32] = sqrtf(tot);
            r[static_cast<int64_t>(j) * k + j] = red[32];
        }
        __syncthreads();
        const float inv = red[32] > 0.f ? 1.f / red[32] : 0.f;
        for (int64_t i = t; i < m; i += blockDim.x) qj[i] *= inv;
        __syncthreads();
    }
}

// ------------------------------------------------------------------ small k x k pieces

// Warp-per-column substitutions with R (k x k upper, FP32) staged in shared memory twice: rc
// column-major (column a contiguous: R(0:a, a)) and rt row-major (row a contiguous: R(a, a:k)),
// so that every step's reads are contiguous across the lanes.  Lane l holds rows l, l + 32, ...
// (KQ blocks of 32); the steps run by block from a compile-time register index.
__device__ __forceinline__ void stage_r_both(const float* __restrict__ R, int k, float* rc, float* rt) {
    for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) {
        const int a = idx / k, r = idx - a * k;          // R(r, a) = R[a k + r]
        const float v = R[idx];
        rc[idx] = v;
        rt[r * k + a] = v;
    }
}

// y = R^-T t (forward substitution: y_a = (t_a - sum_{i<a} R(i,a) y_i) / R(a,a)).
template <int KQ>
__device__ __forceinline__ void warp_fwd_rt(float (&t)[KQ], const float* rc, const float* rt, int k, int lane) {
#pragma unroll
    for (int qa = 0; qa < KQ; ++qa) {
        const int a_end = min(32 * qa + 32, k);
        for (int a = 32 * qa; a < a_end; ++a) {
            const int i = a - 32 * qa;
            const float ya = __shfl_sync(0xffffffffu, t[qa], i) / rc[a * k + a];
            const float* row = rt + a * k + lane;           // R(a, lane + 32 q)
            if (lane == i) t[qa] = ya;
            else if (lane > i && lane + 32 * qa < k) t[qa] = fmaf(-row[32 * qa], ya, t[qa]);
#pragma unroll
            for (int q = qa + 1; q < KQ; ++q)
                if (lane + 32 * q < k) t[q] = fmaf(-row[32 * q], ya, t[q]);
        }
    }
}

// x = R^-1 t (back substitution).
template <int KQ>
__device__ __forceinline__ void warp_back_r(float (&t)[KQ], const float* rc, int k, int lane) {
#pragma unroll
    for (int qa = KQ - 1; qa >= 0; --qa) {
        for (int a = min(32 * qa + 31, k - 1); a >= 32 * qa; --a) {
            const int i = a - 32 * qa;
            const float xa = __shfl_sync(0xffffffffu, t[qa], i) / rc[a * k + a];
            const float* col = rc + a * k + lane;           // R(lane + 32 q, a)
            if (lane == i) t[qa] = xa;
            else if (lane < i) t[qa] = fmaf(-col[32 * qa], xa, t[qa]);
#pragma unroll
            for (int q = 0; q < qa; ++q) t[q] = fmaf(-col[32 * q], xa, t[q]);
        }
    }
}

// B1 = B0 + R^-T Tb (Tb nullable), then B2 = R^-1 B1, for the columns of one matrix
// (blockIdx.y): a warp per column.
template <int KQ>
__global__ void __launch_bounds__(256) k_bwd_b(const float* __restrict__ R, int k, int64_t ncols,
                                               const float* __restrict__ B0, const float* __restrict__ Tb, int64_t ldtb,
                                               int64_t strideTb, float* __restrict__ B1, float* __restrict__ B2) {
    extern __shared__ float rs[];
    const int64_t b = blockIdx.y;
    float* rc = rs;
    float* rt = rs + k * k;
    stage_r_both(R + b * k * k, k, rc, rt);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    for (int64_t c = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); c < ncols;
         c += nwarps) {
        const float* b0 = B0 + (b * ncols + c) * k;
        float y[KQ], x[KQ];
#pragma unroll
        for (int q = 0; q < KQ; ++q) {
            const int r = lane + 32 * q;
            y[q] = (Tb && r < k) ? Tb[b * strideTb + c * ldtb + r] : 0.f;
        }
        if (Tb) warp_fwd_rt<KQ>(y, rc, rt, k, lane);
#pragma unroll
        for (int q = 0; q < KQ; ++q) {
            const int r = lane + 32 * q;
            x[q] = r < k ? b0[r] + y[q] : 0.f;
            if (r < k) B1[(b * ncols + c) * k + r] = x[q];
        }
        warp_back_r<KQ>(x, rc, k, lane);
#pragma unroll
        for (int q = 0; q < KQ; ++q) {
            const int r = lane + 32 * q;
            if (r < k) B2[(b * ncols + c) * k + r] = x[q];
        }
    }
}

// K2 = H + R^-T E (k x k column-major per matrix; E nullable): a warp per column.
template <int KQ>
__global__ void __launch_bounds__(256) k_bwd_k2(const float* __restrict__ R, int k, const float* __restrict__ H,
                                                const float* __restrict__ E, float* __restrict__ K2) {
    extern __shared__ float rs[];
    const int64_t b = blockIdx.y;
    float* rc = rs;
    float* rt = rs + k * k;
    stage_r_both(R + b * k * k, k, rc, rt);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= k) return;
    const float* hb = H + b * k * k + static_cast<int64_t>(c) * k;
    float y[KQ];
#pragma unroll
    for (int q = 0; q < KQ; ++q) {
        const int r = lane + 32 * q;
        y[q] = (E && r < k) ? E[b * k * k + static_cast<int64_t>(c) * k + r] : 0.f;
    }
    if (E) warp_fwd_rt<KQ>(y, rc, rt, k, lane);
#pragma unroll
    for (int q = 0; q < KQ; ++q) {
        const int r = lane + 32 * q;
        if (r < k) K2[b * k * k + static_cast<int64_t>(c) * k + r] = hb[r] + y[q];
    }
}

template <int KQ>
static cudaError_t launch_bwd_small(bool is_b, const float* R, int k, int64_t ncols, const float* B0, const float* Tb,
                                    int64_t ldtb, int64_t strideTb, float* B1, float* B2, const float* H,
                                    const float* E, float* K2, int64_t batch, cudaStream_t s) {
    const size_t smem = 2 * static_cast<size_t>(k) * k * sizeof(float);
    cudaError_t e;
    if (is_b) {
        auto kern = k_bwd_b<KQ>;
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem))) !=
            cudaSuccess)
            return e;
        const int64_t blocks = std::min<int64_t>((ncols + 7) / 8, 64);
        kern<<<dim3(static_cast<unsigned>(blocks), static_cast<unsigned>(batch)), 256, smem, s>>>(
            R, k, ncols, B0, Tb, ldtb, strideTb, B1, B2);
    } else {
        auto kern = k_bwd_k2<KQ>;
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem))) !=
            cudaSuccess)
            return e;
        kern<<<dim3(static_cast<unsigned>((k + 7) / 8), static_cast<unsigned>(batch)), 256, smem, s>>>(R, k, H, E,
                                                                                                   K2);
    }
    return cudaGetLastError();
}

static cudaError_t bwd_small(bool is_b, const float* R, int k, int64_t ncols, const float* B0, const float* Tb,
                             int64_t ldtb, int64_t strideTb, float* B1, float* B2, const float* H, const float* E,
                             float* K2, int64_t batch, cudaStream_t s) {
    switch ((k + 31) / 32) {
        case 1: return launch_bwd_small<1>(is_b, R, k, ncols, B0, Tb, ldtb, strideTb, B1, B2, H, E, K2, batch, s);
        case 2: return launch_bwd_small<2>(is_b, R, k, ncols, B0, Tb, ldtb, strideTb, B1, B2, H, E, K2, batch, s);
        case 3: return launch_bwd_small<3>(is_b, R, k, ncols, B0, Tb, ldtb, strideTb, B1, B2, H, E, K2, batch, s);
        default: return launch_bwd_small<4>(is_b, R, k, ncols, B0, Tb, ldtb, strideTb, B1, B2, H, E, K2, batch, s);
    }
}

// dA(:, J[0:k]) += G_s (or 0) : X_bar starts as G_s, the GEMMs accumulate Z - Q K2 into it.
__global__ void k_copy_cols(const float* __restrict__ G, int64_t ldg, int64_t strideG, int64_t m,
                            const int32_t* __restrict__ J, int64_t strideJ, int k, float* __restrict__ D,
                            int64_t ldd, int64_t strideD) {
    const int64_t b = blockIdx.z;
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (i >= m || c >= k) return;
    const int64_t col = J[b * strideJ + c];
    D[b * strideD + col * ldd + i] = G ? G[b * strideG + col * ldg + i] : 0.f;
}

__global__ void k_t_to_f32(const double* __restrict__ T, int64_t ldt, int64_t strideT, int k, int64_t ncols,
                           float* __restrict__ Tf) {
    const int64_t b = blockIdx.y;
    const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= ncols * k) return;
    const int64_t c = idx / k, a = idx % k;
    Tf[(b * ncols + c) * k + a] = static_cast<float>(T[b * strideT + c * ldt + a]);
}

// ------------------------------------------------------------------ orchestration

struct BwdWork {
    float *Q, *R, *Tf, *Tbf, *B0, *B1, *B2, *H, *E, *K2;
};

static size_t bwd_carve(void* base, int64_t batch, int64_t m, int64_t n, int k, BwdWork* w) {
    Carver c(base);
    const int64_t nc = n - k;
    BwdWork x;
    x.Q = c.take<float>(batch * m * k);
    x.R = c.take<float>(batch * k * k);
    x.Tf = c.take<float>(batch * nc * k);
    x.Tbf = c.take<float>(batch * nc * k);
    x.B0 = c.take<float>(batch * nc * k);
    x.B1 = c.take<float>(batch * nc * k);
    x.B2 = c.take<float>(batch * nc * k);
    x.H = c.take<float>(batch * k * k);
    x.E = c.take<float>(batch * k * k);
    x.K2 = c.take<float>(batch * k * k);
    if (w) *w = x;
    return c.off + 256;
}

size_t backward_workspace_bytes(int64_t batch, int64_t m, int64_t n, int k) {
    return bwd_carve(nullptr, batch, m, n, k, nullptr);
}

cudaError_t launch_backward(int64_t batch, const float* A, int64_t m, int64_t n, int64_t lda, int64_t strideA,
                            const int32_t* J, int64_t strideJ, int k, const double* T, int64_t ldt, int64_t strideT,
                            const float* G, int64_t ldg, int64_t strideG, const double* Tb64, int64_t ldtb64,
                            int64_t strideTb64, float* dA, int64_t ldd, int64_t strideD, void* work, cudaStream_t s) {
    BwdWork w;
    bwd_carve(work, batch, m, n, k, &w);
    const int64_t nc = n - k;
    cudaError_t e;
    // dL/dT arrives in double (like T); the arithmetic below is FP32
    const float* Tb = nullptr;
    const int64_t ldtb = k, strideTb = nc * k;
    if (Tb64 && nc > 0) {
        dim3 g0(static_cast<unsigned>((nc * k + 255) / 256), static_cast<unsigned>(batch));
        k_t_to_f32<<<g0, 256, 0, s>>>(Tb64, ldtb64, strideTb64, k, nc, w.Tbf);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        Tb = w.Tbf;
    }
    // thin QR of the skeleton
    k_cgs2<<<static_cast<unsigned>(batch), 512, (128 + 33) * sizeof(float), s>>>(A, lda, strideA, m, J, strideJ, k,
                                                                                   w.Q, w.R);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (nc > 0) {
        dim3 g1(static_cast<unsigned>((nc * k + 255) / 256), static_cast<unsigned>(batch));
        k_t_to_f32<<<g1, 256, 0, s>>>(T, ldt, strideT, k, nc, w.Tf);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // X_bar starts as G_s (or zero)
    {
        dim3 gc(static_cast<unsigned>((m + 255) / 256), static_cast<unsigned>(k), static_cast<unsigned>(batch));
        k_copy_cols<<<gc, 256, 0, s>>>(G, ldg, strideG, m, J, strideJ, k, dA, ldd, strideD);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const GOp Qt{w.Q, m * k, m, 1, nullptr, 0, 0};                       // Q^T (k x m): (i, j) = Q[j + i m]
    const GOp Qn{w.Q, m * k, 1, m, nullptr, 0, 0};                       // Q   (m x k)
    const GOp Gc{G, strideG, 1, ldg, J, strideJ, k};                     // G_c (m x nc), columns J[k + j]
    const GOp Cc{A, strideA, 1, lda, J, strideJ, k};                     // C   (m x nc)
    const GOp TfT{w.Tf, nc * k, k, 1, nullptr, 0, 0};                    // T^T (nc x k): (i, j) = T(j, i) = Tf[i k + j]
    if (nc > 0) {
        // B0 = Q^T G_c  (k x nc), stored column-major ld k
        if (G) {
            GemmArgs g{Qt, Gc, GOut{w.B0, nc * k, 1, k, nullptr, 0, 0}, k, nc, m, 1.f, 0.f};
            if ((e = gemm(g, batch, s)) != cudaSuccess) return e;
        } else {
            if ((e = cudaMemsetAsync(w.B0, 0, sizeof(float) * batch * nc * k, s)) != cudaSuccess) return e;
        }
        // B1 = B0 + R^-T Tb, B2 = R^-1 B1
        if ((e = bwd_small(true, w.R, k, nc, w.B0, Tb, ldtb, strideTb, w.B1, w.B2, nullptr, nullptr, nullptr, batch,
                           s)) != cudaSuccess)
            return e;
        // Z = G_c T^T + C B2^T  accumulated into X_bar (= dA(:, J[0:k]))
        const GOut Xb{dA, strideD, 1, ldd, J, strideJ, 0};
        if (G) {
            GemmArgs g{Gc, TfT, Xb, m, k, nc, 1.f, 1.f};
            if ((e = gemm(g, batch, s)) != cudaSuccess) return e;
        }
        {
            // B operand (nc x k): (kk, j) = B2(j, kk) = B2[kk * k + j]
            GemmArgs g{Cc, GOp{w.B2, nc * k, k, 1, nullptr, 0, 0}, Xb, m, k, nc, 1.f, 1.f};
            if ((e = gemm(g, batch, s)) != cudaSuccess) return e;
        }
        // E = Tb T^T (k x k)
        if (Tb) {
            GemmArgs g{GOp{Tb, strideTb, 1, ldtb, nullptr, 0, 0}, TfT, GOut{w.E, k * k, 1, k, nullptr, 0, 0}, k, k, nc,
                       1.f, 0.f};
            if ((e = gemm(g, batch, s)) != cudaSuccess) return e;
        }
    }
    // H = Q^T Z with Z = X_bar - G_s: H = Q^T X_bar - Q^T G_s
    {
        const GOp Xbar{dA, strideD, 1, ldd, J, strideJ, 0};
        GemmArgs g{Qt, Xbar, GOut{w.H, k * k, 1, k, nullptr, 0, 0}, k, k, m, 1.f, 0.f};
        if ((e = gemm(g, batch, s)) != cudaSuccess) return e;
        if (G) {
            const GOp Gs{G, strideG, 1, ldg, J, strideJ, 0};
            GemmArgs g2{Qt, Gs, GOut{w.H, k * k, 1, k, nullptr, 0, 0}, k, k, m, -1.f, 1.f};
            if ((e = gemm(g2, batch, s)) != cudaSuccess) return e;
        }
    }
    // K2 = H + R^-T E
    if ((e = bwd_small(false, w.R, k, 0, nullptr, nullptr, 0, 0, nullptr, nullptr, w.H, (Tb && nc > 0) ? w.E : nullptr,
                       w.K2, batch, s)) != cudaSuccess)
        return e;
    // X_bar -= Q K2
    {
        const GOut Xb{dA, strideD, 1, ldd, J, strideJ, 0};
        GemmArgs g{Qn, GOp{w.K2, k * k, 1, k, nullptr, 0, 0}, Xb, m, k, k, -1.f, 1.f};
        if ((e = gemm(g, batch, s)) != cudaSuccess) return e;
    }
    // C_bar = Q B1 -> dA(:, J[k:n])
    if (nc > 0) {
        GemmArgs g{Qn, GOp{w.B1, nc * k, 1, k, nullptr, 0, 0}, GOut{dA, strideD, 1, ldd, J, strideJ, k}, m, nc, k, 1.f,
                   0.f};
        if ((e = gemm(g, batch, s)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// A_hat = A(:, J[0:k]) P: A_hat(:, J[0:k]) = A(:, J[0:k]), A_hat(:, J[k:n]) = A(:, J[0:k]) T.
cudaError_t launch_reconstruct(int64_t batch, const float* A, int64_t m, int64_t n, int64_t lda, int64_t strideA,
                               const int32_t* J, int64_t strideJ, int k, const double* T, int64_t ldt, int64_t strideT,
                               float* Ahat, int64_t ldh, int64_t strideH, void* work, cudaStream_t s) {
    const int64_t nc = n - k;
    float* Tf = static_cast<float*>(work);
    cudaError_t e;
    dim3 gc(static_cast<unsigned>((m + 255) / 256), static_cast<unsigned>(k), static_cast<unsigned>(batch));
    k_copy_cols<<<gc, 256, 0, s>>>(A, lda, strideA, m, J, strideJ, k, Ahat, ldh, strideH);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (nc <= 0) return cudaSuccess;
    dim3 g1(static_cast<unsigned>((nc * k + 255) / 256), static_cast<unsigned>(batch));
    k_t_to_f32<<<g1, 256, 0, s>>>(T, ldt, strideT, k, nc, Tf);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const GOp Xs{A, strideA, 1, lda, J, strideJ, 0};
    GemmArgs g{Xs, GOp{Tf, nc * k, 1, k, nullptr, 0, 0}, GOut{Ahat, strideH, 1, ldh, J, strideJ, k}, m, nc, k, 1.f, 0.f};
    return gemm(g, batch, s);
}

size_t reconstruct_workspace_bytes(int64_t batch, int64_t n, int k) {
    return static_cast<size_t>(batch) * static_cast<size_t>(n > k ? n - k : 0) * k * sizeof(float) + 256;
}

}  // namespace gid

using namespace gid;

extern "C" {

id_status_t id_backward_workspace_size(int64_t batch, int64_t m, int64_t n, int32_t k, size_t* bytes) {
    if (!bytes || batch < 1 || m < 1 || n < 1 || k < 1 || k > 128 || k > n || k > m) return ID_ERR_ARG;
    *bytes = backward_workspace_bytes(batch, m, n, k);
    return ID_OK;
}

id_status_t id_backward(int64_t batch, const float* A, int64_t m, int64_t n, int64_t lda, int64_t strideA,
                        const int32_t* J, int64_t strideJ, int32_t k, const double* T, int64_t ldt, int64_t strideT,
                        const float* dAhat, int64_t ldg, int64_t strideG, const double* dT, int64_t lddt,
                        int64_t strideDT, float* dA, int64_t ldd, int64_t strideD, void* work, size_t work_bytes,
                        void* stream) {
    size_t need = 0;
    if (id_backward_workspace_size(batch, m, n, k, &need) != ID_OK) return ID_ERR_ARG;
    if (!A || !J || !dA || !work || (!T && n > k) || lda < m || ldd < m || ldt < k || strideJ < n) return ID_ERR_ARG;
    if (dAhat && ldg < m) return ID_ERR_ARG;
    if (dT && lddt < k) return ID_ERR_ARG;
    if (work_bytes < need) return ID_ERR_WORKSPACE;
    void* aligned = reinterpret_cast<void*>((reinterpret_cast<uintptr_t>(work) + 255) & ~uintptr_t(255));
    const cudaError_t e = launch_backward(batch, A, m, n, lda, strideA, J, strideJ, k, T, ldt, strideT, dAhat, ldg,
                                          strideG, dT, lddt, strideDT, dA, ldd, strideD, aligned,
                                          static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ID_OK : ID_ERR_CUDA;
}

id_status_t id_reconstruct_workspace_size(int64_t batch, int64_t n, int32_t k, size_t* bytes) {
    if (!bytes || batch < 1 || n < 1 || k < 1 || k > n) return ID_ERR_ARG;
    *bytes = reconstruct_workspace_bytes(batch, n, k);
    return ID_OK;
}

id_status_t id_reconstruct(int64_t batch, const float* A, int64_t m, int64_t n, int64_t lda, int64_t strideA,
                           const int32_t* J, int64_t strideJ, int32_t k, const double* T, int64_t ldt, int64_t strideT,
                           float* Ahat, int64_t ldh, int64_t strideH, void* work, size_t work_bytes, void* stream) {
    size_t need = 0;
    if (id_reconstruct_workspace_size(batch, n, k, &need) != ID_OK) return ID_ERR_ARG;
    if (!A || !J || !Ahat || !work || (!T && n > k) || m < 1 || lda < m || ldh < m || ldt < k || strideJ < n)
        return ID_ERR_ARG;
    if (work_bytes < need) return ID_ERR_WORKSPACE;
    void* aligned = reinterpret_cast<void*>((reinterpret_cast<uintptr_t>(work) + 255) & ~uintptr_t(255));
    const cudaError_t e = launch_reconstruct(batch, A, m, n, lda, strideA, J, strideJ, k, T, ldt, strideT, Ahat, ldh,
                                             strideH, aligned, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ID_OK : ID_ERR_CUDA;
}

}  // extern "C"
