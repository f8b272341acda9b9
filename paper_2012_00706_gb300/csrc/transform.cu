// Data movement for the row and two-sided IDs: a transpose (the row ID of A is the column
// ID of A^T) and a gather of selected columns (the two-sided ID takes the row ID of the
// column skeleton A(:,J[0:k])).  Both keep the element type; 32 x 32 tiles through shared
// memory make the transpose's reads and writes coalesced.
#include "common.cuh"
#include "internal.h"

#include <algorithm>

namespace gid {

constexpr int kTrTile = 32;

// B (n x m, ldb) = A^T, A m x n column-major (lda).  Block (bx, by) moves the tile of rows
// [32 bx, +32) and columns [32 by, +32) of A; 32 x 8 threads, four rows each.
template <typename T>
__global__ void __launch_bounds__(256) k_transpose(const T* __restrict__ A, int64_t m, int64_t n, int64_t lda,
                                                   T* __restrict__ B, int64_t ldb) {
    __shared__ T tile[kTrTile][kTrTile + 1];
    const int64_t i0 = static_cast<int64_t>(blockIdx.x) * kTrTile, j0 = static_cast<int64_t>(blockIdx.y) * kTrTile;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t i = i0 + tx, j = j0 + ty + 8 * q;
        if (i < m && j < n) tile[ty + 8 * q][tx] = A[j * lda + i];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t j = j0 + tx, i = i0 + ty + 8 * q;
        if (i < m && j < n) B[i * ldb + j] = tile[tx][ty + 8 * q];
    }
}

cudaError_t launch_transpose(const void* A, int f64, int64_t m, int64_t n, int64_t lda, void* B, int64_t ldb,
                             cudaStream_t s) {
    const int64_t gx = (m + kTrTile - 1) / kTrTile, gy = (n + kTrTile - 1) / kTrTile;
    if (gy > 65535) return cudaErrorInvalidValue;
    const dim3 g(static_cast<unsigned>(gx), static_cast<unsigned>(gy));
    if (f64)
        k_transpose<double><<<g, 256, 0, s>>>(static_cast<const double*>(A), m, n, lda, static_cast<double*>(B), ldb);
    else
        k_transpose<float><<<g, 256, 0, s>>>(static_cast<const float*>(A), m, n, lda, static_cast<float*>(B), ldb);
    return cudaGetLastError();
}

// C(:, b) = A(:, J[b]) for b < k (C m x k, ldc).
template <typename T>
__global__ void k_gather_cols(const T* __restrict__ A, int64_t m, int64_t lda, const int32_t* __restrict__ J, int k,
                              T* __restrict__ C, int64_t ldc) {
    for (int b = blockIdx.y; b < k; b += gridDim.y) {
        const T* src = A + static_cast<int64_t>(J[b]) * lda;
        for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < m;
             i += static_cast<int64_t>(gridDim.x) * blockDim.x)
            C[b * ldc + i] = src[i];
    }
}

cudaError_t launch_gather_cols(const void* A, int f64, int64_t m, int64_t lda, const int32_t* J, int k, void* C,
                               int64_t ldc, cudaStream_t s) {
    const dim3 g(static_cast<unsigned>(std::min<int64_t>((m + 255) / 256, 64)), static_cast<unsigned>(std::min(k, 65535)));
    if (f64)
        k_gather_cols<double><<<g, 256, 0, s>>>(static_cast<const double*>(A), m, lda, J, k, static_cast<double*>(C),
                                                ldc);
    else
        k_gather_cols<float><<<g, 256, 0, s>>>(static_cast<const float*>(A), m, lda, J, k, static_cast<float*>(C), ldc);
    return cudaGetLastError();
}

}  // namespace gid
