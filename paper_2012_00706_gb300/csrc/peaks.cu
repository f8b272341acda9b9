// Profiling aid: the FP32 (FFMA) and FP64 (DFMA) arithmetic rates of this GPU, the
// denominators of the rooflines of the kernels bound by plain ALU arithmetic (the
// pivoted QR, the T solve, the plain FP64 path).  Every thread of a grid that fills
// all SMs runs eight independent multiply-add chains, so the pipe, not the chain
// latency, sets the pace; the rate is the counted flops over the CUDA-event time of
// one launch after a warm-up launch.
#include "common.cuh"
#include "internal.h"

namespace gid {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 1024;
constexpr int kProbeBlocksPerSm = 2;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_chains(T b, T c, int iters, T* sink) {
    T a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = static_cast<T>(threadIdx.x + j) * c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    // never true for the arguments the host passes; keeps the chains live
    if (sink && s == static_cast<T>(-1)) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
cudaError_t probe(int iters, double* tflops, cudaStream_t s) {
    const DeviceInfo& dev = device_info();
    const int grid = dev.sm_count * kProbeBlocksPerSm;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const T b = static_cast<T>(0.999999), c = static_cast<T>(1e-6);
    if (e == cudaSuccess) {
        k_fma_chains<T><<<grid, kProbeThreads, 0, s>>>(b, c, iters / 8, nullptr);   // warm-up
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
        k_fma_chains<T><<<grid, kProbeThreads, 0, s>>>(b, c, iters, nullptr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    const double flops = 2.0 * kChains * static_cast<double>(iters) * grid * kProbeThreads;
    *tflops = ms > 0.f ? flops / (ms * 1e-3) / 1e12 : 0.0;
    return cudaSuccess;
}

// Every float bit pattern u = base + i (i < count) widened by f64_of_f32 and by the
// hardware conversion: the bits must agree, except that a NaN need only stay a NaN (the
// hardware may return a canonical NaN).  The mismatches are counted.
__global__ void k_widen_check(uint64_t base, uint64_t count, unsigned long long* mismatches) {
    unsigned long long bad = 0;
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < count;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const float x = __uint_as_float(static_cast<uint32_t>(base + i));
        const double a = f64_of_f32(x);
        const double b = static_cast<double>(x);
        if (isnan(x) ? !isnan(a) : __double_as_longlong(a) != __double_as_longlong(b)) ++bad;
    }
    if (bad) atomicAdd(mismatches, bad);
}

}  // namespace
}  // namespace gid

extern "C" id_status_t id_check_widen(uint64_t* mismatches, void* stream) {
    if (!mismatches) return ID_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned long long* d = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&d), sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) {
        const gid::DeviceInfo& dev = gid::device_info();
        gid::k_widen_check<<<dev.sm_count * 8, 256, 0, s>>>(0ull, 1ull << 32, d);
        e = cudaGetLastError();
    }
    unsigned long long h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (d) cudaFreeAsync(d, s);
    if (e != cudaSuccess) return ID_ERR_CUDA;
    *mismatches = h;
    return ID_OK;
}

extern "C" id_status_t id_probe_fma_peak(int32_t which, double* tflops, void* stream) {
    if (!tflops || (which != 0 && which != 1)) return ID_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // about 30 ms of work at the GB300 rates (FP32 ~75 TFLOP/s, FP64 ~1.2 TFLOP/s)
    const cudaError_t e = which == 0 ? gid::probe<float>(1 << 19, tflops, s) : gid::probe<double>(1 << 13, tflops, s);
    return e == cudaSuccess ? ID_OK : ID_ERR_CUDA;
}
