// id_sketch_noalloc: the sketch Y = Omega A without any caller workspace.
//
// Some callers cannot allocate device memory when they call the library: a
// plug-in whose host framework owns every device allocation, a service whose
// memory budget is fixed when it starts, code that must not allocate while it
// runs.  For them the split-K partial sums of the sketch live in a file-scope
// device array of ID_NOALLOC_SCRATCH_BYTES bytes instead of the `work` buffer.
// Every GPU that loads this library holds that array until the process exits.
//
// The array is shared by every call on a device and keeps the last call's
// contents: calls that overlap on the GPU (different streams, or different
// host threads on one device) race on it and must be serialised by the caller.
// Nothing in it has to start at zero: each call writes every partial sum it
// later reads.  No cudaMalloc, cudaFree or allocating library routine is used.
#include "common.cuh"
#include "internal.h"

#include <mutex>
#include <vector>

namespace gid {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[ID_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress once per device (with that device current) and cached.
cudaError_t scratch_address(void** out) {
    static std::mutex mu;
    static std::vector<void*> addr;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (static_cast<int>(addr.size()) <= dev) addr.resize(dev + 1, nullptr);
    if (!addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        addr[dev] = p;
    }
    *out = addr[dev];
    return cudaSuccess;
}

bool is_mixed_precision(int p) {
    return p == ID_MIXED_BF16 || p == ID_MIXED_F16 || p == ID_MIXED_BF16X2 || p == ID_MIXED_BF16X3;
}

}  // namespace
}  // namespace gid

using namespace gid;

extern "C" id_status_t id_sketch_noalloc(const void* A, id_dtype_t a_dtype, int64_t m, int64_t n, int64_t lda,
                                         const void* omega, int64_t omega_ld, int32_t ell, int32_t precision,
                                         void* Y, int64_t ldy, int32_t* info, void* stream) {
    if (!A || !omega || !Y || m < 1 || n < 1 || lda < m || ell < 1 || ell > m || ldy < ell) return ID_ERR_ARG;
    if (a_dtype != ID_F64 && a_dtype != ID_F32) return ID_ERR_ARG;
    const int64_t ldo = omega_ld > 0 ? omega_ld : m;
    if (ldo < m) return ID_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    size_t need = 0;
    SketchPlan sp;
    SketchF64Plan sp64;
    if (precision == ID_PLAIN_F64) {
        if (a_dtype != ID_F64) return ID_ERR_ARG;
        sketch_plan_f64(m, n, ell, &sp64);
        need = static_cast<size_t>(sp64.kslabs) * static_cast<size_t>(n) * sp64.lp * sizeof(double);
    } else if (is_mixed_precision(precision)) {
        if (ell > ID_MAX_ELL || (ldo % 8) != 0 || (reinterpret_cast<uintptr_t>(omega) & 15u) != 0) return ID_ERR_ARG;
        if (!sketch_plan_lowp(m, n, ell, a_dtype == ID_F64, precision_nsplit(precision), &sp))
            return ID_ERR_UNSUPPORTED;
        need = sketch_partial_bytes_lowp(sp, n);
    } else {
        return ID_ERR_ARG;
    }
    if (need > static_cast<size_t>(ID_NOALLOC_SCRATCH_BYTES)) return ID_ERR_WORKSPACE;
    void* scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return ID_ERR_CUDA;
    cudaError_t e = cudaSuccess;
    if (info) e = cudaMemsetAsync(info, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return ID_ERR_CUDA;
    if (precision == ID_PLAIN_F64) {
        e = launch_sketch_f64(static_cast<const double*>(A), m, n, lda, static_cast<const double*>(omega), ldo, ell,
                              sp64, static_cast<double*>(scratch), static_cast<double*>(Y), ldy, info, s);
    } else {
        e = launch_sketch_lowp(A, a_dtype == ID_F64, m, n, lda, static_cast<const uint16_t*>(omega), ldo, ell,
                               precision, sp, static_cast<float*>(scratch), static_cast<float*>(Y), ldy, info,
                               4000000000ull, s);
    }
    return e == cudaSuccess ? ID_OK : ID_ERR_CUDA;
}
