// State shared by the two cooperative-grid pivoted-QR kernels (cpqr.cu: columns streamed
// through the working copy in global memory; cpqr_resident.cu: columns resident in shared
// memory): the per-CTA candidate record, the grid-barrier control word, the parameters,
// and the final listing of the unselected columns.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace gid {

// One CTA's best remaining candidate for the next step.
struct Cand {
    double nu;      // best residual squared norm in the slice (-1 if none)
    double sumnu;   // sum of residual squared norms of unselected columns in the slice
    double total;   // initial sum of squares of the slice (first table only)
    double s2;      // exact squared norm of the best column below the next step's row
    double alpha;   // the best column's entry on the next step's row
    double sv;      // streaming kernel, row mode: the best column's pending update coefficient
    int idx;        // column of the best norm (-1 if none)
    int stamp;      // resident kernel: step + 1 the record is for, stored last (release)
};

struct CpqrCtrl {
    uint32_t counter;
    int abort;
    uint32_t pad[62];
};

template <typename T>
struct CpqrParams {
    T* X;              // working copy r x n (ldx): streamed columns, or the resident kernel's input
    int64_t r, n, ldx;
    const void* src;   // initial values (nullptr: X already holds them)
    int src_f64;
    int64_t ldsrc;
    int kcap;
    double rel_tol;
    int32_t* J;
    int32_t* k_out;
    int32_t* info;
    double* R;
    int64_t ldr;
    uint8_t* sel;
    CpqrCtrl* ctrl;
    Cand* cand;        // [2][gridDim.x]
    T* pub;            // resident kernel: [2][gridDim.x][r] published candidate columns; streaming
                       // kernel, row mode: [2][r] each step's pivot column brought up to date
    int resident;
    int64_t cpb_max;   // columns per CTA at most (shared-memory layout)
    uint64_t limit_ns;
    int64_t out_j;     // grouped launch: J = J_base + out_j, k_out / info = their base + out_i
    int32_t out_i;
    int32_t colmode;   // streaming kernel: a warp per column (else the rows split over all threads);
                       // must equal the launch's mode
    int64_t rstage;    // streaming kernel, column mode: rows of the pivot column staged in shared memory (0: none)
};

// The FP64 fields of the records hold FP32 values exactly on the FP32 path; they come back
// by their bits (GB300's FP64 pipe would take a conversion per thread and step).  Values
// outside the normal float range go through the hardware conversion (exact as well).
__device__ __forceinline__ float narrow_exact(double x, float) {
    const uint32_t hi = static_cast<uint32_t>(__double2hiint(x));
    const uint32_t lo = static_cast<uint32_t>(__double2loint(x));
    const uint32_t e = (hi >> 20) & 0x7FFu;
    if (e >= 897u && e <= 1150u)
        return __uint_as_float((hi & 0x80000000u) | ((e - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
    if (((hi & 0x7FFFFFFFu) | lo) == 0u) return __uint_as_float(hi & 0x80000000u);
    return __double2float_rn(x);
}
__device__ __forceinline__ double narrow_exact(double x, double) { return x; }

// Pivot keys: the bits of a residual norm (non-negative; the sign bit of a -0 cleared) plus
// one compare as unsigned integers in the order of the values, on the integer pipe; 0 means
// "no candidate", and a NaN norm (a non-finite input, reported in info) is none.
__device__ __forceinline__ uint64_t norm_bits_key(float v) {
    const uint32_t a = __float_as_uint(v) & 0x7FFFFFFFu;
    return a > 0x7F800000u ? 0ull : static_cast<uint64_t>(a) + 1ull;
}
__device__ __forceinline__ uint64_t norm_bits_key(double v) {
    const uint64_t a = static_cast<uint64_t>(__double_as_longlong(v)) & 0x7FFFFFFFFFFFFFFFull;
    return a > 0x7FF0000000000000ull ? 0ull : a + 1ull;
}
__device__ __forceinline__ double key_norm_f64(uint64_t key, float) {
    return key ? f64_of_f32(__uint_as_float(static_cast<uint32_t>(key - 1ull))) : -1.0;
}
__device__ __forceinline__ double key_norm_f64(uint64_t key, double) {
    return key ? __longlong_as_double(static_cast<long long>(key - 1ull)) : -1.0;
}
// x > 0 for a double, on the integer pipe (false for zeros, negatives and NaNs).
__device__ __forceinline__ bool positive_bits(double x) {
    const long long u = __double_as_longlong(x);
    return u > 0 && u <= 0x7FF0000000000000ll;
}

// Candidate entries written by other CTAs are read from L2 (never from a stale L1 line).
__device__ __forceinline__ Cand load_cand(const Cand* p) {
    Cand c;
    c.nu = __ldcg(&p->nu);
    c.sumnu = __ldcg(&p->sumnu);
    c.total = __ldcg(&p->total);
    c.s2 = __ldcg(&p->s2);
    c.alpha = __ldcg(&p->alpha);
    c.sv = __ldcg(&p->sv);
    c.idx = __ldcg(&p->idx);
    c.stamp = 0;
    return c;
}

// CTA 0 after the last step: the rank and the complement J[k:n] in ascending column order
// (a block-wide exclusive scan of the unselected flags).  cnt: shared scratch of one int
// per warp.
__device__ __forceinline__ void list_complement(int32_t* J, const uint8_t* sel, int64_t n, int k, int32_t* k_out,
                                                int* cnt) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5, nt = blockDim.x;
    if (tid == 0) *k_out = k;
    int base = k;
    for (int64_t i0 = 0; i0 < n; i0 += nt) {
        const int64_t i = i0 + tid;
        const int flag = (i < n && !__ldcg(sel + i)) ? 1 : 0;
        const unsigned bal = __ballot_sync(0xffffffffu, flag);
        const int wpre = __popc(bal & ((1u << lane) - 1u));
        __syncthreads();
        if (lane == 0) cnt[warp] = __popc(bal);
        __syncthreads();
        int off = 0, tot = 0;
        for (int w = 0; w < nw; ++w) {
            if (w < warp) off += cnt[w];
            tot += cnt[w];
        }
        if (flag) J[base + off + wpre] = static_cast<int32_t>(i);
        base += tot;
    }
}

// Shared-memory bytes of the resident kernel for a CTA of at most cpb columns of r rows:
// norms, selection flags, the columns, and a copy of the step's pivot column.
template <typename T>
__host__ __device__ inline size_t resident_smem_bytes(int64_t cpb, int64_t r) {
    return static_cast<size_t>(cpb) * sizeof(T) + ((static_cast<size_t>(cpb) + 15) & ~size_t(15)) +
           static_cast<size_t>(cpb + 1) * r * sizeof(T);
}

template <typename T>
cudaError_t launch_cpqr_resident(const CpqrParams<T>& P, int grid, size_t smem, cudaStream_t s);

// Grouped streaming pivoted QR: ngroups matrices, gsize CTAs each, in one cooperative
// launch; groups (device) holds one parameter block per matrix, each with its own control
// word and candidate table [2][gsize], zeroed before the launch.  The outputs of group g
// are J_base + out_j, k_out_base[out_i] and info_base[out_i].  smem from
// cpqr_grouped_smem(the largest columns per CTA of any group).  colmode: the mode every
// group's parameters name (a group whose parameters differ reports -3 in its info).
template <typename T>
cudaError_t launch_cpqr_grouped(const CpqrParams<T>* groups, int ngroups, int gsize, int colmode, size_t smem,
                                int32_t* J_base, int32_t* k_out_base, int32_t* info_base, cudaStream_t s);
size_t cpqr_grouped_smem(int64_t cpb, int64_t rstage, int f64);
// The streaming kernel's mode for a slice of at most cpb columns of r rows: a warp per
// column, and the rows of the pivot column it stages in shared memory (0: none).
int cpqr_grouped_colmode(int64_t cpb);
int64_t cpqr_grouped_rstage(int64_t cpb, int64_t r, int elem_bytes);
constexpr int kCpqrGroupedThreads = 512;

}  // namespace gid
