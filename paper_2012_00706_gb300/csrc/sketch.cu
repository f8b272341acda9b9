// Sketch Y = Omega A on GB300.
//
// Mixed precision (Algorithm 2 cast + the sketching the paper names as
// future work in Sec. 5): every 64-row block of every column of A is scaled by
// a power of two chosen from the block's largest magnitude, taken at FP32
// precision, split into 1-3 bfloat16/half pieces, and multiplied by the
// low-precision Gaussian Omega on the 5th-generation tensor cores
// (tcgen05.mma kind::f16, FP32 accumulation in tensor memory).  The kernel is
// bound by the single HBM pass over A: one CTA per SM streams a 128-column
// tile of A through shared memory with 1-D bulk copies, converter warps build
// the swizzled K-major operand, one thread issues the MMAs, and epilogue warps
// drain each chunk's accumulator, apply the block's 2^s and keep the running
// sum in tensor memory.  Split-K partial sums are reduced by a second kernel.
//
// Plain FP64 twin: the same product with FP64 Omega by DFMA, register tiled.
#include "common.cuh"
#include "internal.h"

#include <algorithm>
#include <cstring>
#include <cudaTypedefs.h>

namespace gid {

// ---------------------------------------------------------------- cast helpers

// Shift of a scaling block from the largest magnitude's biased exponent
// (bits of |x|): bfloat16 puts the maximum in [0.5, 1), half in [2^13, 2^14).
// A zero or subnormal maximum gives shift 0.
__device__ __forceinline__ int shift_from_max_f64hi(uint32_t max_abs_hi, int f16) {
    const int e = static_cast<int>(max_abs_hi >> 20);
    if (e == 0) return 0;
    const int e2 = e - 1022;
    return f16 ? e2 - 14 : e2;
}

__device__ __forceinline__ int shift_from_max_f32(uint32_t max_abs, int f16) {
    const int e = static_cast<int>(max_abs >> 23);
    if (e == 0) return 0;
    const int e2 = e - 126;
    return f16 ? e2 - 14 : e2;
}

// x * 2^-s rounded once to float, through FP64 (rare path: results outside the
// float normal range, zero/subnormal doubles).  Both factors are normal
// doubles, so each FP64 product is exact while the result stays normal.
__device__ __noinline__ float scaled_slow(double x, int s) {
    const int a = -s / 2, b = -s - a;
    const double fa = __hiloint2double((1023 + a) << 20, 0);
    const double fb = __hiloint2double((1023 + b) << 20, 0);
    return __double2float_rn(__dmul_rn(__dmul_rn(x, fa), fb));
}

// fl32(x 2^-s) for double x using integer operations only: the exponent is
// rebiased and the 52-bit significand rounded to 23 bits, ties to even.
__device__ __forceinline__ float scaled_f32_from_f64(double x, int s) {
    const uint32_t hi = static_cast<uint32_t>(__double2hiint(x));
    const uint32_t lo = static_cast<uint32_t>(__double2loint(x));
    const uint32_t sign = hi & 0x80000000u, ah = hi & 0x7fffffffu;
    const int e = static_cast<int>(ah >> 20);
    const int e32 = e - s - 896;
    if (e != 0 && e32 >= 1 && e32 <= 253) {
        uint32_t t = (static_cast<uint32_t>(e32) << 23) | ((ah & 0xFFFFFu) << 3) | (lo >> 29);
        const uint32_t rb = (lo >> 28) & 1u;
        const uint32_t st = (lo & 0x0FFFFFFFu) != 0u ? 1u : 0u;
        t += rb & (st | (t & 1u));
        return __uint_as_float(sign | t);
    }
    if ((ah | lo) == 0u) return __uint_as_float(sign);
    return scaled_slow(x, s);
}

// Per-block constants of the converter's FP64 fast path for a block shift s:
// kb3 rebiases the exponent from 1023 to 127 and applies 2^-s (added to the high
// word before it is shifted left by 3, hence the division by 8; the sum is exact
// modulo 2^32 whenever the result is a normal float), thr is the smallest
// (hi << 1) whose scaled value is a normal float, less 2^21 (so that one unsigned
// compare of (hi << 1) - 2^21 against it also passes the zero-exponent elements),
// and a block with s < -872 is redone exactly (its zero-exponent elements could
// scale to nonzero floats).
struct F64CastBlock {
    uint32_t kb3, thr;
    bool slow;
};

__device__ __forceinline__ F64CastBlock f64_cast_block(int s) {
    F64CastBlock b;
    b.kb3 = (0x40000000u - (static_cast<uint32_t>(s) << 23)) >> 3;
    b.thr = static_cast<uint32_t>(max(1, 897 + s) - 1) << 21;
    b.slow = s < -872;
    return b;
}

// Branch-free fast path of scaled_f32_from_f64 for the sketch's converter, for an
// element at or below its block's largest magnitude.  The round-to-nearest-even
// increment is the carry out of lo + 0x0FFFFFFF + lsb (lsb = bit 29 of lo, the last
// kept bit), which the same add chain carries into the rebiased high word; a funnel
// shift then takes the exponent's low 9 bits and 23 significand bits.  An element
// with a zero exponent (zero or subnormal double) maps to a signed zero; `slow` is
// set when the scaled value of a nonzero-exponent element is below the normal range.
// ha = hi << 1.
__device__ __forceinline__ float scaled_f32_from_f64_fast(double x, uint32_t ha, const F64CastBlock& b,
                                                          bool& slow) {
    const uint32_t hi = static_cast<uint32_t>(__double2hiint(x));
    const uint32_t lo = static_cast<uint32_t>(__double2loint(x));
    const uint32_t t = ((lo >> 29) & 1u) + 0x0FFFFFFFu;
    uint32_t lo2, hi2;
    asm("add.cc.u32 %0, %2, %3;\n\taddc.u32 %1, %4, %5;" : "=r"(lo2), "=r"(hi2) : "r"(lo), "r"(t), "r"(hi), "r"(b.kb3));
    const uint32_t u = __funnelshift_l(lo2, hi2, 3);
    const bool zero = ha < 0x00200000u;
    slow |= ha - 0x00200000u < b.thr;
    return __uint_as_float((zero ? 0u : u) | (hi & 0x80000000u));
}

// fl32(x 2^-s) for float x: exponent adjust when both ends are normal.
__device__ __forceinline__ float scaled_f32_from_f32(float x, int s) {
    const uint32_t u = __float_as_uint(x);
    const int e = static_cast<int>((u >> 23) & 0xFFu);
    const int e2 = e - s;
    if (e >= 1 && e <= 254 && e2 >= 1 && e2 <= 254)
        return __uint_as_float(u - (static_cast<uint32_t>(s) << 23));
    if ((u & 0x7fffffffu) == 0u) return x;
    return scaled_slow(static_cast<double>(x), s);
}

// Branch-free fast path for float input: exponent adjust of a normal float.
__device__ __forceinline__ float scaled_f32_from_f32_fast(float x, int s, bool& slow) {
    const uint32_t u = __float_as_uint(x);
    const uint32_t e = (u >> 23) & 0xFFu;
    const bool zero = (u << 1) == 0u;
    slow |= !zero && ((e - 1u) > 253u || (static_cast<uint32_t>(static_cast<int>(e) - s - 1) > 253u));
    return zero ? x : __uint_as_float(u - (static_cast<uint32_t>(s) << 23));
}

// Two low-format pieces at once (packed round-to-nearest-even conversion) and
// the exact remainders; the first value goes to the low 16 bits.
__device__ __forceinline__ uint32_t take_piece2(float& a, float& b, int f16) {
    if (f16) {
        const __half2 h = __floats2half2_rn(a, b);
        const float2 f = __half22float2(h);
        a = a - f.x;
        b = b - f.y;
        return *reinterpret_cast<const uint32_t*>(&h);
    }
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const uint32_t w = *reinterpret_cast<const uint32_t*>(&h);
    a = a - __uint_as_float(w << 16);
    b = b - __uint_as_float(w & 0xFFFF0000u);
    return w;
}

int precision_nsplit(int precision) {
    switch (precision) {
        case ID_MIXED_BF16: return 1;
        case ID_MIXED_F16: return 1;
        case ID_MIXED_BF16X2: return 2;
        case ID_MIXED_BF16X3: return 3;
        default: return 0;
    }
}

int precision_is_f16(int precision) { return precision == ID_MIXED_F16 ? 1 : 0; }

// ------------------------------------------------------ tensor-core sketch

// Warp roles: 0 producer (TMA), 1 MMA issuer, 2 TMEM allocator, 3 idle,
// 4..19 converters (four threads per column), 20..23 epilogue.
constexpr int kConvWarps = 16;
// Elements of a converter thread's 16 (rows 16q .. 16q + 3 of the chunk) cast on the FP64
// pipe, the rest in integer arithmetic: four balances the two pipes on GB300 (measured
// against two to eight).
constexpr int kF2F = 4;
constexpr int kFirstConvWarp = 4;
constexpr int kFirstEpiWarp = kFirstConvWarp + kConvWarps;
constexpr int kSketchThreads = (kFirstEpiWarp + 4) * 32;
constexpr uint32_t kAopTileBytes = kTileCols * 128;   // 128 rows x 64 bf16 (16 KB)
constexpr uint32_t kSlabBytes = kTileCols * 128;      // one A box: 128 columns x 128 bytes
// L2 prefetch: every kPrefetchGroup chunks, the next kPrefetchGroup chunks starting
// kPrefetchAhead chunks ahead are prefetched with one tensor prefetch (2 KB per column).
constexpr int kPrefetchGroup = 4;
constexpr int kPrefetchAhead = 8;
#ifndef GID_SKETCH_L2_PREFETCH
#define GID_SKETCH_L2_PREFETCH 0
#endif
constexpr int kSketchL2Prefetch = GID_SKETCH_L2_PREFETCH;

struct LowpParams {
    const void* A;
    int64_t lda, m, n;
    int a_f64, nsplit, f16, lp, lpa;
    int64_t nchunks, chunks_per_slab;
    int stages, aop_bufs, omega_bufs, acc_bufs;
    uint32_t stage_bytes, omega_tile_bytes;
    int direct;          // A is not TMA-addressable: converters load it from global memory
    int aop_in_stage;    // the MMA operand is built inside the consumed A stage (no separate buffers)
    int prefetch;        // issue L2 tensor prefetches ahead of the loads
    float* partial;      // [kslabs][n][lp]
    int32_t* info;
    uint64_t limit_ns;
    // batch mode: CTA b computes unit b of the table; matrix i is read through maps[i]
    const SketchUnit* units;
    const BatchTask* tasks;
    const CUtensorMap* maps;
    int32_t* infos;
    int64_t ntasks, partial_total;
};

struct LowpSmem {
    uint8_t* aop;        // [aop_bufs][nsplit][16 KB]   swizzled K-major MMA operand (A columns)
    uint8_t* omega;      // [omega_bufs][omega tile]   swizzled K-major MMA operand (Omega rows)
    uint8_t* stage;      // [stages][stage_bytes]      A chunks as landed by TMA (128-byte swizzle)
    int32_t* shifts;     // [aop_bufs + acc_bufs][128]
    uint64_t* bars;
    uint32_t* tmem_holder;
    int* abort;
};

__host__ __device__ inline size_t lowp_carve(uintptr_t base, const LowpParams& P, LowpSmem* S) {
    uintptr_t p = base;
    auto take = [&](size_t bytes, size_t align) {
        p = (p + align - 1) & ~(uintptr_t)(align - 1);
        uintptr_t r = p;
        p += bytes;
        return r;
    };
    const int H = P.aop_bufs + P.acc_bufs;
    uintptr_t aop = take(P.aop_in_stage ? 0 : (size_t)P.aop_bufs * P.nsplit * kAopTileBytes, 1024);
    uintptr_t om = take((size_t)P.omega_bufs * P.omega_tile_bytes, 1024);
    uintptr_t st = take((size_t)P.stages * P.stage_bytes, 1024);
    uintptr_t sh = take((size_t)H * kTileCols * 4, 16);
    const int nbars = 2 * P.stages + 2 * P.omega_bufs + 2 * P.aop_bufs + 2 * P.acc_bufs + 2 * H;
    uintptr_t bars = take((size_t)nbars * 8, 8);
    uintptr_t th = take(4, 4);
    uintptr_t ab = take(4, 4);
    if (S) {
        S->aop = reinterpret_cast<uint8_t*>(aop);
        S->omega = reinterpret_cast<uint8_t*>(om);
        S->stage = reinterpret_cast<uint8_t*>(st);
        S->shifts = reinterpret_cast<int32_t*>(sh);
        S->bars = reinterpret_cast<uint64_t*>(bars);
        S->tmem_holder = reinterpret_cast<uint32_t*>(th);
        S->abort = reinterpret_cast<int*>(ab);
    }
    return static_cast<size_t>(p - base);
}

__device__ __forceinline__ void prefetch_tensor_2d(const CUtensorMap* map, int32_t c0, int32_t c1) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(c0), "r"(c1)
                 : "memory");
}

// Convert 8 scaled values into NSPLIT pieces and store them as one 16-byte chunk of
// row t (K group g) of each swizzled operand tile; the last piece needs no remainder.
template <int NSPLIT, bool F16>
__device__ __forceinline__ void store_pieces(uint8_t* aop_buf, int t, int g, float (&v)[8]) {
    const uint32_t off = (t >> 3) * 1024u + (t & 7) * 128u + ((g ^ (t & 7)) << 4);
#pragma unroll
    for (int p = 0; p < NSPLIT; ++p) {
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (p + 1 < NSPLIT) {
                w[q] = take_piece2(v[2 * q], v[2 * q + 1], F16 ? 1 : 0);
            } else if (F16) {
                const __half2 h = __floats2half2_rn(v[2 * q], v[2 * q + 1]);
                w[q] = *reinterpret_cast<const uint32_t*>(&h);
            } else {
                const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
                w[q] = *reinterpret_cast<const uint32_t*>(&h);
            }
        }
        *reinterpret_cast<uint4*>(aop_buf + (size_t)p * kAopTileBytes + off) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Slot and phase parity of a ring of n buffers, advanced once per chunk (the ring sizes
// are runtime values, so this replaces a division per use).
struct Ring {
    int slot = 0, n;
    uint32_t phase = 0;
    __device__ explicit Ring(int n_) : n(n_) {}
    __device__ void next() {
        if (++slot == n) {
            slot = 0;
            phase ^= 1u;
        }
    }
};

// After a watchdog abort: wait (bounded) until the last loads a producer issued into a ring
// of n buffers have landed, so that no bulk copy still writes into this CTA's shared memory
// when it leaves.  Load i went to slot i % n and completes phase (i / n) & 1 of its barrier;
// loads older than the last n were consumed before their slot was reused.
__device__ __forceinline__ void drain_issued(uint64_t* full, int n, int issued, uint64_t limit_ns) {
    volatile int keep_waiting = 0;
    for (int i = max(0, issued - n); i < issued; ++i)
        mbar_wait(&full[i % n], static_cast<uint32_t>((i / n) & 1), &keep_waiting, limit_ns);
}

// BATCH = false: one ID, CTA (x, y) computes 128-column tile x over row slab y of A.
// BATCH = true: CTA b computes unit b of the batch table (a tile and row slab of one
// matrix), reading that matrix through its own tensor map in global memory.
template <bool BATCH, bool F64, int NSPLIT, bool F16>
__global__ void __launch_bounds__(kSketchThreads, 1)
k_sketch_lowp(const __grid_constant__ CUtensorMap tm_omega, const __grid_constant__ CUtensorMap tm_a,
              const __grid_constant__ CUtensorMap tm_pf, const LowpParams P) {
    extern __shared__ uint8_t smem_raw[];
    const uintptr_t base = (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023);
    LowpSmem S;
    lowp_carve(base, P, &S);
    const int NS = P.stages, NO = P.omega_bufs, NA = P.aop_bufs, NC = P.acc_bufs, H = NA + NC;
    uint64_t* stage_full = S.bars;
    uint64_t* stage_free = stage_full + NS;
    uint64_t* omg_full = stage_free + NS;
    uint64_t* omg_free = omg_full + NO;
    uint64_t* aop_full = omg_free + NO;
    uint64_t* aop_free = aop_full + NA;
    uint64_t* acc_full = aop_free + NA;
    uint64_t* acc_empty = acc_full + NC;
    uint64_t* sh_full = acc_empty + NC;
    uint64_t* sh_free = sh_full + H;
    volatile int* abort = S.abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t col0, ch_begin, ch_end;
    int lp, ncols_valid;
    float* dst_tile;                  // partial sums of column col0 (column stride lp)
    int32_t* info;
    const CUtensorMap* amap;
    if constexpr (BATCH) {
        const SketchUnit su = P.units[blockIdx.x];
        // a unit that does not fit its matrix or the plan is reported, never executed
        if (su.task < 0 || su.task >= P.ntasks) return;
        const BatchTask& bt = P.tasks[su.task];
        const int64_t nch = (bt.m + kChunkRows - 1) / kChunkRows;
        if (su.tile < 0 || static_cast<int64_t>(su.tile) * kTileCols >= bt.n || su.c0 < 0 || su.nloc < 1 ||
            su.c0 + su.nloc > nch || su.slab < 0 || su.slab >= bt.kslabs || bt.lp < 16 || bt.lp > P.lp ||
            (bt.lp & 15) != 0 || bt.partial_off < 0 ||
            bt.partial_off + static_cast<int64_t>(bt.kslabs) * bt.n * bt.lp > P.partial_total) {
            if (threadIdx.x == 0) set_info(P.infos + su.task, kInfoBadTable);
            return;
        }
        col0 = static_cast<int64_t>(su.tile) * kTileCols;
        ch_begin = su.c0;
        ch_end = static_cast<int64_t>(su.c0) + su.nloc;
        lp = bt.lp;
        ncols_valid = static_cast<int>(min(static_cast<int64_t>(kTileCols), bt.n - col0));
        dst_tile = P.partial + bt.partial_off + (static_cast<int64_t>(su.slab) * bt.n + col0) * bt.lp;
        info = P.infos + su.task;
        amap = P.maps + su.task;
    } else {
        col0 = static_cast<int64_t>(blockIdx.x) * kTileCols;
        ch_begin = static_cast<int64_t>(blockIdx.y) * P.chunks_per_slab;
        ch_end = min(P.nchunks, ch_begin + P.chunks_per_slab);
        lp = P.lp;
        ncols_valid = static_cast<int>(min(static_cast<int64_t>(kTileCols), P.n - col0));
        dst_tile = P.partial + (static_cast<int64_t>(blockIdx.y) * P.n + col0) * P.lp;
        info = P.info;
        amap = &tm_a;
    }
    const int nloc = static_cast<int>(ch_end - ch_begin);
    constexpr int elem = F64 ? 8 : 4;
    const int slab_rows = 128 / elem;                     // rows per 128-byte box line
    const int nslabs = kChunkRows / slab_rows;            // boxes per chunk

    if (threadIdx.x == 0) {
        for (int i = 0; i < NS; ++i) {
            mbar_init(&stage_full[i], 1);
            mbar_init(&stage_free[i], P.aop_in_stage ? 1 : kConvWarps);
        }
        for (int i = 0; i < NO; ++i) { mbar_init(&omg_full[i], 1); mbar_init(&omg_free[i], 1); }
        for (int i = 0; i < NA; ++i) { mbar_init(&aop_full[i], kConvWarps); mbar_init(&aop_free[i], 1); }
        for (int i = 0; i < NC; ++i) { mbar_init(&acc_full[i], 1); mbar_init(&acc_empty[i], 4); }
        for (int i = 0; i < H; ++i) { mbar_init(&sh_full[i], kConvWarps); mbar_init(&sh_free[i], 4); }
        *S.abort = 0;
        fence_barrier_init();
    }
    if (warp == 2) {
        tmem_alloc(S.tmem_holder, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *S.tmem_holder;

    if (warp == 0) {
        // ---------------- A producer: the A boxes of each chunk (one thread issues TMA)
        if (lane == 0) {
            if constexpr (BATCH) {
                // the map was written to global memory before the launch; order the
                // tensor-map proxy's view of it after that write
                asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                                 reinterpret_cast<uint64_t>(amap))
                             : "memory");
            }
            if (!P.direct) prefetch_tensormap(amap);
            if (P.prefetch && !P.direct) {
                prefetch_tensormap(&tm_pf);
                for (int g = 0; g < kPrefetchAhead; g += kPrefetchGroup)
                    if (ch_begin + g < ch_end)
                        prefetch_tensor_2d(&tm_pf, static_cast<int32_t>((ch_begin + g) * kChunkRows),
                                           static_cast<int32_t>(col0));
            }
            Ring rs(NS);
            int issued = 0;
            for (int i = 0; i < nloc; ++i, rs.next()) {
                const int64_t c = ch_begin + i;
                const int s = rs.slot;
                if (P.prefetch && !P.direct && (i % kPrefetchGroup) == 0 && c + kPrefetchAhead < ch_end)
                    prefetch_tensor_2d(&tm_pf, static_cast<int32_t>((c + kPrefetchAhead) * kChunkRows),
                                       static_cast<int32_t>(col0));
                if (!mbar_wait(&stage_free[s], rs.phase ^ 1u, abort, P.limit_ns)) break;
                if (P.direct) {
                    mbar_arrive(&stage_full[s]);
                } else {
                    mbar_arrive_expect_tx(&stage_full[s], P.stage_bytes);
                    uint8_t* dst = S.stage + (size_t)s * P.stage_bytes;
                    for (int sl = 0; sl < nslabs; ++sl)
                        tma_load_2d(dst + (size_t)sl * kSlabBytes, amap,
                                    static_cast<int32_t>(c * kChunkRows + sl * slab_rows),
                                    static_cast<int32_t>(col0), &stage_full[s]);
                    issued = i + 1;
                }
            }
            if (*abort) drain_issued(stage_full, NS, issued, P.limit_ns);
        }
    } else if (warp == 3) {
        // ---------------- Omega producer: one swizzled Omega tile per chunk
        if (lane == 0) {
            prefetch_tensormap(&tm_omega);
            Ring ro(NO);
            int issued = 0;
            for (int i = 0; i < nloc; ++i, ro.next()) {
                const int64_t c = ch_begin + i;
                const int o = ro.slot;
                if (!mbar_wait(&omg_free[o], ro.phase ^ 1u, abort, P.limit_ns)) break;
                mbar_arrive_expect_tx(&omg_full[o], P.omega_tile_bytes);
                tma_load_2d(S.omega + (size_t)o * P.omega_tile_bytes, &tm_omega,
                            static_cast<int32_t>(c * kChunkRows), 0, &omg_full[o]);
                issued = i + 1;
            }
            if (*abort) drain_issued(omg_full, NO, issued, P.limit_ns);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (one thread)
        if (lane == 0) {
            const uint32_t idesc = umma_idesc_f16(F16 ? 0u : 1u, 128u, static_cast<uint32_t>(lp));
            int issued = 0;
            Ring ra(NA), ro(NO), rb(NC);
            for (int i = 0; i < nloc; ++i, ra.next(), ro.next(), rb.next()) {
                const int a = ra.slot, o = ro.slot, b = rb.slot;
                if (!mbar_wait(&aop_full[a], ra.phase, abort, P.limit_ns)) break;
                if (!mbar_wait(&omg_full[o], ro.phase, abort, P.limit_ns)) break;
                if (!mbar_wait(&acc_empty[b], rb.phase ^ 1u, abort, P.limit_ns)) break;
                tc_fence_after();
                const uint32_t d = tmem + static_cast<uint32_t>(b * P.lpa);
                const uint32_t bbase = smem_addr(S.omega + (size_t)o * P.omega_tile_bytes);
                uint8_t* aop_base = P.aop_in_stage ? S.stage + (size_t)a * P.stage_bytes
                                                   : S.aop + (size_t)a * NSPLIT * kAopTileBytes;
#pragma unroll
                for (int p = 0; p < NSPLIT; ++p) {
                    const uint32_t abase = smem_addr(aop_base + (size_t)p * kAopTileBytes);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        umma_f16(d, umma_desc_sw128(abase + 32u * kk), umma_desc_sw128(bbase + 32u * kk), idesc,
                                 (p | kk) != 0 ? 1u : 0u);
                }
                umma_commit(P.aop_in_stage ? &stage_free[a] : &aop_free[a]);
                umma_commit(&omg_free[o]);
                umma_commit(&acc_full[b]);
                issued = i + 1;
            }
            if (*abort && issued > 0) {
                // leave only after the MMAs already issued are done (bounded wait)
                volatile int keep_waiting = 0;
                const int b = (issued - 1) % NC;
                mbar_wait(&acc_full[b], ((issued - 1) / NC) & 1, &keep_waiting, P.limit_ns);
            }
        }
    } else if (warp >= kFirstConvWarp && warp < kFirstEpiWarp) {
        // ---------------- converters: lane = column (8 per warp) + 8 * quarter (16 rows each)
        const int cw = warp - kFirstConvWarp;
        const int q = lane >> 3;
        const int t = cw * 8 + (lane & 7);
        const int64_t col = col0 + t;
        const bool valid = t < ncols_valid;
        Ring rs(NS), ra(NA), rh(H);
        for (int i = 0; i < nloc; ++i, rs.next(), ra.next(), rh.next()) {
            const int64_t c = ch_begin + i;
            const int s = rs.slot, a = P.aop_in_stage ? s : ra.slot, h = rh.slot;
            if (!mbar_wait(&stage_full[s], rs.phase, abort, P.limit_ns)) break;
            if (!P.aop_in_stage && !mbar_wait(&aop_free[a], ra.phase ^ 1u, abort, P.limit_ns)) break;
            if (!mbar_wait(&sh_free[h], rh.phase ^ 1u, abort, P.limit_ns)) break;
            const int64_t row0 = c * kChunkRows;
            const int rows = static_cast<int>(min(static_cast<int64_t>(kChunkRows), P.m - row0));
            const uint8_t* stg = S.stage + (size_t)s * P.stage_bytes;
            uint8_t* aop_buf = P.aop_in_stage ? S.stage + (size_t)s * P.stage_bytes
                                              : S.aop + (size_t)a * NSPLIT * kAopTileBytes;
            uint32_t mx = 0;
            int shift;
            float f[16];
            bool slow = false;
            if constexpr (F64) {
                double v[16];
                if (!P.direct) {
                    // box q holds rows 16q..16q+15 of all 128 columns, 128 bytes per column, swizzled
                    const uint8_t* line = stg + (size_t)q * kSlabBytes + (size_t)t * 128;
#pragma unroll
                    for (int cc = 0; cc < 8; ++cc) {
                        const double2 d2 = *reinterpret_cast<const double2*>(line + ((cc ^ (t & 7)) << 4));
                        v[2 * cc] = d2.x;
                        v[2 * cc + 1] = d2.y;
                    }
                } else {
                    const double* g = static_cast<const double*>(P.A) + col * P.lda + row0;
#pragma unroll
                    for (int r = 0; r < 16; ++r) v[r] = (valid && 16 * q + r < rows) ? __ldg(g + 16 * q + r) : 0.0;
                }
                // in-place pieces: piece p of column t lands on line t of box p of the stage,
                // which only the four threads of column t (one warp) read, so the warp's reads
                // must be done before its writes, and no other warp's
                if (P.aop_in_stage) __syncwarp();
                // high words without the sign (hi << 1), their maximum three at a time
                uint32_t ha[16];
#pragma unroll
                for (int r = 0; r < 16; ++r) ha[r] = static_cast<uint32_t>(__double2hiint(v[r])) << 1;
#pragma unroll
                for (int r = 0; r < 16; r += 2) mx = __vimax3_u32(mx, ha[r], ha[r + 1]);
                mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 8));
                mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 16));
                mx >>= 1;
                if (q == 0 && (mx >> 20) == 0x7FFu) set_info(info, kInfoNonFinite);
                shift = shift_from_max_f64hi(mx, F16 ? 1 : 0);
                const F64CastBlock cb = f64_cast_block(shift);
                slow = cb.slow;
                // the first kF2F elements through the FP64 pipe's conversion (idle otherwise) and
                // an exact FP32 power-of-two scale: fl32(x) 2^-s = fl32(x 2^-s) while both are
                // normal floats, i.e. for a nonzero exponent e >= max(897, 897 + s) (one compare
                // like the integer path's); zero exponents give signed zeros both ways, a shift
                // outside [-126, 127] sends the block to the exact routine below
                if (kF2F > 0) slow |= shift < -126 || shift > 127;
                const float sc = __uint_as_float(static_cast<uint32_t>(127 - shift) << 23);
                const uint32_t thr_f2f = max(cb.thr, 896u << 21);
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    if (r < kF2F) {
                        f[r] = __double2float_rn(v[r]) * sc;
                        slow |= ha[r] - 0x00200000u < thr_f2f;
                    } else {
                        f[r] = scaled_f32_from_f64_fast(v[r], ha[r], cb, slow);
                    }
                }
                if (__any_sync(0xffffffffu, slow) && slow) {
#pragma unroll
                    for (int r = 0; r < 16; ++r) f[r] = scaled_f32_from_f64(v[r], shift);
                }
            } else {
                float v[16];
                if (!P.direct) {
                    // box q/2 holds rows 32(q/2)..+31; this thread's 16 rows are 16-byte chunks 4(q&1)..+3
                    const uint8_t* line = stg + (size_t)(q >> 1) * kSlabBytes + (size_t)t * 128;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int cc = 4 * (q & 1) + k;
                        const float4 f4 = *reinterpret_cast<const float4*>(line + ((cc ^ (t & 7)) << 4));
                        v[4 * k] = f4.x; v[4 * k + 1] = f4.y; v[4 * k + 2] = f4.z; v[4 * k + 3] = f4.w;
                    }
                } else {
                    const float* g = static_cast<const float*>(P.A) + col * P.lda + row0;
#pragma unroll
                    for (int r = 0; r < 16; ++r) v[r] = (valid && 16 * q + r < rows) ? __ldg(g + 16 * q + r) : 0.f;
                }
                if (P.aop_in_stage) __syncwarp();     // as above: rows 0-31 are box 0, rows 32-63 box 1
#pragma unroll
                for (int r = 0; r < 16; ++r) mx = max(mx, __float_as_uint(v[r]) & 0x7fffffffu);
                mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 8));
                mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 16));
                if (q == 0 && (mx >> 23) == 0xFFu) set_info(info, kInfoNonFinite);
                shift = shift_from_max_f32(mx, F16 ? 1 : 0);
#pragma unroll
                for (int r = 0; r < 16; ++r) f[r] = scaled_f32_from_f32_fast(v[r], shift, slow);
                if (__any_sync(0xffffffffu, slow) && slow) {
#pragma unroll
                    for (int r = 0; r < 16; ++r) f[r] = scaled_f32_from_f32(v[r], shift);
                }
            }
#pragma unroll
            for (int gg = 0; gg < 2; ++gg) {
                float f8[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) f8[k] = f[8 * gg + k];
                store_pieces<NSPLIT, F16>(aop_buf, t, 2 * q + gg, f8);
            }
            if (q == 0) S.shifts[h * kTileCols + t] = shift;
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                if (!P.aop_in_stage) mbar_arrive(&stage_free[s]);
                mbar_arrive(&aop_full[a]);
                mbar_arrive(&sh_full[h]);
            }
        }
    } else if (warp >= kFirstEpiWarp) {
        // ---------------- epilogue: drain each chunk, scale by 2^s, accumulate in TMEM
        const int q = warp & 3;
        const int t = 32 * q + lane;
        const uint32_t lane_base = tmem + (static_cast<uint32_t>(32 * q) << 16);
        const uint32_t run_col = static_cast<uint32_t>(NC * P.lpa);
        const int nsl = lp / 16;
        bool ok = true;
        Ring rb(NC), rh(H);
        for (int i = 0; i < nloc; ++i, rb.next(), rh.next()) {
            const int b = rb.slot, h = rh.slot;
            if (!mbar_wait(&acc_full[b], rb.phase, abort, P.limit_ns)) { ok = false; break; }
            if (!mbar_wait(&sh_full[h], rh.phase, abort, P.limit_ns)) { ok = false; break; }
            tc_fence_after();
            const float sc = ldexpf(1.0f, S.shifts[h * kTileCols + t]);
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh_free[h]);
            // two 16-column slices per round trip: the tensor-memory load latency, not the
            // arithmetic, sets the pace here
            const uint32_t acc_col = static_cast<uint32_t>(b * P.lpa);
            for (int sl = 0; sl < nsl; sl += 2) {
                const bool two = sl + 1 < nsl;
                float acc0[16], acc1[16], run0[16], run1[16];
                tmem_ld16(lane_base + acc_col + 16u * sl, acc0);
                if (two) tmem_ld16(lane_base + acc_col + 16u * (sl + 1), acc1);
                if (i > 0) {
                    tmem_ld16(lane_base + run_col + 16u * sl, run0);
                    if (two) tmem_ld16(lane_base + run_col + 16u * (sl + 1), run1);
                }
                tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 16; ++j) run0[j] = (i > 0) ? fmaf(acc0[j], sc, run0[j]) : acc0[j] * sc;
                tmem_st16(lane_base + run_col + 16u * sl, run0);
                if (two) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) run1[j] = (i > 0) ? fmaf(acc1[j], sc, run1[j]) : acc1[j] * sc;
                    tmem_st16(lane_base + run_col + 16u * (sl + 1), run1);
                }
            }
            tmem_st_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
        }
        if (ok && nloc > 0) {
            // all lanes take part in the warp-wide loads; lanes past n do not store
            float* dst = dst_tile + static_cast<int64_t>(t) * lp;
            for (int sl = 0; sl < nsl; ++sl) {
                float run[16];
                tmem_ld16(lane_base + run_col + 16u * sl, run);
                tmem_ld_wait();
                if (t < ncols_valid) {
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        *reinterpret_cast<float4*>(dst + 16 * sl + j) =
                            make_float4(run[j], run[j + 1], run[j + 2], run[j + 3]);
                }
            }
        }
    }
    if (*abort) set_info(info, kInfoWatchdog);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 2) tmem_dealloc(tmem, 512);
}

// Y(l, j) = sum over split-K slabs of the partial sums [kslabs][n][lp] (fixed slab
// order).  Warp w of a block reduces column j = 4 blockIdx.x + w: lane i sums rows
// i, i + 32, i + 64, i + 96 of each group of 128, with the loads of eight slabs for
// all four rows issued before their sums (the partial sums are in L2; the time is
// load latency); info flags a non-finite sum (an FP32 sketch that overflowed).
constexpr int kReduceCols = 4;
constexpr int kReduceRows = 4;
constexpr int kReduceSlabs = 8;

template <typename T>
__global__ void __launch_bounds__(kReduceCols * 32)
k_reduce_partials(const T* __restrict__ partial, int kslabs, int64_t n, int lp, int ell, T* __restrict__ Y,
                  int64_t ldy, int32_t* info) {
    const int64_t j = static_cast<int64_t>(blockIdx.x) * kReduceCols + (threadIdx.x >> 5);
    if (j >= n) return;
    const int lane = threadIdx.x & 31;
    const int64_t slab = n * lp;
    const T* src = partial + j * lp;
    for (int l0 = 0; l0 < ell; l0 += 32 * kReduceRows) {
        T s[kReduceRows];
#pragma unroll
        for (int r = 0; r < kReduceRows; ++r) s[r] = T(0);
        for (int k0 = 0; k0 < kslabs; k0 += kReduceSlabs) {
            T v[kReduceSlabs][kReduceRows];
#pragma unroll
            for (int kk = 0; kk < kReduceSlabs; ++kk)
#pragma unroll
                for (int r = 0; r < kReduceRows; ++r) {
                    const int l = l0 + 32 * r + lane;
                    v[kk][r] = (k0 + kk < kslabs && l < ell) ? src[(k0 + kk) * slab + l] : T(0);
                }
#pragma unroll
            for (int kk = 0; kk < kReduceSlabs; ++kk)
#pragma unroll
                for (int r = 0; r < kReduceRows; ++r)
                    if (k0 + kk < kslabs) s[r] += v[kk][r];
        }
#pragma unroll
        for (int r = 0; r < kReduceRows; ++r) {
            const int l = l0 + 32 * r + lane;
            if (l < ell) {
                if (info && !isfinite(s[r])) set_info(info, kInfoNonFinite);
                Y[j * ldy + l] = s[r];
            }
        }
    }
}

// ------------------------------------------------------------- host plans

static PFN_cuTensorMapEncodeTiled_v12000 get_encode_tiled() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// The kernel instance for an input type and precision (pieces, format).
template <bool BATCH>
static void* sketch_kernel(int a_f64, int precision) {
    const int nsplit = precision_nsplit(precision), f16 = precision_is_f16(precision);
    if (a_f64) {
        if (f16) return reinterpret_cast<void*>(k_sketch_lowp<BATCH, true, 1, true>);
        switch (nsplit) {
            case 1: return reinterpret_cast<void*>(k_sketch_lowp<BATCH, true, 1, false>);
            case 2: return reinterpret_cast<void*>(k_sketch_lowp<BATCH, true, 2, false>);
            default: return reinterpret_cast<void*>(k_sketch_lowp<BATCH, true, 3, false>);
        }
    }
    if (f16) return reinterpret_cast<void*>(k_sketch_lowp<BATCH, false, 1, true>);
    switch (nsplit) {
        case 1: return reinterpret_cast<void*>(k_sketch_lowp<BATCH, false, 1, false>);
        case 2: return reinterpret_cast<void*>(k_sketch_lowp<BATCH, false, 2, false>);
        default: return reinterpret_cast<void*>(k_sketch_lowp<BATCH, false, 3, false>);
    }
}

static cudaError_t launch_sketch_kernel(void* kern, dim3 grid, size_t smem, cudaStream_t s, const CUtensorMap& tm_om,
                                        const CUtensorMap& tm_a, const CUtensorMap& tm_pf, const LowpParams& P) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    void* args[] = {const_cast<CUtensorMap*>(&tm_om), const_cast<CUtensorMap*>(&tm_a), const_cast<CUtensorMap*>(&tm_pf),
                    const_cast<LowpParams*>(&P)};
    return cudaLaunchKernel(kern, grid, dim3(kSketchThreads), args, smem, s);
}

bool sketch_pipeline_plan(int lp, int a_f64, int nsplit, SketchPlan* plan) {
    const DeviceInfo& dev = device_info();
    if (lp < 16 || lp > ID_MAX_ELL || (lp % 16) != 0 || nsplit < 1 || nsplit > 3) return false;
    SketchPlan p = *plan;
    p.lp = lp;
    const int lpa = (lp + 31) / 32 * 32;
    // chunk accumulators in flight between the MMAs and the epilogue, next to the running sum
    p.acc_bufs = (4 * lpa <= 512) ? 3 : (3 * lpa <= 512) ? 2 : 1;
    const uint32_t stage_bytes = static_cast<uint32_t>(kChunkRows * kTileCols * (a_f64 ? 8 : 4));
    const uint32_t omega_tile = (static_cast<uint32_t>(lp) * 128u + 1023u) & ~1023u;
    LowpParams P{};
    P.nsplit = nsplit;
    P.stage_bytes = stage_bytes;
    P.omega_tile_bytes = omega_tile;
    P.acc_bufs = p.acc_bufs;
    const size_t budget = static_cast<size_t>(dev.max_smem_optin) - 1024;
    auto fits = [&](int st, int na, int no) {
        P.stages = st; P.aop_bufs = na; P.omega_bufs = no;
        return lowp_carve(0, P, nullptr) <= budget;
    };
    // The MMA operand lives inside the consumed stage when the stage can hold its pieces,
    // which frees room for more stages in flight.  Prefer load depth (stages), then a
    // second Omega buffer, then (separate operands only) a second operand buffer.
    P.aop_in_stage = stage_bytes >= static_cast<uint32_t>(nsplit) * kAopTileBytes ? 1 : 0;
    int st = 2, na = 1, no = 1;
    if (P.aop_in_stage) na = 2;
    auto fits2 = [&](int st_, int no_) { return fits(st_, P.aop_in_stage ? st_ : na, no_); };
    if (!fits2(st, no)) return false;
    const int max_st = a_f64 ? 3 : 6;
    while (st < max_st && fits2(st + 1, no)) ++st;
    if (fits2(st, 2)) no = 2;
    if (P.aop_in_stage) na = st;
    else if (fits(st, 2, no)) na = 2;
    fits(st, na, no);
    p.stages = st; p.aop_bufs = na; p.omega_bufs = no; p.aop_in_stage = P.aop_in_stage;
    p.smem_bytes = lowp_carve(0, P, nullptr) + 1024;
    *plan = p;
    return true;
}

bool sketch_plan_lowp(int64_t m, int64_t n, int ell, int a_f64, int nsplit, SketchPlan* plan) {
    const DeviceInfo& dev = device_info();
    if (ell < 1) return false;
    SketchPlan p;
    p.tiles = static_cast<int>((n + kTileCols - 1) / kTileCols);
    p.nchunks = (m + kChunkRows - 1) / kChunkRows;
    int target = std::max(1, dev.sm_count);
    int64_t kslabs = std::max<int64_t>(1, std::min<int64_t>(p.nchunks, target / std::max(1, p.tiles)));
    p.chunks_per_slab = (p.nchunks + kslabs - 1) / kslabs;
    p.kslabs = static_cast<int>((p.nchunks + p.chunks_per_slab - 1) / p.chunks_per_slab);
    if (!sketch_pipeline_plan((ell + 15) / 16 * 16, a_f64, nsplit, &p)) return false;
    *plan = p;
    return true;
}

size_t sketch_partial_bytes_lowp(const SketchPlan& p, int64_t n) {
    return static_cast<size_t>(p.kslabs) * static_cast<size_t>(n) * p.lp * sizeof(float);
}

cudaError_t launch_sketch_lowp(const void* A, int a_f64, int64_t m, int64_t n, int64_t lda,
                               const uint16_t* omega, int64_t ldo, int ell, int precision,
                               const SketchPlan& plan, float* partial, float* Y, int64_t ldy,
                               int32_t* info, uint64_t limit_ns, cudaStream_t s, cudaEvent_t after_main) {
    auto encode = get_encode_tiled();
    if (!encode) return cudaErrorNotSupported;
    const int f16 = precision_is_f16(precision);
    const int elem = a_f64 ? 8 : 4;
    CUtensorMap tm_om, tm_a, tm_pf;
    memset(&tm_a, 0, sizeof(tm_a));
    memset(&tm_pf, 0, sizeof(tm_pf));
    {
        cuuint64_t gdim[2] = {static_cast<cuuint64_t>(m), static_cast<cuuint64_t>(ell)};
        cuuint64_t gstride[1] = {static_cast<cuuint64_t>(ldo) * 2};
        cuuint32_t box[2] = {static_cast<cuuint32_t>(kChunkRows), static_cast<cuuint32_t>(plan.lp)};
        cuuint32_t estr[2] = {1, 1};
        if (encode(&tm_om, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                   const_cast<uint16_t*>(omega), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    const int direct = ((reinterpret_cast<uintptr_t>(A) & 15u) != 0 || ((lda * elem) & 15) != 0) ? 1 : 0;
    bool prefetch = false;
    if (!direct) {
        const CUtensorMapDataType dt = a_f64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
        cuuint64_t gdim[2] = {static_cast<cuuint64_t>(m), static_cast<cuuint64_t>(n)};
        cuuint64_t gstride[1] = {static_cast<cuuint64_t>(lda) * elem};
        cuuint32_t estr[2] = {1, 1};
        cuuint32_t box[2] = {static_cast<cuuint32_t>(128 / elem), static_cast<cuuint32_t>(kTileCols)};
        if (encode(&tm_a, dt, 2, const_cast<void*>(A), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
        // prefetch boxes: kPrefetchGroup chunks of rows x 128 columns (2 KB-class runs per column)
        cuuint32_t pbox[2] = {static_cast<cuuint32_t>(std::min<int64_t>(256, kPrefetchGroup * kChunkRows)),
                              static_cast<cuuint32_t>(kTileCols)};
        prefetch = encode(&tm_pf, dt, 2, const_cast<void*>(A), gdim, gstride, pbox, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }

    LowpParams P{};
    P.A = A; P.lda = lda; P.m = m; P.n = n; P.a_f64 = a_f64;
    P.nsplit = precision_nsplit(precision); P.f16 = f16;
    P.lp = plan.lp; P.lpa = (plan.lp + 31) / 32 * 32;
    P.nchunks = plan.nchunks; P.chunks_per_slab = plan.chunks_per_slab;
    P.stages = plan.stages; P.aop_bufs = plan.aop_bufs; P.omega_bufs = plan.omega_bufs;
    P.acc_bufs = plan.acc_bufs;
    P.stage_bytes = static_cast<uint32_t>(kChunkRows * kTileCols * elem);
    P.omega_tile_bytes = (static_cast<uint32_t>(plan.lp) * 128u + 1023u) & ~1023u;
    P.direct = direct;
    P.aop_in_stage = plan.aop_in_stage;
    P.prefetch = prefetch ? kSketchL2Prefetch : 0;
    P.partial = partial; P.info = info; P.limit_ns = limit_ns;

    cudaError_t e = launch_sketch_kernel(sketch_kernel<false>(a_f64, precision), dim3(plan.tiles, plan.kslabs),
                                         plan.smem_bytes, s, tm_om, tm_a, tm_pf, P);
    if (e != cudaSuccess) return e;
    if (after_main) cudaEventRecord(after_main, s);
    if (!Y) return cudaSuccess;   // the consumer adds the partial sums itself
    k_reduce_partials<float><<<static_cast<unsigned>((n + kReduceCols - 1) / kReduceCols), kReduceCols * 32, 0, s>>>(
        partial, plan.kslabs, n, plan.lp, ell, Y, ldy, info);
    return cudaGetLastError();
}

bool encode_a_map(const void* A, int a_f64, int64_t m, int64_t n, int64_t lda, CUtensorMap* map) {
    auto encode = get_encode_tiled();
    if (!encode) return false;
    const int elem = a_f64 ? 8 : 4;
    if ((reinterpret_cast<uintptr_t>(A) & 15u) != 0 || ((lda * elem) & 15) != 0) return false;
    const CUtensorMapDataType dt = a_f64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    cuuint64_t gdim[2] = {static_cast<cuuint64_t>(m), static_cast<cuuint64_t>(n)};
    cuuint64_t gstride[1] = {static_cast<cuuint64_t>(lda) * elem};
    cuuint32_t estr[2] = {1, 1};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(128 / elem), static_cast<cuuint32_t>(kTileCols)};
    return encode(map, dt, 2, const_cast<void*>(A), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_sketch_lowp_batched(const SketchUnit* units, int64_t nunits, const BatchTask* tasks,
                                       const CUtensorMap* maps, int a_f64, const uint16_t* omega, int64_t ldo,
                                       int64_t m_rows, int ell_rows, int precision, const SketchPlan& plan,
                                       float* partial, int64_t partial_total, int64_t ntasks, int32_t* infos,
                                       uint64_t limit_ns, cudaStream_t s) {
    auto encode = get_encode_tiled();
    if (!encode) return cudaErrorNotSupported;
    const int f16 = precision_is_f16(precision);
    const int elem = a_f64 ? 8 : 4;
    CUtensorMap tm_om, tm_unused;
    memset(&tm_unused, 0, sizeof(tm_unused));
    cuuint64_t gdim[2] = {static_cast<cuuint64_t>(m_rows), static_cast<cuuint64_t>(ell_rows)};
    cuuint64_t gstride[1] = {static_cast<cuuint64_t>(ldo) * 2};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(kChunkRows), static_cast<cuuint32_t>(plan.lp)};
    cuuint32_t estr[2] = {1, 1};
    if (encode(&tm_om, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
               const_cast<uint16_t*>(omega), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    LowpParams P{};
    P.a_f64 = a_f64;
    P.nsplit = precision_nsplit(precision); P.f16 = f16;
    P.lp = plan.lp; P.lpa = (plan.lp + 31) / 32 * 32;
    P.stages = plan.stages; P.aop_bufs = plan.aop_bufs; P.omega_bufs = plan.omega_bufs;
    P.acc_bufs = plan.acc_bufs;
    P.stage_bytes = static_cast<uint32_t>(kChunkRows * kTileCols * elem);
    P.omega_tile_bytes = (static_cast<uint32_t>(plan.lp) * 128u + 1023u) & ~1023u;
    P.direct = 0;
    P.aop_in_stage = plan.aop_in_stage;
    P.prefetch = 0;
    P.partial = partial;
    P.limit_ns = limit_ns;
    P.units = units; P.tasks = tasks; P.maps = maps; P.infos = infos;
    P.ntasks = ntasks; P.partial_total = partial_total;
    if (nunits <= 0) return cudaSuccess;
    const cudaError_t e = launch_sketch_kernel(sketch_kernel<true>(a_f64, precision),
                                               dim3(static_cast<unsigned>(nunits)), plan.smem_bytes, s, tm_om,
                                               tm_unused, tm_unused, P);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// ------------------------------------------------------ plain FP64 sketch

constexpr int kF64Tile = 64;
constexpr int kF64K = 16;

// Y partial for rows [64 by, +64) of Omega and columns [64 bx, +64) of A over a
// K slab; 256 threads, 4 x 4 outputs each, FP64 FMAs.
__global__ void __launch_bounds__(256)
k_sketch_f64(const double* __restrict__ A, int64_t m, int64_t n, int64_t lda,
             const double* __restrict__ omega, int64_t ldo, int ell, int64_t k_per_slab, int lp,
             double* __restrict__ partial) {
    __shared__ double Os[kF64K][kF64Tile + 1];
    __shared__ double As[kF64K][kF64Tile + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t c0 = static_cast<int64_t>(blockIdx.x) * kF64Tile;
    const int r0 = blockIdx.y * kF64Tile;
    const int64_t kb = static_cast<int64_t>(blockIdx.z) * k_per_slab;
    const int64_t ke = min(m, kb + k_per_slab);
    double acc[4][4] = {};
    for (int64_t k0 = kb; k0 < ke; k0 += kF64K) {
        for (int idx = threadIdx.x; idx < kF64K * kF64Tile; idx += 256) {
            const int kk = idx % kF64K, i = idx / kF64K;
            const int64_t kg = k0 + kk;
            Os[kk][i] = (r0 + i < ell && kg < ke) ? omega[(r0 + i) * ldo + kg] : 0.0;
            As[kk][i] = (c0 + i < n && kg < ke) ? A[(c0 + i) * lda + kg] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kF64K; ++kk) {
            double o[4], a[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { o[q] = Os[kk][ty * 4 + q]; a[q] = As[kk][tx * 4 + q]; }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fma(o[p], a[q], acc[p][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t col = c0 + tx * 4 + q;
        if (col >= n) continue;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int row = r0 + ty * 4 + p;
            if (row < lp) partial[(static_cast<int64_t>(blockIdx.z) * n + col) * lp + row] = acc[p][q];
        }
    }
}

void sketch_plan_f64(int64_t m, int64_t n, int ell, SketchF64Plan* plan) {
    const DeviceInfo& dev = device_info();
    const int64_t tiles = ((n + kF64Tile - 1) / kF64Tile) * ((ell + kF64Tile - 1) / kF64Tile);
    const int64_t want = std::max<int64_t>(1, (2LL * dev.sm_count + tiles - 1) / tiles);
    int64_t kps = (m + want - 1) / want;
    kps = std::max<int64_t>(kF64K, (kps + kF64K - 1) / kF64K * kF64K);
    plan->k_per_slab = kps;
    plan->kslabs = static_cast<int>((m + kps - 1) / kps);
    plan->lp = ell;
}

cudaError_t launch_sketch_f64(const double* A, int64_t m, int64_t n, int64_t lda, const double* omega,
                              int64_t ldo, int ell, const SketchF64Plan& plan, double* partial,
                              double* Y, int64_t ldy, int32_t* info, cudaStream_t s, cudaEvent_t after_main) {
    dim3 grid(static_cast<unsigned>((n + kF64Tile - 1) / kF64Tile),
              static_cast<unsigned>((ell + kF64Tile - 1) / kF64Tile), static_cast<unsigned>(plan.kslabs));
    k_sketch_f64<<<grid, 256, 0, s>>>(A, m, n, lda, omega, ldo, ell, plan.k_per_slab, plan.lp, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (after_main) cudaEventRecord(after_main, s);
    k_reduce_partials<double><<<static_cast<unsigned>((n + kReduceCols - 1) / kReduceCols), kReduceCols * 32, 0, s>>>(
        partial, plan.kslabs, n, plan.lp, ell, Y, ldy, info);
    return cudaGetLastError();
}

// --------------------------------------------------- standalone scaled cast

// One thread per (64-row block, column): the cast exactly as the sketch's
// converter warps perform it, written out as format bits and shifts.
__global__ void k_scale_cast(const void* __restrict__ A, int a_f64, int64_t m, int64_t n, int64_t lda,
                             int nsplit, int f16, uint16_t* __restrict__ pieces,
                             int32_t* __restrict__ shifts, int32_t* info) {
    const int64_t nb = (m + kChunkRows - 1) / kChunkRows;
    const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= nb * n) return;
    const int64_t j = idx / nb, b = idx - j * nb;
    const int64_t r0 = b * kChunkRows;
    const int rows = static_cast<int>(min(static_cast<int64_t>(kChunkRows), m - r0));
    int shift;
    if (a_f64) {
        const double* col = static_cast<const double*>(A) + j * lda + r0;
        uint32_t mx = 0;
        for (int r = 0; r < rows; ++r)
            mx = max(mx, static_cast<uint32_t>(__double2hiint(col[r])) & 0x7fffffffu);
        if ((mx >> 20) == 0x7FFu) set_info(info, kInfoNonFinite);
        shift = shift_from_max_f64hi(mx, f16);
        const F64CastBlock cb = f64_cast_block(shift);
        // the converter's fast path, with the exact routine for out-of-range values
        auto conv = [&](double x) {
            bool slow = cb.slow;
            const float f = scaled_f32_from_f64_fast(x, static_cast<uint32_t>(__double2hiint(x)) << 1, cb, slow);
            return slow ? scaled_f32_from_f64(x, shift) : f;
        };
        for (int r = 0; r < rows; r += 2) {
            float v0 = conv(col[r]);
            float v1 = r + 1 < rows ? conv(col[r + 1]) : 0.f;
            for (int p = 0; p < nsplit; ++p) {
                const uint32_t w = take_piece2(v0, v1, f16);
                pieces[(p * n + j) * m + r0 + r] = static_cast<uint16_t>(w & 0xFFFFu);
                if (r + 1 < rows) pieces[(p * n + j) * m + r0 + r + 1] = static_cast<uint16_t>(w >> 16);
            }
        }
    } else {
        const float* col = static_cast<const float*>(A) + j * lda + r0;
        uint32_t mx = 0;
        for (int r = 0; r < rows; ++r) mx = max(mx, __float_as_uint(col[r]) & 0x7fffffffu);
        if ((mx >> 23) == 0xFFu) set_info(info, kInfoNonFinite);
        shift = shift_from_max_f32(mx, f16);
        auto conv = [&](float x) {
            bool slow = false;
            const float f = scaled_f32_from_f32_fast(x, shift, slow);
            return slow ? scaled_f32_from_f32(x, shift) : f;
        };
        for (int r = 0; r < rows; r += 2) {
            float v0 = conv(col[r]);
            float v1 = r + 1 < rows ? conv(col[r + 1]) : 0.f;
            for (int p = 0; p < nsplit; ++p) {
                const uint32_t w = take_piece2(v0, v1, f16);
                pieces[(p * n + j) * m + r0 + r] = static_cast<uint16_t>(w & 0xFFFFu);
                if (r + 1 < rows) pieces[(p * n + j) * m + r0 + r + 1] = static_cast<uint16_t>(w >> 16);
            }
        }
    }
    shifts[j * nb + b] = shift;
}

cudaError_t launch_scale_cast(const void* A, int a_f64, int64_t m, int64_t n, int64_t lda, int precision,
                              uint16_t* pieces, int32_t* shifts, int32_t* info, cudaStream_t s) {
    const int64_t nb = (m + kChunkRows - 1) / kChunkRows;
    const int64_t total = nb * n;
    k_scale_cast<<<static_cast<unsigned>((total + 127) / 128), 128, 0, s>>>(
        A, a_f64, m, n, lda, precision_nsplit(precision), precision_is_f16(precision), pieces, shifts,
        info);
    return cudaGetLastError();
}

// ------------------------------------------------- the low-precision matrix A_L

// A_L of Algorithm 2 as FP32 values: every entry of every (64-row block, column) becomes
// 2^s fl_low(x 2^-s), the first piece of the scaled cast above times the block's power of
// two (exact in FP32 while the result is a normal float).  One thread per (block, column).
__global__ void k_low_cast(const void* __restrict__ A, int a_f64, int64_t m, int64_t n, int64_t lda, int f16,
                           float* __restrict__ out, int64_t ldo, int32_t* info) {
    const int64_t nb = (m + kChunkRows - 1) / kChunkRows;
    const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= nb * n) return;
    const int64_t j = idx / nb, b = idx - j * nb;
    const int64_t r0 = b * kChunkRows;
    const int rows = static_cast<int>(min(static_cast<int64_t>(kChunkRows), m - r0));
    float* dst = out + j * ldo + r0;
    if (a_f64) {
        const double* col = static_cast<const double*>(A) + j * lda + r0;
        uint32_t mx = 0;
        for (int r = 0; r < rows; ++r) mx = max(mx, static_cast<uint32_t>(__double2hiint(col[r])) & 0x7fffffffu);
        if ((mx >> 20) == 0x7FFu) set_info(info, kInfoNonFinite);
        const int shift = shift_from_max_f64hi(mx, f16);
        const F64CastBlock cb = f64_cast_block(shift);
        for (int r = 0; r < rows; r += 2) {
            auto conv = [&](double x) {
                bool slow = cb.slow;
                const float f = scaled_f32_from_f64_fast(x, static_cast<uint32_t>(__double2hiint(x)) << 1, cb, slow);
                return slow ? scaled_f32_from_f64(x, shift) : f;
            };
            float v0 = conv(col[r]);
            float v1 = r + 1 < rows ? conv(col[r + 1]) : 0.f;
            const uint32_t w = take_piece2(v0, v1, f16);
            const float p0 = f16 ? __half2float(__ushort_as_half(static_cast<unsigned short>(w & 0xFFFFu)))
                                 : __uint_as_float(w << 16);
            const float p1 = f16 ? __half2float(__ushort_as_half(static_cast<unsigned short>(w >> 16)))
                                 : __uint_as_float(w & 0xFFFF0000u);
            dst[r] = ldexpf(p0, shift);
            if (r + 1 < rows) dst[r + 1] = ldexpf(p1, shift);
        }
    } else {
        const float* col = static_cast<const float*>(A) + j * lda + r0;
        uint32_t mx = 0;
        for (int r = 0; r < rows; ++r) mx = max(mx, __float_as_uint(col[r]) & 0x7fffffffu);
        if ((mx >> 23) == 0xFFu) set_info(info, kInfoNonFinite);
        const int shift = shift_from_max_f32(mx, f16);
        for (int r = 0; r < rows; r += 2) {
            auto conv = [&](float x) {
                bool slow = false;
                const float f = scaled_f32_from_f32_fast(x, shift, slow);
                return slow ? scaled_f32_from_f32(x, shift) : f;
            };
            float v0 = conv(col[r]);
            float v1 = r + 1 < rows ? conv(col[r + 1]) : 0.f;
            const uint32_t w = take_piece2(v0, v1, f16);
            const float p0 = f16 ? __half2float(__ushort_as_half(static_cast<unsigned short>(w & 0xFFFFu)))
                                 : __uint_as_float(w << 16);
            const float p1 = f16 ? __half2float(__ushort_as_half(static_cast<unsigned short>(w >> 16)))
                                 : __uint_as_float(w & 0xFFFF0000u);
            dst[r] = ldexpf(p0, shift);
            if (r + 1 < rows) dst[r + 1] = ldexpf(p1, shift);
        }
    }
}

cudaError_t launch_low_cast(const void* A, int a_f64, int64_t m, int64_t n, int64_t lda, int f16, float* out,
                            int64_t ldo, int32_t* info, cudaStream_t s) {
    const int64_t total = ((m + kChunkRows - 1) / kChunkRows) * n;
    k_low_cast<<<static_cast<unsigned>((total + 127) / 128), 128, 0, s>>>(A, a_f64, m, n, lda, f16, out, ldo, info);
    return cudaGetLastError();
}

}  // namespace gid
