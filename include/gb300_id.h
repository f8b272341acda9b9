/*
 * gb300_id.h -- C ABI of the GB300 column interpolative decomposition library.
 *
 * The column ID (Dunton & Fox, "Mixed precision matrix interpolative
 * decompositions for model reduction", Sec. 1.1) approximates an m x n matrix
 * by k of its own columns:
 *
 *     A ~= A(:, J[0:k]) P,   P(:, J[0:k]) = I_k,   P(:, J[k:n]) = T,
 *
 * where J is the column permutation Z of a column-pivoted QR  A Z = Q R  and
 * T = R11^-1 R12 (Eq. (idconstruction); Algorithm 1).  This library computes
 * it on one GPU, optionally on a Gaussian sketch Y = Omega A instead of A, in
 * plain FP64 or in the mixed-precision form of Algorithm 2 (low-precision
 * cast and sketch, FP32 pivoted QR, FP64 coefficient solve).
 *
 * Conventions shared by every entry point
 *   - Matrices are column-major with an explicit leading dimension (ld >= rows);
 *     columns are the unit of the ID.  Omega is row-major (ell x m, row i
 *     contiguous).  Column indices are 0-based int32.
 *   - Every array argument is a DEVICE pointer owned by the caller unless the
 *     comment says "host".  The library allocates no device memory: scratch
 *     comes from the caller's `work` buffer (size from id_workspace_size).
 *   - `stream` is a cudaStream_t passed as void*.  Every call only enqueues
 *     work on that stream and returns; outputs are valid once the stream has
 *     reached that point.
 *   - The return value reports only errors the host can see before launching
 *     (bad arguments, too small a workspace, a CUDA launch error).  Numerical
 *     problems are reported in the device `info` word:
 *        0   success
 *        j>0 the pivot at step j-1 had zero residual norm: the rank is j-1
 *            and k_out = j-1
 *        -1  A (or Omega A) holds a non-finite value
 *        -2  a bounded device wait gave up (watchdog); outputs are invalid
 *        -3  (batched calls) a work-unit table entry did not fit its matrix
 *   - The complement J[k:n] is listed in ascending column index.
 */
#ifndef GB300_ID_H
#define GB300_ID_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ID_OK = 0,
    ID_ERR_ARG = 1,          /* invalid argument (sizes, null pointer, unsupported combination) */
    ID_ERR_WORKSPACE = 2,    /* work_bytes smaller than id_workspace_size() */
    ID_ERR_CUDA = 3,         /* a CUDA runtime call failed */
    ID_ERR_TIMEOUT = 4,      /* a synchronous check found the device watchdog fired */
    ID_ERR_UNSUPPORTED = 5   /* shape or option outside what this build implements */
} id_status_t;

typedef enum {
    ID_F64 = 0,              /* double */
    ID_F32 = 1               /* float */
} id_dtype_t;

/* Arithmetic of the factorisation.
 *   PLAIN_F64     everything in FP64 (Algorithm 1).  With a sketch, Omega is FP64.
 *   PLAIN_F32     pivoted QR in FP32 of the given matrix (no sketch; FP64 input is
 *                 rounded to FP32 as it is loaded), T in FP64.
 *   MIXED_BF16    Algorithm 2 re-cast for GB300: A is scaled by powers of two per
 *                 (64-row block, column), rounded to bfloat16, sketched on the
 *                 tensor cores with FP32 accumulation; pivoted QR of Y in FP32;
 *                 T = R11^-1 R12 in FP64 with iterative refinement.
 *                 Omega is bfloat16.
 *   MIXED_F16     as MIXED_BF16 with IEEE half (Omega is half).
 *   MIXED_BF16X2  A split into 2 bfloat16 pieces (hi + lo), both sketched.
 *   MIXED_BF16X3  A split into 3 bfloat16 pieces: an FP32-accurate sketch at the
 *                 same HBM traffic.
 *   LOW_BF16      Algorithm 2 as the paper states it (no sketch): the whole of A is
 *   LOW_F16       cast to the low-precision matrix A_L (bfloat16 / half, scaled by
 *                 powers of two per (64-row block, column) like the mixed sketch's
 *                 cast), and the pivoted QR of A_L runs in FP32 arithmetic on those
 *                 values (low-precision data, single-precision accumulation); T in FP64
 *                 with refinement.  The ID's columns can then be taken from A (the
 *                 mixed ID A_hat_M = A(:,J) P) or from A_L (the low ID
 *                 A_hat_L = A_L(:,J) P, A_L from id_low_cast). */
typedef enum {
    ID_PLAIN_F64 = 0,
    ID_PLAIN_F32 = 1,
    ID_MIXED_BF16 = 2,
    ID_MIXED_F16 = 3,
    ID_MIXED_BF16X2 = 4,
    ID_MIXED_BF16X3 = 5,
    ID_LOW_BF16 = 6,
    ID_LOW_F16 = 7
} id_precision_t;

/* Rows per power-of-two scaling block of the low-precision cast (a block of
 * rows of one column shares one shift). */
#define ID_SCALE_BLOCK_ROWS 64

/* Largest sketch size ell (= k + oversampling) of the tensor-core sketch. */
#define ID_MAX_ELL 256

typedef struct {
    int32_t k;               /* target rank when rel_tol == 0 (Algorithm 1) */
    double rel_tol;          /* > 0: rank = smallest k with ||R22||_F <= rel_tol ||W||_F,
                                W the matrix being pivoted (A or Y), capped by k_max */
    int32_t k_max;           /* cap for rel_tol mode (and T's row capacity) */
    int32_t sketch;          /* 0: pivot A itself; 1: pivot Y = Omega A */
    int32_t ell;             /* rows of Omega (k + oversampling) when sketch = 1 */
    int32_t precision;       /* id_precision_t */
    const void* omega;       /* device, ell x m row-major: bfloat16 bits (MIXED_BF16*),
                                half bits (MIXED_F16), double (PLAIN_F64) */
    int64_t omega_ld;        /* row stride of omega in elements (>= m; 0 means m).  The
                                tensor-core sketch reads omega with TMA: it needs
                                omega 16-byte aligned and omega_ld a multiple of 8 */
    int32_t refine_steps;    /* iterative-refinement steps of the T solve (default 1) */
    int32_t estimate_error;  /* 1: write err_out = ||A - A(:,J)P||_F / ||A||_F (FP64) */
    int64_t watchdog_ms;     /* time limit of every device wait in ms; 0 = default (4000) */
} id_opts_t;

/* Fill opts with defaults: k = 0, rel_tol = 0, k_max = 0, sketch = 0,
 * ell = 0, precision = PLAIN_F64, omega = NULL, omega_ld = 0,
 * refine_steps = 1, estimate_error = 0, watchdog_ms = 0. */
void id_opts_default(id_opts_t* opts);

/* Device bytes of scratch id_factor needs for this problem (host call, no
 * GPU work).  Returns ID_ERR_ARG / ID_ERR_UNSUPPORTED for invalid options. */
id_status_t id_workspace_size(id_dtype_t a_dtype, int64_t m, int64_t n,
                              const id_opts_t* opts, size_t* bytes);

/* One column ID of A (m x n, column-major, lda >= m; dtype a_dtype).
 *   Sketch (optional, Sec. 5 future work): Y = Omega A, ell x n.
 *   Pivoted QR (Sec. 1.1, Algorithm 1, the pivoted QR): truncated Householder QR with
 *   Businger-Golub pivoting and column-norm downdating on W = Y or A.
 *   Coefficients (Algorithm 1, the coefficient solve): T = R11^-1 R12 in FP64.
 * Outputs (device):
 *   J      [n]  int32, J[0:k] the skeleton in pivot order, J[k:n] the rest
 *   T      k_cap x (n - k) doubles, column-major, ldt >= k_cap where
 *          k_cap = k (fixed rank) or k_max (rel_tol mode); only the first
 *          k_out rows and n - k_out columns are meaningful
 *   k_out  [1]  the rank used
 *   info   [1]  status word (see above)
 *   err_out[1]  nullable; relative Frobenius residual when estimate_error = 1
 * Errors: ID_ERR_ARG for m, n < 1, lda < m, k outside [1, min(rows, n)],
 * ell outside [k, min(m, ID_MAX_ELL)], null outputs, precision / dtype
 * combinations not listed above (mixed precisions require sketch = 1;
 * PLAIN_F32 requires sketch = 0 and takes A as ID_F32, or as ID_F64 whose
 * values are rounded to FP32 (nearest even) when the pivoted QR loads them;
 * LOW_* require sketch = 0; PLAIN_F64 with a sketch requires ID_F64). */
id_status_t id_factor(const void* A, id_dtype_t a_dtype, int64_t m, int64_t n, int64_t lda,
                      const id_opts_t* opts,
                      int32_t* J, double* T, int64_t ldt, int32_t* k_out, int32_t* info,
                      double* err_out, void* work, size_t work_bytes, void* stream);

/* Rank-adaptive randomized ID: the sketching the paper names as a next step (Sec. 5),
 * grown by blocks of Omega's rows until the ID meets a tolerance on A itself.  For
 * ell = block, 2 block, ... up to opts->ell:
 *   Y(ell - b : ell, :) = Omega(ell - b : ell, :) A     (only the new rows are sketched),
 *   rank k = min(opts->k_max, ell - oversample, n): pivoted QR of Y(0:ell, :), T,
 *   e = ||A - A(:,J) P||_F / ||A||_F in FP64 (as estimate_error),
 * and it stops at the first ell with e <= opts->rel_tol (or after the last block).  The
 * rank therefore grows with the sketch and is the smallest multiple-of-block step that
 * meets the tolerance.  opts: rel_tol > 0 the target, k_max the rank cap (<= ell -
 * oversample), sketch = 1, ell = rows of omega available, precision PLAIN_F64 or MIXED_*,
 * omega / omega_ld as for id_factor.  Outputs as id_factor (T with ldt >= k_max), err_out
 * (device, required) the final e, *ell_out (host, nullable) the sketch rows used.
 * Synchronises the stream once per block (the stopping test reads e on the host).
 * Errors: ID_ERR_ARG, ID_ERR_WORKSPACE, ID_ERR_UNSUPPORTED, ID_ERR_CUDA, ID_ERR_TIMEOUT. */
id_status_t id_adaptive_workspace_size(id_dtype_t a_dtype, int64_t m, int64_t n, const id_opts_t* opts,
                                       int32_t block, int32_t oversample, size_t* bytes);
id_status_t id_factor_adaptive(const void* A, id_dtype_t a_dtype, int64_t m, int64_t n, int64_t lda,
                               const id_opts_t* opts, int32_t block, int32_t oversample, int32_t* J, double* T,
                               int64_t ldt, int32_t* k_out, int32_t* info, double* err_out, int32_t* ell_out,
                               void* work, size_t work_bytes, void* stream);

/* Row ID (the standard companion of the column ID of Sec. 1.1; the paper has only the
 * column form): A ~= X A(I[0:k], :) with X(I[0:k], :) = I_k and X(I[k:m], :) = T^T, i.e.
 * row I[k+c] of A ~= sum_b T(b, c) row I[b].  It is the column ID of A^T: A is
 * transposed into the workspace (tiled copy) and id_factor runs on it with the same
 * options (a sketch then uses Omega of ell x n, sketching A^T's columns).  Outputs as
 * id_factor with the roles of m and n exchanged: I [m], T k_cap x (m - k) (ldt >= k_cap),
 * k_out, info, err_out (the same relative Frobenius residual).  Workspace from
 * id_rows_workspace_size.  Errors as id_factor. */
id_status_t id_rows_workspace_size(id_dtype_t a_dtype, int64_t m, int64_t n, const id_opts_t* opts, size_t* bytes);
id_status_t id_factor_rows(const void* A, id_dtype_t a_dtype, int64_t m, int64_t n, int64_t lda, const id_opts_t* opts,
                           int32_t* I, double* T, int64_t ldt, int32_t* k_out, int32_t* info, double* err_out,
                           void* work, size_t work_bytes, void* stream);

/* Two-sided ID A ~= X A(I[0:k], J[0:k]) P at a fixed rank k (opts->rel_tol = 0): the
 * column ID of A with opts (J, Tc as id_factor), then the rank-k row ID of the column
 * skeleton C = A(:, J[0:k]) in plain precision (FP64 for ID_F64 data, FP32 for ID_F32)
 * giving I [m] and Tr k x (m - k) (ldtr >= k); X is the row ID's interpolation matrix.
 * k_out[2], info[2] (device): [0] the column stage, [1] the row stage.  Workspace from
 * id_two_sided_workspace_size.  Errors as id_factor; ID_ERR_ARG for a tolerance. */
id_status_t id_two_sided_workspace_size(id_dtype_t a_dtype, int64_t m, int64_t n, const id_opts_t* opts,
                                        size_t* bytes);
id_status_t id_factor_two_sided(const void* A, id_dtype_t a_dtype, int64_t m, int64_t n, int64_t lda,
                                const id_opts_t* opts, int32_t* J, double* Tc, int64_t ldtc, int32_t* I, double* Tr,
                                int64_t ldtr, int32_t* k_out, int32_t* info, void* work, size_t work_bytes,
                                void* stream);

/* The sketch step alone (the sketching of Sec. 5; Algorithm 2 for
 * the cast): Y = Omega A (ell x n, column-major, ldy >= ell).
 * PLAIN_F64: Omega and Y are double.  MIXED_*: Omega is bfloat16/half bits,
 * A is scaled per (ID_SCALE_BLOCK_ROWS rows, column) by a power of two,
 * rounded to nearest-even in the low format (1-3 pieces), multiplied on the
 * tensor cores with FP32 accumulation, and Y is float.  info (device, nullable)
 * is set to -1 if A holds a non-finite value or an entry of Y is not finite
 * (a column whose scaled blocks reach past the FP32 range overflows the FP32
 * accumulation; its entries of Y are then inf or NaN), else 0. */
id_status_t id_sketch(const void* A, id_dtype_t a_dtype, int64_t m, int64_t n, int64_t lda,
                      const void* omega, int64_t omega_ld, int32_t ell, int32_t precision,
                      void* Y, int64_t ldy, int32_t* info,
                      void* work, size_t work_bytes, void* stream);

/* id_sketch without a workspace.  The paper has no counterpart: this entry
 * point is for callers that cannot allocate device memory when they call the
 * library (a plug-in whose host framework owns every device allocation, a
 * service whose memory budget is fixed at start-up, code that must not
 * allocate while it runs).  Same arguments and results as id_sketch, minus
 * work/work_bytes: the split-K scratch lives in a static device array of
 * ID_NOALLOC_SCRATCH_BYTES bytes that every GPU loading this library holds
 * until the process exits.
 *   - Returns ID_ERR_WORKSPACE, without launching anything, when the problem's
 *     split-K scratch exceeds ID_NOALLOC_SCRATCH_BYTES; that scratch is
 *     id_sketch_workspace_size minus the 512 bytes of alignment slack it adds
 *     for a caller's buffer (the static array is already aligned).  Other
 *     errors as id_sketch.
 *   - The array is shared by all calls on a device and keeps the last call's
 *     contents.  Calls that overlap on the GPU race on it: serialise them
 *     (one stream, or explicit ordering between streams and host threads).
 *   - The first call on a device looks up the array's device address (with
 *     that device current); make that first call before any stream capture.
 *   - Allocates nothing: no cudaMalloc, cudaFree or allocating library call. */
#define ID_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
id_status_t id_sketch_noalloc(const void* A, id_dtype_t a_dtype, int64_t m, int64_t n, int64_t lda,
                              const void* omega, int64_t omega_ld, int32_t ell, int32_t precision,
                              void* Y, int64_t ldy, int32_t* info, void* stream);

/* Scratch bytes id_sketch needs. */
id_status_t id_sketch_workspace_size(id_dtype_t a_dtype, int64_t m, int64_t n, int32_t ell,
                                     int32_t precision, size_t* bytes);

/* The scaled low-precision cast of Algorithm 2 on its own, as the
 * mixed sketch performs it: for every block of ID_SCALE_BLOCK_ROWS rows of a
 * column, shift s = exponent that puts the block's largest magnitude in
 * [0.5, 1) (bfloat16) or [2^13, 2^14) (half), zero block -> 0; each entry x
 * becomes nsplit pieces q_t = fl(x 2^-s - q_0 - ... - q_{t-1}).
 * Outputs: pieces, nsplit consecutive m x n column-major uint16 matrices
 * (ld = m) of format bits; shifts, ceil(m / ID_SCALE_BLOCK_ROWS) x n int32
 * column-major.  precision selects the format and nsplit (MIXED_BF16: 1,
 * MIXED_BF16X2: 2, MIXED_BF16X3: 3, MIXED_F16: 1).  info as in id_sketch. */
id_status_t id_scale_cast(const void* A, id_dtype_t a_dtype, int64_t m, int64_t n, int64_t lda,
                          int32_t precision, uint16_t* pieces, int32_t* shifts,
                          int32_t* info, void* stream);

/* The low-precision matrix A_L of Algorithm 2 (A_L = fl(A)), as FP32 values: for every
 * block of ID_SCALE_BLOCK_ROWS rows of a column, the shift s of id_scale_cast and
 * A_L(i,j) = 2^s fl_low(x 2^-s), fl_low the first piece of that cast (bfloat16 for
 * LOW_BF16 / MIXED_BF16*, half for LOW_F16 / MIXED_F16), x = A(i,j) taken at FP32
 * precision.  This is the matrix the LOW_* precisions of id_factor pivot.  AL: m x n
 * floats, column-major, ldal >= m.  info (nullable) -1 if A holds a non-finite value.
 * A_L entries below the FP32 normal range (data spanning more than the FP32 range)
 * round to FP32 subnormals or zero.  Errors: ID_ERR_ARG, ID_ERR_CUDA. */
id_status_t id_low_cast(const void* A, id_dtype_t a_dtype, int64_t m, int64_t n, int64_t lda, int32_t precision,
                        float* AL, int64_t ldal, int32_t* info, void* stream);

/* A_hat = A(:,J[0:k]) P of one matrix (Sec. 1.1; Algorithm 2's last line with A = A_D
 * for the mixed ID, A = A_L for the low ID): A m x n of a_dtype (column-major, lda),
 * J as id_factor returns it, T k x (n-k) doubles (ldt >= k).  Ahat: m x n of a_dtype
 * (ldh >= m), columns J[0:k] copied from A, columns J[k:n] accumulated in FP64.
 * Ahat must not alias A.  Errors: ID_ERR_ARG, ID_ERR_CUDA. */
id_status_t id_reconstruct_one(const void* A, id_dtype_t a_dtype, int64_t m, int64_t n, int64_t lda,
                               const int32_t* J, int32_t k, const double* T, int64_t ldt, void* Ahat, int64_t ldh,
                               void* stream);

/* Adjoint of the column ID with the pivot set J held fixed (the
 * differentiable form; the paper does not differentiate the ID), FP32.
 * The map is the fixed-pivot least-squares ID: X = A(:,J[0:k]),
 * C = A(:,J[k:n]), T = X^+ C (what a column-pivoted QR of A gives as
 * R11^-1 R12, Sec. 1.1), A_hat = A(:,J[0:k]) P (Algorithm 1).
 * Given dL/dA_hat (dAhat, nullable) and dL/dT (dT, nullable) it writes
 * dA = dL/dA (every column).  With the thin QR X = Q R:
 *   B1 = Q^T G_c + R^-T dT,  Z = G_c T^T + C (R^-1 B1)^T,
 *   dA(:,J[0:k]) = G_s + Z - Q (Q^T Z + R^-T dT T^T),  dA(:,J[k:n]) = Q B1.
 * Batched over `batch` matrices of equal shape: matrix b starts at
 * A + b*strideA (column-major, lda), J + b*strideJ (a permutation of 0..n-1
 * as id_factor returns it), T + b*strideT (k x (n-k) doubles, ldt), dAhat +
 * b*strideG (m x n, ldg), dT + b*strideDT (k x (n-k) doubles, lddt), dA +
 * b*strideD (m x n, ldd, must not alias the inputs).  1 <= k <= min(m, n, 128).
 * X must have full column rank.  Errors: ID_ERR_ARG, ID_ERR_WORKSPACE,
 * ID_ERR_CUDA. */
id_status_t id_backward_workspace_size(int64_t batch, int64_t m, int64_t n, int32_t k, size_t* bytes);
id_status_t id_backward(int64_t batch, const float* A, int64_t m, int64_t n, int64_t lda, int64_t strideA,
                        const int32_t* J, int64_t strideJ, int32_t k, const double* T, int64_t ldt, int64_t strideT,
                        const float* dAhat, int64_t ldg, int64_t strideG, const double* dT, int64_t lddt,
                        int64_t strideDT, float* dA, int64_t ldd, int64_t strideD, void* work, size_t work_bytes,
                        void* stream);

/* Reconstruction A_hat = A(:,J[0:k]) P with P(:,J[0:k]) = I, P(:,J[k:n]) = T
 * (Sec. 1.1; Algorithm 1, the reconstruction), FP32, batched like id_backward.  Ahat is
 * m x n (ldh) per matrix. */
id_status_t id_reconstruct_workspace_size(int64_t batch, int64_t n, int32_t k, size_t* bytes);
id_status_t id_reconstruct(int64_t batch, const float* A, int64_t m, int64_t n, int64_t lda, int64_t strideA,
                           const int32_t* J, int64_t strideJ, int32_t k, const double* T, int64_t ldt, int64_t strideT,
                           float* Ahat, int64_t ldh, int64_t strideH, void* work, size_t work_bytes, void* stream);

/* ------------------------------------------------------------ batched IDs
 * Many independent mixed-precision IDs of uneven sizes in one stream-ordered
 * launch sequence (the batched form; the paper factors one matrix at a
 * time).  Matrix i is m[i] x n[i] (column-major, lda[i]) with target rank
 * k[i]; it is sketched with the leading ell_i = min(k[i] + oversample, m[i])
 * rows and m[i] columns of one shared low-precision Gaussian Omega, then
 * pivoted (FP32) and solved (FP32 solves, FP64 refinement residual) as
 * id_factor does for one matrix with the same precision and Omega.
 *
 * Shapes are fixed when the plan is made, because they set the launch shapes;
 * the matrices' addresses are fixed when they are bound (each matrix gets its
 * own TMA tensor map, stored in the workspace).  Work is split into units
 * (128-column tiles times row slabs for the sketch, one cluster of CTAs per
 * matrix for the pivoted QR, blocks of T columns for the solve), ordered
 * largest first; the unit sizes come from id_batch_opts_t or from the
 * autotuner's cache.  A captured CUDA graph of id_factor_batched replays on
 * new values written to the bound matrices.
 *
 * Calls, in order:
 *   id_batch_plan_create  host only: checks shapes, builds the tables.
 *   id_batch_plan_query / id_batch_workspace_size
 *   id_batch_bind         encodes the matrices' tensor maps and copies the
 *                         plan's tables into the head of `work` (stream-
 *                         ordered); again after id_batch_autotune only if the
 *                         addresses change.
 *   id_factor_batched     launches only (graph-capturable).
 *   id_batch_plan_destroy
 * One call of a plan may be in flight at a time (it owns the fork/join
 * streams and events of its pivoted-QR launches). */
typedef struct id_batch_plan id_batch_plan_t;

typedef struct {
    int32_t precision;       /* ID_MIXED_BF16, ID_MIXED_F16, ID_MIXED_BF16X2 or ID_MIXED_BF16X3 */
    int32_t oversample;      /* p: ell_i = min(k_i + p, m_i) <= 160; default 10 */
    int32_t refine_steps;    /* refinement steps of the T solve; default 1 */
    double rel_tol;          /* 0: fixed ranks k_i; > 0: stop at the first step whose remaining
                                norm is <= rel_tol times the initial one, k_i the cap */
    int64_t watchdog_ms;     /* bound of every device wait; 0 = 4000 ms */
    int32_t slab_chunks;     /* sketch unit height in 64-row chunks: 16, 32 or 64 (0 = 32) */
    int32_t cpqr_tpc;        /* pivoted-QR threads per column, 2 or 4 (0 = 4) */
    int32_t solve_warps;     /* warps per solve CTA, 1..16 (0 = 8) */
    int32_t solve_cols;      /* T columns per solve CTA, >= 16 (0 = 32) */
    const char* tune_cache;  /* host, nullable: autotuner cache (JSON lines) whose entry for this
                                device and batch overrides the four shape fields above */
} id_batch_opts_t;

id_batch_opts_t id_batch_opts_default(void);

/* m, n, lda, k: HOST arrays of length batch.  Requirements per matrix:
 * 1 <= k[i] <= min(m[i], n[i], 128), lda[i] >= m[i], ell_i <= 160,
 * n[i] <= 2048.  Errors: ID_ERR_ARG, ID_ERR_UNSUPPORTED (a shape the kernels
 * do not cover).
 * precision = ID_PLAIN_F64 (FP64 matrices, fixed ranks only) makes the plan of
 * the FP64 twin: matrix i's sketched FP64 ID exactly as id_factor computes it
 * (sketch = 1, ell_i, PLAIN_F64, the shared FP64 Omega), the matrices one after
 * the other on the caller's stream, each in its own slice of the workspace.
 * It takes any shape id_factor takes (no limits on k, ell or n), ignores the
 * tuning fields, and id_batch_autotune rejects it (ID_ERR_ARG).
 * precision = ID_PLAIN_F32 (FP64 or FP32 matrices, fixed ranks or a tolerance,
 * k[i] <= 128, any m and n) pivots every matrix itself, without a sketch, in
 * FP32 (Algorithm 1 on A in single precision, as id_factor's PLAIN_F32): the
 * matrices go in waves whose FP32 working copies fit half of L2, each wave one
 * cooperative launch in which a group of CTAs factors each matrix, and then one
 * batched T solve (FP32 solves, one refinement step) for all of them.  Omega
 * is not read (NULL allowed); id_batch_autotune rejects it (ID_ERR_ARG). */
id_status_t id_batch_plan_create(int32_t batch, id_dtype_t a_dtype, const int64_t* m, const int64_t* n,
                                 const int64_t* lda, const int32_t* k, const id_batch_opts_t* opts,
                                 id_batch_plan_t** plan);
void id_batch_plan_destroy(id_batch_plan_t* plan);

/* Sizes of the caller's buffers (all host outputs, each nullable):
 *   work_bytes       workspace for id_batch_bind / id_factor_batched;
 *   j_offsets[batch+1]  J of matrix i is J[j_offsets[i] .. +n[i]) (int32);
 *   t_offsets[batch+1]  T of matrix i starts at T + t_offsets[i], k[i] x tcols_i
 *                    doubles with ldt = k[i]; tcols_i = n[i] - k[i] for fixed
 *                    ranks, n[i] - 1 under a tolerance (first n[i] - k_out[i] used);
 *   ell_max, m_max   Omega must have at least ell_max rows and m_max columns. */
id_status_t id_batch_plan_query(const id_batch_plan_t* plan, size_t* work_bytes, int64_t* j_offsets,
                                int64_t* t_offsets, int32_t* ell_max, int64_t* m_max);

/* The plan's unit shapes and counts as a one-line JSON object (host buffer;
 * truncated to len - 1 characters).  Returns the length it needed. */
int64_t id_batch_plan_describe(const id_batch_plan_t* plan, char* buf, int64_t len);

id_status_t id_batch_workspace_size(const id_batch_plan_t* plan, size_t* bytes);

/* A: HOST array of batch DEVICE pointers to the matrices (a_dtype of the plan).
 * Every matrix of a mixed plan must be addressable by TMA: its address and
 * lda[i] * element size multiples of 16 bytes (ID_ERR_ARG otherwise).  work: 256-byte aligned,
 * at least work_bytes; it holds the tables from now on. */
id_status_t id_batch_bind(id_batch_plan_t* plan, const void* const* A, void* work, size_t work_bytes,
                          void* stream);

/* omega: bfloat16/half bits (per the precision), row-major with omega_ld >=
 * m_max, omega_ld a multiple of 8, 16-byte aligned, >= ell_max rows; for a
 * PLAIN_F64 plan, doubles, row-major with omega_ld >= m_max and >= ell_max rows;
 * for a PLAIN_F32 plan not read (NULL allowed).
 * J (packed int32), T (packed double), k_out[batch], info[batch]: outputs as
 * laid out by id_batch_plan_query; info per matrix as for id_factor, plus -3
 * when a table entry does not fit its matrix (never expected; nothing of that
 * matrix is computed).  Errors: ID_ERR_ARG (also: work not the buffer last
 * bound), ID_ERR_WORKSPACE, ID_ERR_CUDA. */
id_status_t id_factor_batched(const id_batch_plan_t* plan, const void* omega, int64_t omega_ld, int32_t* J,
                              double* T, int32_t* k_out, int32_t* info, void* work, size_t work_bytes,
                              void* stream);

/* Autotuner: times id_factor_batched on the bound buffers for each candidate
 * sketch unit height, pivoted-QR threads per column, and solve CTA shape
 * (coordinate search, median of `reps` timed calls after one warm-up), keeps
 * the fastest in the plan, rewrites the tables in `work`, and, when cache_path
 * is not NULL, writes the choice under this device's and this batch's key as
 * one JSON line of that file (replacing an older line with the same key).
 * The device synchronises.  best_ms (host, nullable) receives the tuned time.
 * Errors: as id_factor_batched, ID_ERR_ARG when the cache file cannot be
 * written. */
id_status_t id_batch_autotune(id_batch_plan_t* plan, const void* omega, int64_t omega_ld, int32_t* J, double* T,
                              int32_t* k_out, int32_t* info, void* work, size_t work_bytes, void* stream,
                              int32_t reps, const char* cache_path, double* best_ms);

/* Split a batch over `world` GPUs (one process each) by longest-processing-time:
 * matrices in decreasing order of their sketch + pivoted-QR + solve work, each
 * to the least loaded rank so far (ties to the lower rank).  Host only and
 * deterministic, so every rank computes the same split without communication.
 * m, n, k: HOST arrays of length batch; rank_of (HOST, length batch) receives
 * the rank of each matrix; load (HOST, length world, nullable) receives each
 * rank's modelled work in flop.  ell_i = min(k_i + oversample, m_i) as in
 * id_batch_plan_create.  Errors: ID_ERR_ARG. */
id_status_t id_batch_shard(int32_t batch, const int64_t* m, const int64_t* n, const int32_t* k, int32_t oversample,
                           int32_t world, int32_t* rank_of, double* load);

/* Profiling aid (not part of the computation).  When set, the next id_factor
 * calls made from this host thread record the caller's CUDA events (cudaEvent_t
 * passed as void*) on their stream at the stage boundaries:
 *   events[0] start, [1] after the sketch kernel, [2] after the sketch's
 *   split-K reduction, [3] after the pivoted QR, [4] after the T solve,
 *   [5] end.
 * Stages a call does not run record at the same point as the previous one.
 * count <= 0 or events == NULL switches recording off.  Always ID_OK. */
id_status_t id_set_stage_events(void* const* events, int32_t count);

/* Profiling aid (not part of the computation): the FP32 (which = 0, FFMA) or FP64
 * (which = 1, DFMA) multiply-add rate of the current GPU in TFLOP/s (host output),
 * measured as eight independent FMA chains per thread on a grid filling every SM,
 * flops over the CUDA-event time of one launch after a warm-up launch (about 30 ms).
 * These are the peaks the ALU-bound kernels' rooflines are reported against.
 * Synchronises the stream.  Errors: ID_ERR_ARG, ID_ERR_CUDA. */
id_status_t id_probe_fma_peak(int32_t which, double* tflops, void* stream);

/* Self-check (not part of the computation): widens every one of the 2^32 FP32 bit
 * patterns to FP64 with the integer routine the FP32 pivoted-QR kernels use to store
 * their R entries (IEEE 754 binary32 -> binary64: exponent rebiased, significand moved,
 * subnormals normalised) and with the hardware conversion, and writes to *mismatches
 * (host output) how many differ in bits (a NaN need only stay a NaN).  About 10 ms;
 * synchronises the stream.  Errors: ID_ERR_ARG (mismatches NULL), ID_ERR_CUDA. */
id_status_t id_check_widen(uint64_t* mismatches, void* stream);

/* Human-readable name of a status code (static string, never NULL). */
const char* id_status_string(id_status_t status);

/* Library version string (static). */
const char* id_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GB300_ID_H */
