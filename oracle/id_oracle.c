/*
 * FP64 CPU oracle for the column interpolative decomposition (ID).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, obviously correct
 * restatement of what the GPU library computes.  It shares no code, header,
 * table or constant with the GPU library, and nothing in the library calls it:
 * only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * load it.
 *
 * What it computes (Dunton & Fox, "Mixed precision matrix interpolative
 * decompositions for model reduction"):
 *
 *   - the column ID A ~= A(:,I) P of Sec. 1.1, built from a column-pivoted QR
 *     AZ = QR truncated after k steps, with T = R11^-1 R12 and
 *     P(:,I) = [I_k  T] (Sec. 1.1, Eq. (idconstruction); Algorithm 1);
 *   - the pivoted QR as Householder reflections with greedy (largest residual
 *     column norm) pivoting.  The paper uses modified Gram-Schmidt for the
 *     same greedy selection; both give the same pivots and the same T in
 *     exact arithmetic.  An MGS variant is kept here as a cross-check;
 *   - residual column norms either recomputed exactly at every step (the
 *     plain definition of greedy selection) or downdated, nu_i -= R(j,i)^2,
 *     with the recompute-on-cancellation test of Drmac and Bujanovic
 *     ("On the failure of rank-revealing QR factorization software", ACM
 *     TOMS 35(2), 2008);
 *   - the optional Gaussian sketch Y = Omega A (the paper names sketching as
 *     future work in Sec. 5);
 *   - the low-precision cast of Algorithm 2 (A_L = fl(A)) as round-to-
 *     nearest-even to bfloat16 or IEEE half after an exact power-of-two
 *     scaling of each block of rows of each column (the scaled value is
 *     taken at FP32 precision first, then split into 1-3 low-format
 *     pieces), and the sketch of the cast matrix evaluated exactly enough
 *     (FP64) to bound an FP32-accumulated sketch.
 *
 * Storage: matrices are column-major with an explicit leading dimension.
 * Omega is row-major (ell x m, row i contiguous).  Column indices are 0-based.
 * The complement Jc = J[k:n] is listed in ascending original column index.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>

#define A_(M, ld, i, j) ((M)[(int64_t)(j) * (ld) + (i)])

/* ------------------------------------------------------------------ sketch */

/* Y = Omega A, FP64, one dot product per entry in natural order.
 * Omega: ell x m row-major; A: m x n col-major (lda); Y: ell x n col-major (ldy). */
void orc_sketch_f64(const double* omega, int64_t ell, int64_t m,
                    const double* A, int64_t lda, int64_t n,
                    double* Y, int64_t ldy)
{
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < ell; ++i) {
            double s = 0.0;
            const double* w = omega + i * m;
            for (int64_t l = 0; l < m; ++l) s += w[l] * A_(A, lda, l, j);
            A_(Y, ldy, i, j) = s;
        }
}

/* ------------------------------------------------------- low-precision cast */

/* Formats: 0 = bfloat16 (8 significant bits, normal exponents -126..127),
 *          1 = IEEE half (11 significant bits, normal exponents -14..15). */
static void fmt_params(int fmt, int* p, int* emin, int* emax)
{
    if (fmt == 0) { *p = 8;  *emin = -126; *emax = 127; }
    else          { *p = 11; *emin = -14;  *emax = 15;  }
}

/* Round x to the nearest value of the format, ties to even (IEEE 754
 * roundTiesToEven): quantum q = 2^(max(E, emin) - (p-1)) with
 * E = floor(log2|x|); result = nearbyint(x/q) * q; beyond the largest finite
 * value the result is +-inf.  x/q and the product are exact in FP64. */
double orc_round_fmt(double x, int fmt)
{
    int p, emin, emax;
    fmt_params(fmt, &p, &emin, &emax);
    if (x == 0.0 || !isfinite(x)) return x;
    int e2;
    (void)frexp(x, &e2);          /* |x| = f 2^e2, f in [0.5, 1) */
    int E = e2 - 1;               /* |x| = g 2^E, g in [1, 2) */
    int qe = (E > emin ? E : emin) - (p - 1);
    double r = ldexp(nearbyint(ldexp(x, -qe)), qe);
    double maxfin = ldexp(2.0 - ldexp(1.0, 1 - p), emax);
    if (fabs(r) > maxfin) return copysign(INFINITY, x);
    return r;
}

/* Power-of-two shift s for a block whose largest magnitude is mx:
 * bfloat16 places mx * 2^-s in [0.5, 1); half places it in [2^13, 2^14).
 * The shift is read from the binary exponent of mx, so a block whose largest
 * magnitude is zero or subnormal in the input format (below 2^-1022 for
 * double input, 2^-126 for float input) gets s = 0. */
int orc_block_shift(double mx, int fmt, int in_f32)
{
    double tiny = in_f32 ? ldexp(1.0, -126) : DBL_MIN;
    if (!(mx >= tiny)) return 0;
    int e2;
    (void)frexp(mx, &e2);
    return fmt == 0 ? e2 : e2 - 14;
}

/* Scaled cast of A (Algorithm 2, A_L = fl(A)) with per-(block, column)
 * power-of-two scaling.  Rows are split in blocks of block_rows; block b of
 * column j gets shift s(b,j) from its largest magnitude.  Each entry is scaled
 * by 2^-s(b,j) and rounded to the nearest FP32 value (ties to even; exact for
 * FP32 inputs), x32 = fl32(x 2^-s); x32 is then split into low-format pieces
 * piece 0 = fl(x32), piece 1 = fl(x32 - piece0), piece 2 = fl(x32 - piece0 -
 * piece1) (nsplit = 1, 2 or 3; three bfloat16 pieces sum to x32 exactly).
 * in_f32 says the values of A came from float storage.  Outputs (doubles):
 *   Q: nsplit consecutive m x n col-major matrices (ld = m) of piece values,
 *   S: shifts, nblocks x n col-major (ld = nblocks).
 * Returns 0, or -1 if A holds a non-finite value. */
int orc_quantize(const double* A, int64_t m, int64_t n, int64_t lda,
                 int fmt, int nsplit, int64_t block_rows, int in_f32,
                 double* Q, int32_t* S)
{
    int64_t nb = (m + block_rows - 1) / block_rows;
    int bad = 0;
    for (int64_t j = 0; j < n; ++j)
        for (int64_t b = 0; b < nb; ++b) {
            int64_t r0 = b * block_rows, r1 = r0 + block_rows < m ? r0 + block_rows : m;
            double mx = 0.0;
            for (int64_t i = r0; i < r1; ++i) {
                double a = A_(A, lda, i, j);
                if (!isfinite(a)) bad = 1;
                if (fabs(a) > mx) mx = fabs(a);
            }
            int s = orc_block_shift(mx, fmt, in_f32);
            S[j * nb + b] = s;
            for (int64_t i = r0; i < r1; ++i) {
                double x32 = (double)(float)ldexp(A_(A, lda, i, j), -s);
                double acc = 0.0;
                for (int t = 0; t < nsplit; ++t) {
                    double piece = orc_round_fmt(x32 - acc, fmt);
                    Q[(int64_t)t * m * n + j * m + i] = piece;
                    acc += piece;
                }
            }
        }
    return bad ? -1 : 0;
}

/* Sketch of the scaled cast: Y(i,j) = sum_b 2^s(b,j) sum_t sum_{l in b}
 * Omega(i,l) piece_t(l,j), in FP64.  Each product of two low-format values is
 * exact in FP64; only the FP64 sums round, so this bounds an FP32-accumulated
 * evaluation of the same quantity. */
int orc_sketch_lowp(const double* omega, int64_t ell, int64_t m,
                    const double* A, int64_t lda, int64_t n,
                    int fmt, int nsplit, int64_t block_rows, int in_f32,
                    double* Y, int64_t ldy)
{
    int64_t nb = (m + block_rows - 1) / block_rows;
    double* Q = (double*)malloc(sizeof(double) * (size_t)(nsplit * m * n));
    int32_t* S = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nb * n));
    if (!Q || !S) { free(Q); free(S); return -2; }
    int rc = orc_quantize(A, m, n, lda, fmt, nsplit, block_rows, in_f32, Q, S);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < ell; ++i) {
            double y = 0.0;
            for (int64_t b = 0; b < nb; ++b) {
                int64_t r0 = b * block_rows, r1 = r0 + block_rows < m ? r0 + block_rows : m;
                double part = 0.0;
                for (int t = 0; t < nsplit; ++t)
                    for (int64_t l = r0; l < r1; ++l)
                        part += omega[i * m + l] * Q[(int64_t)t * m * n + j * m + l];
                y += ldexp(part, S[j * nb + b]);
            }
            A_(Y, ldy, i, j) = y;
        }
    free(Q); free(S);
    return rc;
}

/* ------------------------------------------------- column-pivoted Householder QR */

static double col_sq(const double* X, int64_t ldx, int64_t r0, int64_t r1, int64_t j)
{
    double s = 0.0;
    for (int64_t t = r0; t < r1; ++t) s += A_(X, ldx, t, j) * A_(X, ldx, t, j);
    return s;
}

/* Truncated column-pivoted Householder QR of W (r x n), Sec. 1.1 (AZ = QR,
 * blocks R11, R12) with the greedy pivot of Businger and Golub.
 *
 * Step j (0-based) selects p = argmax of the residual squared norms nu_i over
 * unselected columns (ties: smallest original index), forms the reflector
 * H = I - tau v v^T with v(0) = 1 that maps x = X(j:r, p) to beta e_1,
 * beta = -sign(alpha) ||x|| (sign(0) = +1), alpha = x(0),
 * v = x / (alpha - beta), tau = (beta - alpha) / beta, applies it to every
 * unselected column and records row j of R: R(j,p) = beta, R(j,i) = X(j,i)
 * for the unselected i.
 *
 * Rank: rel_tol <= 0 runs exactly min(k_req, r, n) steps.  rel_tol > 0 stops
 * before step j when sqrt(sum of unselected nu) <= rel_tol ||W||_F (that sum
 * is ||R22||_F^2), at most min(k_max, r, n) steps.
 *
 * norm_mode 0: nu recomputed exactly from X at every step.
 * norm_mode 1: nu downdated by R(j,i)^2; recomputed exactly when
 *   max(0, 1 - R(j,i)^2/nu_i) * nu_i / nu_ref_i <= sqrt(u), u = 2^-53,
 *   where nu_ref_i is the value at the last exact computation
 *   (Drmac and Bujanovic 2008).
 *
 * Outputs: J[n] (J[0:k] pivots in order, J[k:n] the rest ascending), R with
 * rows 0..k-1 (col-major, ldr >= steps, columns by original index), *k_out,
 * gaps[j] = (nu_1 - nu_2)/nu_1 of the two largest unselected nu at step j
 * (1 if only one column is left).  Returns 0, or j+1 if at step j every
 * unselected nu was zero (the rank is then j; *k_out = j), or -1 for a
 * non-finite input. */
int orc_cpqr(const double* W, int64_t r, int64_t n, int64_t ldw,
             int32_t k_req, double rel_tol, int32_t k_max, int32_t norm_mode,
             int32_t* J, double* R, int64_t ldr, int32_t* k_out, double* gaps)
{
    int64_t cap = (rel_tol > 0.0) ? k_max : k_req;
    if (cap > r) cap = r;
    if (cap > n) cap = n;
    if (cap < 0) cap = 0;
    double* X = (double*)malloc(sizeof(double) * (size_t)(r * n + 1));
    double* nu = (double*)malloc(sizeof(double) * (size_t)(n + 1));
    double* nuref = (double*)malloc(sizeof(double) * (size_t)(n + 1));
    double* v = (double*)malloc(sizeof(double) * (size_t)(r + 1));
    char* sel = (char*)calloc((size_t)n + 1, 1);
    int info = 0;
    double total = 0.0;
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < r; ++i) {
            double a = A_(W, ldw, i, j);
            if (!isfinite(a)) info = -1;
            A_(X, r, i, j) = a;
            total += a * a;
        }
    for (int64_t i = 0; i < n; ++i) { nu[i] = col_sq(X, r, 0, r, i); nuref[i] = nu[i]; }
    const double sqrt_u = sqrt(ldexp(1.0, -53));
    int64_t k = 0;
    if (info == 0)
    for (int64_t j = 0; j < cap; ++j) {
        if (norm_mode == 0)
            for (int64_t i = 0; i < n; ++i) if (!sel[i]) nu[i] = col_sq(X, r, j, r, i);
        if (rel_tol > 0.0) {
            double rest = 0.0;
            for (int64_t i = 0; i < n; ++i) if (!sel[i]) rest += nu[i];
            if (sqrt(rest) <= rel_tol * sqrt(total)) break;
        }
        int64_t p = -1;
        double best = -1.0, second = -1.0;
        for (int64_t i = 0; i < n; ++i) {
            if (sel[i]) continue;
            if (nu[i] > best) { second = best; best = nu[i]; p = i; }
            else if (nu[i] > second) second = nu[i];
        }
        if (gaps) gaps[j] = (second < 0.0 || best <= 0.0) ? 1.0 : (best - second) / best;
        if (p < 0 || best <= 0.0) { info = (int)j + 1; break; }
        /* Householder reflector for x = X(j:r, p) */
        double alpha = A_(X, r, j, p);
        double s = sqrt(col_sq(X, r, j, r, p));
        double beta = (alpha >= 0.0) ? -s : s;
        double tau = (beta - alpha) / beta;
        double denom = alpha - beta;
        v[0] = 1.0;
        for (int64_t t = j + 1; t < r; ++t) v[t - j] = A_(X, r, t, p) / denom;
        sel[p] = 1;
        J[j] = (int32_t)p;
        A_(R, ldr, j, p) = beta;
        for (int64_t i = 0; i < n; ++i) {
            if (sel[i]) continue;
            double w = 0.0;
            for (int64_t t = j; t < r; ++t) w += v[t - j] * A_(X, r, t, i);
            for (int64_t t = j; t < r; ++t) A_(X, r, t, i) -= tau * w * v[t - j];
            double rho = A_(X, r, j, i);
            A_(R, ldr, j, i) = rho;
            if (norm_mode == 1) {
                if (nu[i] > 0.0) {
                    double t1 = 1.0 - rho * rho / nu[i];
                    if (t1 < 0.0) t1 = 0.0;
                    if (t1 * (nu[i] / nuref[i]) <= sqrt_u) {
                        nu[i] = col_sq(X, r, j + 1, r, i);
                        nuref[i] = nu[i];
                    } else {
                        nu[i] = nu[i] * t1;
                    }
                }
            }
        }
        /* earlier pivots keep R(j, J[l]) = 0 for l < j (upper triangular) */
        for (int64_t l = 0; l < j; ++l) A_(R, ldr, j, J[l]) = 0.0;
        k = j + 1;
    }
    int64_t c = k;
    for (int64_t i = 0; i < n; ++i) if (!sel[i]) J[c++] = (int32_t)i;
    *k_out = (int32_t)k;
    free(X); free(nu); free(nuref); free(v); free(sel);
    return info;
}

/* Greedy column selection by modified Gram-Schmidt with column pivoting, the
 * MGSQR of Sec. 1.1 / Algorithm 1, with every projection done twice
 * (reorthogonalised).  Step j picks the unselected column of largest residual
 * norm, normalises it to q_j and removes q_j from every unselected column.
 * Writes J[0:k] and R rows (R(j, i) = q_j^T x_i summed over both passes).
 * Returns 0 or j+1 on a zero pivot. */
int orc_mgs_cpqr(const double* W, int64_t r, int64_t n, int64_t ldw, int32_t k,
                 int32_t* J, double* R, int64_t ldr)
{
    double* X = (double*)malloc(sizeof(double) * (size_t)(r * n + 1));
    double* Qv = (double*)malloc(sizeof(double) * (size_t)(r * (k > 0 ? k : 1) + 1));
    char* sel = (char*)calloc((size_t)n + 1, 1);
    int info = 0;
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < r; ++i) A_(X, r, i, j) = A_(W, ldw, i, j);
    for (int64_t j = 0; j < k; ++j) {
        int64_t p = -1;
        double best = -1.0;
        for (int64_t i = 0; i < n; ++i) {
            if (sel[i]) continue;
            double s = col_sq(X, r, 0, r, i);
            if (s > best) { best = s; p = i; }
        }
        if (p < 0 || best <= 0.0) { info = (int)j + 1; break; }
        double nrm = sqrt(best);
        double* q = Qv + j * r;
        for (int64_t t = 0; t < r; ++t) q[t] = A_(X, r, t, p) / nrm;
        /* reorthogonalise q against earlier q's */
        for (int64_t l = 0; l < j; ++l) {
            double d = 0.0;
            for (int64_t t = 0; t < r; ++t) d += Qv[l * r + t] * q[t];
            for (int64_t t = 0; t < r; ++t) q[t] -= d * Qv[l * r + t];
        }
        double qn = 0.0;
        for (int64_t t = 0; t < r; ++t) qn += q[t] * q[t];
        qn = sqrt(qn);
        for (int64_t t = 0; t < r; ++t) q[t] /= qn;
        sel[p] = 1;
        J[j] = (int32_t)p;
        A_(R, ldr, j, p) = nrm;
        for (int64_t i = 0; i < n; ++i) {
            if (sel[i]) continue;
            double rho = 0.0;
            for (int pass = 0; pass < 2; ++pass) {
                double d = 0.0;
                for (int64_t t = 0; t < r; ++t) d += q[t] * A_(X, r, t, i);
                for (int64_t t = 0; t < r; ++t) A_(X, r, t, i) -= d * q[t];
                rho += d;
            }
            A_(R, ldr, j, i) = rho;
        }
    }
    free(X); free(Qv); free(sel);
    return info;
}

/* T = R11^-1 R12 by back-substitution (Algorithm 1, the coefficient solve; R11 is upper
 * triangular and nonsingular, so its pseudo-inverse is its inverse).
 * R11(a,b) = R(a, J[b]), R12(a,c) = R(a, J[k+c]).  T: k x (n-k) col-major. */
void orc_solve_T(int32_t k, int64_t n, const int32_t* J, const double* R, int64_t ldr,
                 double* T, int64_t ldt)
{
    for (int64_t c = 0; c < n - k; ++c) {
        int32_t jc = J[k + c];
        for (int64_t a = k - 1; a >= 0; --a) {
            double s = A_(R, ldr, a, jc);
            for (int64_t b = a + 1; b < k; ++b) s -= A_(R, ldr, a, J[b]) * A_(T, ldt, b, c);
            A_(T, ldt, a, c) = s / A_(R, ldr, a, J[a]);
        }
    }
}

/* Residual of the ID in the Frobenius norm, squared:
 * ||A(:,Jc) - A(:,J[0:k]) T||_F^2 (the skeleton columns are reproduced
 * exactly, Sec. 1.1). */
double orc_residual_fro2(const double* A, int64_t m, int64_t n, int64_t lda,
                         int32_t k, const int32_t* J, const double* T, int64_t ldt)
{
    double s = 0.0;
    for (int64_t c = 0; c < n - k; ++c)
        for (int64_t i = 0; i < m; ++i) {
            double x = A_(A, lda, i, J[k + c]);
            for (int64_t b = 0; b < k; ++b) x -= A_(A, lda, i, J[b]) * A_(T, ldt, b, c);
            s += x * x;
        }
    return s;
}

/* Full oracle ID (Algorithm 1, with the optional sketch first):
 * W = Omega A when omega != NULL (ell rows), else W = A; truncated CPQR of W;
 * T = R11^-1 R12.  T is written k_cap x (n - k) col-major with ldt.
 * Returns the CPQR info. */
int orc_id(const double* A, int64_t m, int64_t n, int64_t lda,
           const double* omega, int64_t ell,
           int32_t k_req, double rel_tol, int32_t k_max, int32_t norm_mode,
           int32_t* J, double* T, int64_t ldt, int32_t* k_out, double* gaps)
{
    const double* W = A;
    int64_t r = m, ldw = lda;
    double* Y = NULL;
    if (omega) {
        Y = (double*)malloc(sizeof(double) * (size_t)(ell * n + 1));
        orc_sketch_f64(omega, ell, m, A, lda, n, Y, ell);
        W = Y; r = ell; ldw = ell;
    }
    int64_t cap = (rel_tol > 0.0) ? k_max : k_req;
    if (cap > r) cap = r;
    if (cap > n) cap = n;
    if (cap < 1) cap = 1;
    double* R = (double*)calloc((size_t)(cap * n + 1), sizeof(double));
    int info = orc_cpqr(W, r, n, ldw, k_req, rel_tol, k_max, norm_mode, J, R, cap, k_out, gaps);
    if (info >= 0 && *k_out > 0) orc_solve_T(*k_out, n, J, R, cap, T, ldt);
    free(R); free(Y);
    return info;
}
