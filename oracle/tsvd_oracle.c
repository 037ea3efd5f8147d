/*
 * tsvd_oracle.c -- plain, slow, single-threaded CPU oracle for the mixed
 * precision Gram-matrix thin SVD (Carson, Ma, Shao: "Mixed precision thin SVD
 * algorithms based on the Gram matrix", arXiv 2603.11953).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA path; it exists to judge that path.
 *
 * What it computes, step by step (Algorithm 1 of the paper):
 *   Alg. 1 lines 1-2  M_h = A^T A at a precision strictly higher than any the
 *                     GPU uses: every product a_ri*a_rj is formed exactly (as
 *                     a 106-bit integer times a power of two) and summed
 *                     exactly in a fixed-point superaccumulator, then rounded
 *                     once (to FP64, and to a double-double hi+lo pair).
 *   Alg. 1 line 3     spectral decomposition of M_h by the two-sided cyclic
 *                     Jacobi method (Section 2.1: the paper's recommended
 *                     eigensolver, Remark 1), row-cyclic order, Rutishauser's
 *                     rotation formulas, in FP64 or in double-double.
 *   Alg. 1 lines 4-5  sigma = sqrt(lambda) sorted descending; V permuted and
 *                     sign-normalised; both rounded (RN-even) to working,
 *                     once, from the exact value of the (hi, lo) pair.
 *   Alg. 1 line 6     U = A (V Sigma^{-1}): W = RN_w(V_w / sigma_w) and every
 *                     entry of A*W summed exactly then rounded once.
 *
 * Readings of points the paper leaves open:
 *   - the Jacobi skip test is |m_pq| <= tol * sqrt(m_pp * m_qq) (scaled by the
 *     column norms D of A = B D, Section 3); zeta = 0 takes sgn = +1;
 *   - sweeps stop after a sweep with no rotation; failure after max_sweeps;
 *   - lambda_i <= 0 is "not full rank" (the paper assumes full column rank);
 *   - signs: the largest-magnitude entry of each V column is made positive
 *     (lowest row index wins ties); ties in sigma keep the original order.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no fast-math: the
 * double-double and rounding code depends on IEEE semantics).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_NOT_FULL_RANK 1
#define ORC_NO_CONVERGENCE 2
#define ORC_BAD_ARG 3
#define ORC_NONFINITE 4

/* ------------------------------------------------------------------------- */
/* Superaccumulator: an exact fixed-point sum of signed dyadic numbers.      */
/* Value = sum_k limb[k] * 2^(32k + SA_BASE).  Limbs below the top one are   */
/* kept in [0, 2^32) after normalisation; the top limb holds the sign (0 or  */
/* -1).  Between normalisations limbs absorb raw 32-bit pieces as int64.      */
/* Range: products of two doubles have exponents in [-2148, 1942] and        */
/* mantissas below 2^106; sums of up to 2^64 of them stay below 2^2112.       */
/* ------------------------------------------------------------------------- */
#define SA_LIMBS 140
#define SA_BASE (-2240)
#define SA_RENORM_EVERY (1 << 26)

typedef struct {
    int64_t limb[SA_LIMBS];
    int64_t pending;
} superacc;

static void sa_clear(superacc* s) { memset(s, 0, sizeof(*s)); }

static void sa_normalize(superacc* s) {
    int64_t carry = 0;
    for (int k = 0; k < SA_LIMBS - 1; ++k) {
        int64_t v = s->limb[k] + carry;
        carry = v >> 32; /* arithmetic shift = floor(v / 2^32) */
        s->limb[k] = v - carry * ((int64_t)1 << 32);
    }
    s->limb[SA_LIMBS - 1] += carry;
    s->pending = 0;
}

/* Add sign * mant * 2^e exactly (mant < 2^106). */
static void sa_add_int(superacc* s, int negative, unsigned __int128 mant, int e) {
    if (mant == 0) return;
    int o = e - SA_BASE;
    if (o < 0) abort(); /* outside the designed range: cannot happen for finite doubles */
    int k = o >> 5, sh = o & 31;
    for (int piece = 0; piece < 4; ++piece) {
        uint64_t p = (uint64_t)(mant >> (32 * piece)) & 0xffffffffull;
        if (p == 0) continue;
        uint64_t w = p << sh; /* < 2^63 */
        int64_t lo = (int64_t)(w & 0xffffffffull), hi = (int64_t)(w >> 32);
        if (k + piece + 1 >= SA_LIMBS) abort();
        if (negative) {
            s->limb[k + piece] -= lo;
            s->limb[k + piece + 1] -= hi;
        } else {
            s->limb[k + piece] += lo;
            s->limb[k + piece + 1] += hi;
        }
    }
    if (++s->pending >= SA_RENORM_EVERY) sa_normalize(s);
}

/* x = M * 2^e with M an integer below 2^53 (x finite). */
static void split_double(double x, int* neg, uint64_t* M, int* e) {
    int ex;
    double f = frexp(fabs(x), &ex); /* f in [0.5, 1) */
    *neg = signbit(x) ? 1 : 0;
    *M = (uint64_t)ldexp(f, 53); /* exact: f has at most 53 significant bits */
    *e = ex - 53;
}

static void sa_add_product(superacc* s, double x, double y) {
    if (x == 0.0 || y == 0.0) return;
    int nx, ny, ex, ey;
    uint64_t mx, my;
    split_double(x, &nx, &mx, &ex);
    split_double(y, &ny, &my, &ey);
    sa_add_int(s, nx ^ ny, (unsigned __int128)mx * my, ex + ey);
}

static void sa_add_double(superacc* s, double x) {
    if (x == 0.0) return;
    int nx, ex;
    uint64_t mx;
    split_double(x, &nx, &mx, &ex);
    sa_add_int(s, nx, mx, ex);
}

static int sa_bit(const superacc* s, long i) {
    if (i < 0) return 0;
    return (int)((s->limb[i >> 5] >> (i & 31)) & 1);
}

/* Round the exact sum to the nearest (ties to even) binary number with p
 * significant bits, returned as a double (p <= 53).  No overflow/underflow
 * handling is needed for the workloads (results stay far inside the normal
 * range); the function aborts rather than return a wrong value if not. */
static double sa_round(superacc* s, int p) {
    sa_normalize(s);
    superacc mag = *s;
    int negative = 0;
    if (mag.limb[SA_LIMBS - 1] < 0) {
        negative = 1;
        for (int k = 0; k < SA_LIMBS; ++k) mag.limb[k] = -mag.limb[k];
        sa_normalize(&mag);
    }
    if (mag.limb[SA_LIMBS - 1] != 0) abort();
    int top = -1;
    for (int k = SA_LIMBS - 2; k >= 0; --k)
        if (mag.limb[k] != 0) { top = k; break; }
    if (top < 0) return 0.0;
    int b = 31;
    while (((mag.limb[top] >> b) & 1) == 0) --b;
    long msb = (long)top * 32 + b;           /* bit index of the leading 1 */
    long lsb = msb - p + 1;                  /* bit index of the last kept bit */
    uint64_t mant = 0;
    for (long i = msb; i >= lsb; --i) mant = (mant << 1) | (uint64_t)sa_bit(&mag, i);
    int round_bit = sa_bit(&mag, lsb - 1);
    int sticky = 0;
    if (lsb - 1 > 0) {
        long below = lsb - 2; /* highest bit index that feeds the sticky bit */
        long kb = below >> 5;
        uint64_t mask = (below & 31) == 31 ? 0xffffffffull : ((1ull << ((below & 31) + 1)) - 1);
        if ((uint64_t)mag.limb[kb] & mask) sticky = 1;
        for (long k = kb - 1; k >= 0 && !sticky; --k)
            if (mag.limb[k] != 0) sticky = 1;
    }
    if (round_bit && (sticky || (mant & 1))) {
        mant += 1;
        if (mant == (1ull << p)) { mant >>= 1; lsb += 1; }
    }
    long e2 = lsb + SA_BASE;
    if (e2 < -1000 || e2 > 960) abort();
    double v = ldexp((double)mant, (int)e2);
    return negative ? -v : v;
}

/* RN-even of the exact value hi + lo to p significant bits (p <= 53), by one
 * rounding of the exact sum (no intermediate rounding to FP64).  This is the
 * cast of Alg. 1 lines 4-5 from the higher precision to the working one. */
static double round_dd_exact(superacc* s, double hi, double lo, int p) {
    sa_clear(s);
    sa_add_double(s, hi);
    sa_add_double(s, lo);
    return sa_round(s, p);
}

int oracle_round_dd(const double* hi, const double* lo, int64_t count, int p, double* out) {
    if (!hi || !out || count < 0 || p < 2 || p > 53) return ORC_BAD_ARG;
    superacc* s = (superacc*)malloc(sizeof(superacc));
    if (!s) return ORC_BAD_ARG;
    for (int64_t k = 0; k < count; ++k) out[k] = round_dd_exact(s, hi[k], lo ? lo[k] : 0.0, p);
    free(s);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Working-precision element access.                                          */
/* ------------------------------------------------------------------------- */
static double elem(const void* A, int working, int64_t lda, int64_t r, int64_t c) {
    if (working == 0) return (double)((const float*)A)[r + c * lda];
    return ((const double*)A)[r + c * lda];
}

/* ------------------------------------------------------------------------- */
/* Alg. 1 lines 1-2: exact Gram matrix.                                        */
/* G_hi = RN_64(S), G_lo = RN_64(S - G_hi) (a double-double), G_abs =          */
/* (|A|^T |A|) in FP64 (tolerance denominators of eq. (ATA)).  Full n x n,    */
/* column-major with leading dimension n.  Any output pointer may be NULL.    */
/* ------------------------------------------------------------------------- */
int oracle_gram(const void* A, int64_t m, int64_t n, int64_t lda, int working,
                double* G_hi, double* G_lo, double* G_abs) {
    if (!A || m < 0 || n < 1 || lda < (m > 1 ? m : 1) || (working != 0 && working != 1)) return ORC_BAD_ARG;
    for (int64_t c = 0; c < n; ++c)
        for (int64_t r = 0; r < m; ++r)
            if (!isfinite(elem(A, working, lda, r, c))) return ORC_NONFINITE;
    superacc* s = (superacc*)malloc(sizeof(superacc));
    if (!s) return ORC_BAD_ARG;
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t i = 0; i <= j; ++i) {
            sa_clear(s);
            double absum = 0.0;
            for (int64_t r = 0; r < m; ++r) {
                double x = elem(A, working, lda, r, i), y = elem(A, working, lda, r, j);
                sa_add_product(s, x, y);
                absum += fabs(x) * fabs(y);
            }
            double hi = sa_round(s, 53);
            double lo = 0.0;
            if (G_lo) {
                sa_add_double(s, -hi);
                lo = sa_round(s, 53);
            }
            if (G_hi) { G_hi[i + j * n] = hi; G_hi[j + i * n] = hi; }
            if (G_lo) { G_lo[i + j * n] = lo; G_lo[j + i * n] = lo; }
            if (G_abs) { G_abs[i + j * n] = absum; G_abs[j + i * n] = absum; }
        }
    }
    free(s);
    return ORC_OK;
}

/* Exact dot products of selected rows of A with the columns of a matrix W
 * (n x n, column-major, leading dimension ldw, given as doubles), each
 * rounded once to p bits: out[k + j*nrows] = RN_p(sum_c A[rows[k], c] W[c, j]).
 * This is U = A W of Alg. 1 line 6 with W = V Sigma^{-1} supplied by the
 * caller (p = 24 for FP32 working, 53 for FP64 working). */
int oracle_rows_times(const void* A, int64_t m, int64_t n, int64_t lda, int working,
                      const double* W, int64_t ldw, const int64_t* rows, int64_t nrows,
                      int p, double* out) {
    if (!A || !W || !rows || !out || n < 1 || ldw < n || p < 2 || p > 53) return ORC_BAD_ARG;
    superacc* s = (superacc*)malloc(sizeof(superacc));
    if (!s) return ORC_BAD_ARG;
    for (int64_t k = 0; k < nrows; ++k) {
        int64_t r = rows[k];
        if (r < 0 || r >= m) { free(s); return ORC_BAD_ARG; }
        for (int64_t j = 0; j < n; ++j) {
            sa_clear(s);
            for (int64_t c = 0; c < n; ++c) sa_add_product(s, elem(A, working, lda, r, c), W[c + j * ldw]);
            out[k + j * nrows] = sa_round(s, p);
        }
    }
    free(s);
    return ORC_OK;
}

/* Same, summing in double-double-free exact arithmetic but with a second
 * factor: out = RN_p( (sum_c A[r,c] V[c,j]) / sigma_j ) where the division is
 * done on the exactly rounded-to-DD dot.  This is the "explicit U" of
 * A V_h Sigma_h^{-1} with the higher-precision V_h and sigma_h. */
typedef struct { double hi, lo; } dd;
static dd dd_from_sa(superacc* s) {
    dd r;
    r.hi = sa_round(s, 53);
    sa_add_double(s, -r.hi);
    r.lo = sa_round(s, 53);
    return r;
}

/* ------------------------------------------------------------------------- */
/* Double-double arithmetic (Dekker 1971; Knuth's TwoSum), written from the  */
/* published error-free transformations.                                       */
/* ------------------------------------------------------------------------- */
static dd two_sum(double a, double b) {
    double s = a + b, bb = s - a;
    dd r = {s, (a - (s - bb)) + (b - bb)};
    return r;
}
static dd fast_two_sum(double a, double b) { /* |a| >= |b| or a == 0 */
    double s = a + b;
    dd r = {s, b - (s - a)};
    return r;
}
static dd two_prod(double a, double b) {
    double p = a * b;
    dd r = {p, fma(a, b, -p)};
    return r;
}
static dd dd_make(double x) { dd r = {x, 0.0}; return r; }
static dd dd_neg(dd a) { dd r = {-a.hi, -a.lo}; return r; }
static dd dd_add(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi), t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}
static dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
static dd dd_mul(dd a, dd b) {
    dd p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return fast_two_sum(p.hi, p.lo);
}
static dd dd_div(dd a, dd b) {
    double q1 = a.hi / b.hi;
    dd r = dd_sub(a, dd_mul(b, dd_make(q1)));
    double q2 = r.hi / b.hi;
    r = dd_sub(r, dd_mul(b, dd_make(q2)));
    double q3 = r.hi / b.hi;
    dd q = fast_two_sum(q1, q2);
    return dd_add(q, dd_make(q3));
}
static dd dd_sqrt(dd a) { /* one Newton step from the FP64 root doubles its accuracy */
    if (a.hi <= 0.0) return dd_make(0.0);
    double x = sqrt(a.hi);
    dd xx = two_prod(x, x);
    dd resid = dd_sub(a, xx);
    double corr = resid.hi / (2.0 * x);
    return fast_two_sum(x, corr);
}
static double dd_abs_hi(dd a) { return fabs(a.hi); }
static int dd_lt(dd a, dd b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

int oracle_rows_explicit_u(const void* A, int64_t m, int64_t n, int64_t lda, int working,
                           const double* V_hi, const double* V_lo, const double* sig_hi,
                           const double* sig_lo, const int64_t* rows, int64_t nrows, double* out_hi,
                           double* out_lo) {
    if (!A || !V_hi || !sig_hi || !rows || !out_hi || n < 1) return ORC_BAD_ARG;
    superacc* s = (superacc*)malloc(sizeof(superacc));
    if (!s) return ORC_BAD_ARG;
    for (int64_t k = 0; k < nrows; ++k) {
        int64_t r = rows[k];
        if (r < 0 || r >= m) { free(s); return ORC_BAD_ARG; }
        for (int64_t j = 0; j < n; ++j) {
            sa_clear(s);
            for (int64_t c = 0; c < n; ++c) {
                double a = elem(A, working, lda, r, c);
                sa_add_product(s, a, V_hi[c + j * n]);
                if (V_lo) sa_add_product(s, a, V_lo[c + j * n]);
            }
            dd dot = dd_from_sa(s);
            dd sg = {sig_hi[j], sig_lo ? sig_lo[j] : 0.0};
            dd u = dd_div(dot, sg);
            out_hi[k + j * nrows] = u.hi;
            if (out_lo) out_lo[k + j * nrows] = u.lo;
        }
    }
    free(s);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Alg. 1 line 3: two-sided cyclic Jacobi (Section 2.1, Remark 1).            */
/* For each pair p < q in row-cyclic order: skip if m_pq = 0 or                */
/* |m_pq| <= tol*sqrt(m_pp m_qq); otherwise rotate with                        */
/*   zeta = (m_qq - m_pp) / (2 m_pq),  t = sgn(zeta) / (|zeta| + sqrt(1+zeta^2)),
 *   c = 1/sqrt(1+t^2),  s = t c,                                              */
/* M <- J^T M J, V <- V J, with J = I except J_pp = J_qq = c, J_pq = s,        */
/* J_qp = -s; then m_pp -= t m_pq, m_qq += t m_pq, m_pq = m_qp = 0.            */
/* Stop after a sweep with no rotation.                                        */
/* ------------------------------------------------------------------------- */
int oracle_jacobi_fp64(double* M, int n, double tol, int max_sweeps, double* lam, double* V,
                       int* sweeps_out) {
    if (!M || !lam || !V || n < 1 || max_sweeps < 1) return ORC_BAD_ARG;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) V[i + j * n] = (i == j) ? 1.0 : 0.0;
    int sweep = 0, converged = 0;
    while (sweep < max_sweeps) {
        ++sweep;
        int rotations = 0;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double mpq = M[p + q * n], mpp = M[p + p * n], mqq = M[q + q * n];
                if (mpq == 0.0) continue;
                if (fabs(mpq) <= tol * sqrt(fabs(mpp * mqq))) continue;
                double zeta = (mqq - mpp) / (2.0 * mpq);
                double sg = (zeta >= 0.0) ? 1.0 : -1.0;
                double t = sg / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t);
                double s = t * c;
                for (int r = 0; r < n; ++r) { /* columns p, q: M <- M J */
                    if (r == p || r == q) continue;
                    double xp = M[r + p * n], xq = M[r + q * n];
                    M[r + p * n] = c * xp - s * xq;
                    M[r + q * n] = s * xp + c * xq;
                }
                for (int r = 0; r < n; ++r) { /* rows p, q: M <- J^T M (symmetric copy) */
                    if (r == p || r == q) continue;
                    M[p + r * n] = M[r + p * n];
                    M[q + r * n] = M[r + q * n];
                }
                M[p + p * n] = mpp - t * mpq;
                M[q + q * n] = mqq + t * mpq;
                M[p + q * n] = 0.0;
                M[q + p * n] = 0.0;
                for (int r = 0; r < n; ++r) {
                    double vp = V[r + p * n], vq = V[r + q * n];
                    V[r + p * n] = c * vp - s * vq;
                    V[r + q * n] = s * vp + c * vq;
                }
                ++rotations;
            }
        }
        if (rotations == 0) { converged = 1; break; }
    }
    for (int i = 0; i < n; ++i) lam[i] = M[i + i * n];
    if (sweeps_out) *sweeps_out = sweep;
    return converged ? ORC_OK : ORC_NO_CONVERGENCE;
}

/* The same method carried out in double-double (for FP64 working precision,
 * where the higher precision u_h must lie well below 2^-53).  Matrices are
 * given as (hi, lo) pairs, column-major n x n. */
int oracle_jacobi_dd(double* M_hi, double* M_lo, int n, double tol, int max_sweeps, double* lam_hi,
                     double* lam_lo, double* V_hi, double* V_lo, int* sweeps_out) {
    if (!M_hi || !M_lo || !lam_hi || !lam_lo || !V_hi || !V_lo || n < 1 || max_sweeps < 1) return ORC_BAD_ARG;
    dd* M = (dd*)malloc(sizeof(dd) * (size_t)n * n);
    dd* V = (dd*)malloc(sizeof(dd) * (size_t)n * n);
    if (!M || !V) { free(M); free(V); return ORC_BAD_ARG; }
    for (int k = 0; k < n * n; ++k) {
        M[k] = fast_two_sum(M_hi[k], M_lo[k]);
        V[k] = dd_make((k % n) == (k / n) ? 1.0 : 0.0);
    }
    const dd one = dd_make(1.0), two = dd_make(2.0);
    int sweep = 0, converged = 0;
    while (sweep < max_sweeps) {
        ++sweep;
        int rotations = 0;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                dd mpq = M[p + q * n], mpp = M[p + p * n], mqq = M[q + q * n];
                if (mpq.hi == 0.0) continue;
                dd scale = dd_sqrt(dd_mul(mpp, mqq));
                if (dd_abs_hi(mpq) <= tol * scale.hi) continue;
                dd zeta = dd_div(dd_sub(mqq, mpp), dd_mul(two, mpq));
                dd az = zeta.hi < 0.0 ? dd_neg(zeta) : zeta;
                dd t = dd_div(one, dd_add(az, dd_sqrt(dd_add(one, dd_mul(zeta, zeta)))));
                if (zeta.hi < 0.0) t = dd_neg(t);
                dd c = dd_div(one, dd_sqrt(dd_add(one, dd_mul(t, t))));
                dd s = dd_mul(t, c);
                for (int r = 0; r < n; ++r) {
                    if (r == p || r == q) continue;
                    dd xp = M[r + p * n], xq = M[r + q * n];
                    M[r + p * n] = dd_sub(dd_mul(c, xp), dd_mul(s, xq));
                    M[r + q * n] = dd_add(dd_mul(s, xp), dd_mul(c, xq));
                    M[p + r * n] = M[r + p * n];
                    M[q + r * n] = M[r + q * n];
                }
                M[p + p * n] = dd_sub(mpp, dd_mul(t, mpq));
                M[q + q * n] = dd_add(mqq, dd_mul(t, mpq));
                M[p + q * n] = dd_make(0.0);
                M[q + p * n] = dd_make(0.0);
                for (int r = 0; r < n; ++r) {
                    dd vp = V[r + p * n], vq = V[r + q * n];
                    V[r + p * n] = dd_sub(dd_mul(c, vp), dd_mul(s, vq));
                    V[r + q * n] = dd_add(dd_mul(s, vp), dd_mul(c, vq));
                }
                ++rotations;
            }
        }
        if (rotations == 0) { converged = 1; break; }
    }
    for (int i = 0; i < n; ++i) { lam_hi[i] = M[i + i * n].hi; lam_lo[i] = M[i + i * n].lo; }
    for (int k = 0; k < n * n; ++k) { V_hi[k] = V[k].hi; V_lo[k] = V[k].lo; M_hi[k] = M[k].hi; M_lo[k] = M[k].lo; }
    if (sweeps_out) *sweeps_out = sweep;
    free(M);
    free(V);
    return converged ? ORC_OK : ORC_NO_CONVERGENCE;
}

/* ------------------------------------------------------------------------- */
/* Alg. 1 lines 3-5: sigma = sqrt(lambda), descending order, sign rule.       */
/* Inputs lam (hi, lo) and V (hi, lo) from the Jacobi (lo may be NULL).       */
/* Outputs overwrite them in place: sigma sorted descending, V permuted and    */
/* each column negated if its largest-magnitude entry is negative.            */
/* ------------------------------------------------------------------------- */
int oracle_sort_sign(int n, double* lam_hi, double* lam_lo, double* V_hi, double* V_lo,
                     double* sig_hi, double* sig_lo) {
    if (n < 1 || !lam_hi || !V_hi || !sig_hi) return ORC_BAD_ARG;
    int* order = (int*)malloc(sizeof(int) * n);
    double* tmp = (double*)malloc(sizeof(double) * (size_t)n * n * 2);
    if (!order || !tmp) { free(order); free(tmp); return ORC_BAD_ARG; }
    for (int i = 0; i < n; ++i) order[i] = i;
    /* stable insertion sort, descending by lambda (hi, then lo) */
    for (int i = 1; i < n; ++i) {
        int k = order[i], j = i - 1;
        dd lk = {lam_hi[k], lam_lo ? lam_lo[k] : 0.0};
        while (j >= 0) {
            dd lj = {lam_hi[order[j]], lam_lo ? lam_lo[order[j]] : 0.0};
            if (!dd_lt(lj, lk)) break;
            order[j + 1] = order[j];
            --j;
        }
        order[j + 1] = k;
    }
    int status = ORC_OK;
    for (int i = 0; i < n; ++i) if (lam_hi[i] <= 0.0) status = ORC_NOT_FULL_RANK;
    double* lh = tmp;           /* scratch reuse: first n entries */
    double* ll = tmp + n;
    for (int i = 0; i < n; ++i) { lh[i] = lam_hi[order[i]]; ll[i] = lam_lo ? lam_lo[order[i]] : 0.0; }
    for (int i = 0; i < n; ++i) { lam_hi[i] = lh[i]; if (lam_lo) lam_lo[i] = ll[i]; }
    for (int i = 0; i < n; ++i) {
        dd l = {lam_hi[i], lam_lo ? lam_lo[i] : 0.0};
        dd sg = l.hi > 0.0 ? dd_sqrt(l) : dd_make(0.0);
        sig_hi[i] = sg.hi;
        if (sig_lo) sig_lo[i] = sg.lo;
    }
    double* Vh = tmp;
    double* Vl = tmp + (size_t)n * n;
    for (int j = 0; j < n; ++j)
        for (int r = 0; r < n; ++r) {
            Vh[r + j * n] = V_hi[r + order[j] * n];
            Vl[r + j * n] = V_lo ? V_lo[r + order[j] * n] : 0.0;
        }
    for (int j = 0; j < n; ++j) {
        int best = 0;
        for (int r = 1; r < n; ++r) {
            dd a = {fabs(Vh[r + j * n]), Vh[r + j * n] < 0 ? -Vl[r + j * n] : Vl[r + j * n]};
            dd b = {fabs(Vh[best + j * n]), Vh[best + j * n] < 0 ? -Vl[best + j * n] : Vl[best + j * n]};
            if (dd_lt(b, a)) best = r;
        }
        double f = Vh[best + j * n] < 0.0 ? -1.0 : 1.0;
        for (int r = 0; r < n; ++r) {
            V_hi[r + j * n] = f * Vh[r + j * n];
            if (V_lo) V_lo[r + j * n] = f * Vl[r + j * n];
        }
    }
    free(order);
    free(tmp);
    return status;
}

/* ------------------------------------------------------------------------- */
/* Whole pipeline of Algorithm 1 for one matrix.                               */
/*   working: 0 = FP32, 1 = FP64.  higher: 1 = FP64 Gram + FP64 Jacobi,        */
/*   2 = double-double Gram + double-double Jacobi.                           */
/* Outputs (n or n*n doubles; *_lo may be NULL):                               */
/*   sig_hi/lo, V_hi/lo  : higher-precision sigma_h and V_h (sorted, signed)   */
/*   sig_w, V_w          : RN to working precision (stored as doubles)          */
/*   W_w                 : RN_w(V_w(:,j) / sig_w(j))  (the operand of line 6)  */
/*   G_hi/lo             : the exact Gram, rounded (may be NULL)               */
/* Returns the status; *sweeps = Jacobi sweeps used.                           */
/* ------------------------------------------------------------------------- */
int oracle_svd(const void* A, int64_t m, int64_t n, int64_t lda, int working, int higher,
               double tol, int max_sweeps, double* sig_hi, double* sig_lo, double* V_hi,
               double* V_lo, double* sig_w, double* V_w, double* W_w, int* sweeps) {
    if (n < 1 || m < n || (higher != 1 && higher != 2)) return ORC_BAD_ARG;
    size_t nn = (size_t)n * n;
    double* Gh = (double*)malloc(sizeof(double) * nn);
    double* Gl = (double*)malloc(sizeof(double) * nn);
    double* lh = (double*)malloc(sizeof(double) * n);
    double* ll = (double*)malloc(sizeof(double) * n);
    double* Vh = (double*)malloc(sizeof(double) * nn);
    double* Vl = (double*)malloc(sizeof(double) * nn);
    if (!Gh || !Gl || !lh || !ll || !Vh || !Vl) return ORC_BAD_ARG;
    int st = oracle_gram(A, m, n, lda, working, Gh, Gl, NULL);
    int sw = 0;
    if (st == ORC_OK) {
        if (higher == 1) {
            st = oracle_jacobi_fp64(Gh, (int)n, tol, max_sweeps, lh, Vh, &sw);
            for (int64_t i = 0; i < n; ++i) ll[i] = 0.0;
            for (size_t k = 0; k < nn; ++k) Vl[k] = 0.0;
        } else {
            st = oracle_jacobi_dd(Gh, Gl, (int)n, tol, max_sweeps, lh, ll, Vh, Vl, &sw);
        }
    }
    if (st == ORC_OK || st == ORC_NO_CONVERGENCE) {
        int st2 = oracle_sort_sign((int)n, lh, ll, Vh, Vl, sig_hi, sig_lo);
        if (st == ORC_OK) st = st2;
        /* Alg. 1 lines 4-5: one RN-even rounding of the exact (hi, lo) value to the working
         * precision's p bits */
        const int p = working == 0 ? 24 : 53;
        superacc* sa = (superacc*)malloc(sizeof(superacc));
        if (!sa) return ORC_BAD_ARG;
        for (int64_t i = 0; i < n; ++i) sig_w[i] = round_dd_exact(sa, sig_hi[i], sig_lo ? sig_lo[i] : 0.0, p);
        for (size_t k = 0; k < nn; ++k) {
            V_w[k] = round_dd_exact(sa, Vh[k], Vl[k], p);
            if (V_hi) V_hi[k] = Vh[k];
            if (V_lo) V_lo[k] = Vl[k];
        }
        free(sa);
        /* W = RN_w(V_w / sigma_w), the IEEE division in working precision.  For FP32 the
         * quotient is formed in FP64 and rounded to FP32: with 53 >= 2*24 + 2 bits that double
         * rounding equals the correctly rounded FP32 quotient (the classical result on
         * innocuous double rounding for +, -, *, / and sqrt). */
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = 0; i < n; ++i) {
                double q = V_w[i + j * n] / sig_w[j];
                W_w[i + j * n] = working == 0 ? (double)(float)q : q;
            }
    }
    if (sweeps) *sweeps = sw;
    free(Gh); free(Gl); free(lh); free(ll); free(Vh); free(Vl);
    return st;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 2 (the mixed precision eigensolver for the Gram matrix), in the  */
/* paper's order, on a given M_h (n x n, column-major, ld n):                 */
/*   line 1  Cholesky M_h = R_h^T R_h at the higher precision (FP64; R_h upper */
/*           triangular, no pivoting: the algorithm names none);              */
/*   line 2  R = RN_w(R_h), the working precision (FP32 for working = 0);     */
/*   line 3  SVD of R: R = U_R Sigma V^T, so that M_h ~= V Sigma^2 V^T.  The   */
/*           oracle takes this SVD of the working-precision R to FP64         */
/*           accuracy: one-sided cyclic Jacobi (row-cyclic pairs, the scaled   */
/*           skip test with tol >= n 2^-53, the rounding level of a recomputed  */
/*           x_p^T x_q; Rutishauser's rotation) on the columns of R, with the  */
/*           rotations accumulated: R J = U_R Sigma, V = J.  The columns of R  */
/*           carry the column scaling D of A = B D (R = R_C D with R_C^T R_C  */
/*           = C), which one-sided Jacobi on columns resolves to relative       */
/*           accuracy.                                                        */
/* Outputs sigma (descending) and V (sign rule) in FP64.  Returns ORC_OK,     */
/* ORC_NOT_FULL_RANK (a non-positive Cholesky pivot) or ORC_NO_CONVERGENCE.   */
/* ------------------------------------------------------------------------- */
int oracle_alg2(const double* M, int n, int working, double tol, int max_sweeps, double* sigma, double* V,
                int* sweeps_out) {
    if (!M || !sigma || !V || n < 1 || max_sweeps < 1 || (working != 0 && working != 1)) return ORC_BAD_ARG;
    double* Rm = (double*)calloc((size_t)n * n, sizeof(double)); /* R, column-major: R[i + j n], i <= j */
    double* X = (double*)malloc(sizeof(double) * (size_t)n * n);  /* X = R (cast), then R J */
    double* lam = (double*)malloc(sizeof(double) * n);
    if (!Rm || !X || !lam) { free(Rm); free(X); free(lam); return ORC_BAD_ARG; }
    int status = ORC_OK;
    /* line 1: r_jj = sqrt(m_jj - sum_k r_kj^2), r_ji = (m_ji - sum_k r_kj r_ki) / r_jj (i > j) */
    for (int j = 0; j < n && status == ORC_OK; ++j) {
        double d = M[j + (size_t)j * n];
        for (int k = 0; k < j; ++k) d -= Rm[k + (size_t)j * n] * Rm[k + (size_t)j * n];
        if (!(d > 0.0)) { status = ORC_NOT_FULL_RANK; break; }
        const double rjj = sqrt(d);
        Rm[j + (size_t)j * n] = rjj;
        for (int i = j + 1; i < n; ++i) {
            double s = M[j + (size_t)i * n];
            for (int k = 0; k < j; ++k) s -= Rm[k + (size_t)j * n] * Rm[k + (size_t)i * n];
            Rm[j + (size_t)i * n] = s / rjj;
        }
    }
    int sweep = 0, converged = 0;
    if (status == ORC_OK) {
        /* line 2: the cast; X = R, V = I */
        for (int c = 0; c < n; ++c)
            for (int r = 0; r < n; ++r) {
                const double v = Rm[r + (size_t)c * n];
                X[r + (size_t)c * n] = working == 0 ? (double)(float)v : v;
                V[r + (size_t)c * n] = r == c ? 1.0 : 0.0;
            }
        /* line 3: one-sided Jacobi on the columns of X, V <- V J */
        while (sweep < max_sweeps) {
            ++sweep;
            int rotations = 0;
            for (int p = 0; p < n - 1; ++p)
                for (int q = p + 1; q < n; ++q) {
                    double* xp = X + (size_t)p * n;
                    double* xq = X + (size_t)q * n;
                    double g = 0.0, a = 0.0, b = 0.0;
                    for (int r = 0; r < n; ++r) { g += xp[r] * xq[r]; a += xp[r] * xp[r]; b += xq[r] * xq[r]; }
                    if (g == 0.0 || fabs(g) <= tol * sqrt(a * b)) continue;
                    const double zeta = (b - a) / (2.0 * g);
                    const double sg = zeta >= 0.0 ? 1.0 : -1.0;
                    const double t = sg / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                    const double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
                    double* vp = V + (size_t)p * n;
                    double* vq = V + (size_t)q * n;
                    for (int r = 0; r < n; ++r) {
                        const double u = xp[r], v = xq[r];
                        xp[r] = cs * u - sn * v;
                        xq[r] = sn * u + cs * v;
                        const double s_ = vp[r], t_ = vq[r];
                        vp[r] = cs * s_ - sn * t_;
                        vq[r] = sn * s_ + cs * t_;
                    }
                    ++rotations;
                }
            if (rotations == 0) { converged = 1; break; }
        }
        for (int j = 0; j < n; ++j) {
            double s2 = 0.0;
            for (int r = 0; r < n; ++r) s2 += X[r + (size_t)j * n] * X[r + (size_t)j * n];
            lam[j] = s2;
        }
        int st2 = oracle_sort_sign(n, lam, NULL, V, NULL, sigma, NULL);
        if (st2 != ORC_OK) status = st2;
        if (status == ORC_OK && !converged) status = ORC_NO_CONVERGENCE;
    }
    if (sweeps_out) *sweeps_out = sweep;
    free(Rm);
    free(X);
    free(lam);
    return status;
}

/* ------------------------------------------------------------------------- */
/* Mixed precision Cholesky QR (Sec. 3.1: the Gram matrix at the higher        */
/* precision, its Cholesky factorization at the higher precision, then Q from  */
/* the linear systems Q R = A at the working precision).                      */
/*   oracle_cholesky: R upper triangular with M = R^T R, plain FP64 (no        */
/*     pivoting), column-major n x n, zeros below the diagonal.               */
/*   oracle_cholqr_rows: for the given rows, q = a R_w^-1 (R_w the factor     */
/*     given, normally RN_w(R)) by forward substitution in double-double      */
/*     (q_j = (a_j - sum_{k<j} q_k r_kj) / r_jj), each entry then rounded once */
/*     to p bits: the exact solution to ~2^-100, rounded.                     */
/* ------------------------------------------------------------------------- */
int oracle_cholesky(const double* M, int n, double* R) {
    if (!M || !R || n < 1) return ORC_BAD_ARG;
    for (int k = 0; k < n * n; ++k) R[k] = 0.0;
    for (int j = 0; j < n; ++j) {
        double d = M[j + (size_t)j * n];
        for (int k = 0; k < j; ++k) d -= R[k + (size_t)j * n] * R[k + (size_t)j * n];
        if (!(d > 0.0)) return ORC_NOT_FULL_RANK;
        const double rjj = sqrt(d);
        R[j + (size_t)j * n] = rjj;
        for (int i = j + 1; i < n; ++i) {
            double s = M[j + (size_t)i * n];
            for (int k = 0; k < j; ++k) s -= R[k + (size_t)j * n] * R[k + (size_t)i * n];
            R[j + (size_t)i * n] = s / rjj;
        }
    }
    return ORC_OK;
}

int oracle_cholqr_rows(const void* A, int64_t m, int64_t n, int64_t lda, int working, const double* Rw,
                       const int64_t* rows, int64_t nrows, int p, double* out) {
    if (!A || !Rw || !rows || !out || n < 1 || p < 2 || p > 53) return ORC_BAD_ARG;
    dd* q = (dd*)malloc(sizeof(dd) * (size_t)n);
    superacc* s = (superacc*)malloc(sizeof(superacc));
    if (!q || !s) { free(q); free(s); return ORC_BAD_ARG; }
    for (int64_t k = 0; k < nrows; ++k) {
        const int64_t r = rows[k];
        if (r < 0 || r >= m) { free(q); free(s); return ORC_BAD_ARG; }
        for (int64_t j = 0; j < n; ++j) {
            dd acc = dd_make(elem(A, working, lda, r, j));
            for (int64_t i = 0; i < j; ++i) acc = dd_sub(acc, dd_mul(q[i], dd_make(Rw[i + j * n])));
            q[j] = dd_div(acc, dd_make(Rw[j + j * n]));
            out[k + j * nrows] = round_dd_exact(s, q[j].hi, q[j].lo, p);
        }
    }
    free(q);
    free(s);
    return ORC_OK;
}
