/*
 * oracle.c — plain, slow, obviously correct CPU oracle for the three-precision
 * Newton method of C. T. Kelley, "Newton's Method in Three Precisions"
 * (arXiv 2307.16051).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA path, and the CUDA path never calls
 * it.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (no -ffast-math):
 * every float/double operation below is one IEEE-754 operation rounded to
 * nearest-even, and no multiply-add is contracted, on x86-64 and on AArch64.
 * OpenMP only splits independent rows; every reduction is sequential in index
 * order, so results do not depend on the thread count.
 *
 * Row-major storage throughout: A[i*N + j] is row i, column j (0-based).
 *
 * Paper references use the paper's numbering: sections, equations (x.y) with
 * their LaTeX labels in brackets, Algorithm 1.1 [newton], Algorithm 2.1
 * [newton3p], Algorithm IR of Section 2.2 [ir], Tables 2 (c = .99) and
 * 3 (c = .9999).
 *
 * Parity status: every function here is pinned by a CPU test (fp16 rounding
 * against an independent IEEE implementation, F and J against closed forms
 * and finite differences, LU against exact rational elimination and LAPACK,
 * GMRES against a dense least-squares solve, Newton against the paper's
 * residual tables).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* IEEE binary16 rounding (Section 1.2, Table 1 "IEEE precisions").          */
/* Written from the IEEE 754 definition of round-to-nearest, ties-to-even:  */
/* the result is the binary16 number nearest to x; on a tie the one whose   */
/* last significand bit is 0; |x| at or above 65520 (the midpoint between  */
/* the largest finite value 65504 and 2^16) becomes infinity; subnormals   */
/* (spacing 2^-24 below 2^-14) are kept.                                   */
/* ------------------------------------------------------------------------ */

#define SIGN64 0x8000000000000000ull
#define INF64 0x7FF0000000000000ull

/* fl16(x): nearest binary16 value of a double, returned as a double. */
double orc_fl16(double x)
{
    uint64_t b;
    memcpy(&b, &x, 8);
    uint64_t s = b & SIGN64, a = b & ~SIGN64;
    if (a >= INF64)
        return x; /* inf and NaN pass through */
    int e = (int)(a >> 52) - 1023; /* unbiased exponent of |x| */
    if (e >= 16) {
        a = INF64; /* |x| >= 2^16 lies beyond the overflow boundary 65520 */
    } else if (e < -25) {
        a = 0; /* below half the smallest subnormal 2^-24 */
    } else if (e == -25) {
        /* x in [2^-25, 2^-24): exactly 2^-25 is a tie between 0 (even) and
           2^-24 (odd) and goes to 0; anything above goes to 2^-24 */
        a = (a == 0x3E60000000000000ull) ? 0 : 0x3E70000000000000ull;
    } else {
        /* number of low double-significand bits below one binary16 ulp:
           ulp = 2^(e-10) for normal halves (e >= -14), 2^-24 below that */
        int sh = (e >= -14) ? 42 : 42 + (-14 - e);
        uint64_t half = 1ull << (sh - 1);
        uint64_t mask = (1ull << sh) - 1;
        uint64_t lsb = (a >> sh) & 1ull;
        a = (a + half - 1 + lsb) & ~mask; /* carry propagates into the exponent */
        if (a >= 0x40F0000000000000ull)   /* rounded up to 2^16: overflow */
            a = INF64;
    }
    b = s | a;
    double r;
    memcpy(&r, &b, 8);
    return r;
}

/* binary16 bit pattern of fl16(x). */
uint16_t orc_f16_bits(double x)
{
    double r = orc_fl16(x);
    uint64_t b;
    memcpy(&b, &r, 8);
    uint16_t s = (uint16_t)((b >> 48) & 0x8000u);
    uint64_t a = b & ~SIGN64;
    if (a > INF64)
        return (uint16_t)(s | 0x7E00u); /* NaN */
    if (a == INF64)
        return (uint16_t)(s | 0x7C00u);
    if (a == 0)
        return s;
    double m = fabs(r);
    if (m < 6.103515625e-05) /* below 2^-14: subnormal, value = k * 2^-24 */
        return (uint16_t)(s | (uint16_t)ldexp(m, 24));
    int e = (int)(a >> 52) - 1023;
    return (uint16_t)(s | (uint16_t)((e + 15) << 10) | (uint16_t)((a >> 42) & 0x3FFu));
}

/* value of a binary16 bit pattern. */
double orc_f16_value(uint16_t h)
{
    int s = (h >> 15) & 1, e = (h >> 10) & 0x1F, m = h & 0x3FF;
    double v;
    if (e == 31)
        v = m ? NAN : INFINITY;
    else if (e == 0)
        v = ldexp((double)m, -24);
    else
        v = ldexp((double)(1024 + m), e - 25);
    return s ? -v : v;
}

void orc_fl16_array(int64_t n, const double *in, double *out)
{
    for (int64_t i = 0; i < n; ++i)
        out[i] = orc_fl16(in[i]);
}

void orc_f16_bits_array_f32(int64_t n, const float *in, uint16_t *out)
{
    for (int64_t i = 0; i < n; ++i)
        out[i] = orc_f16_bits((double)in[i]);
}

/* ------------------------------------------------------------------------ */
/* The test problem (Section 3, eq. (3.2) [hmid]): composite midpoint rule   */
/* for the Chandrasekhar H-equation,                                         */
/*   F(x)_i = x_i - ( 1 - c/(2N) sum_j x_j mu_i/(mu_j + mu_i) )^{-1},        */
/* with nodes mu_i = (i - 1/2)/N, i = 1..N.                                  */
/* ------------------------------------------------------------------------ */

static double mu_node(int64_t i0, int64_t N) /* i0 is 0-based */
{
    return ((double)i0 + 0.5) / (double)N;
}

/* t_i = c/(2N) sum_j x_j mu_i/(mu_j+mu_i), summed j = 1..N in order. */
static double hsum(int64_t N, double c, const double *x, int64_t i)
{
    double mi = mu_node(i, N), s = 0.0;
    for (int64_t j = 0; j < N; ++j)
        s += x[j] * mi / (mu_node(j, N) + mi);
    return c / (2.0 * (double)N) * s;
}

/* F(x) in double precision (eq. (3.2)). */
void orc_F(int64_t N, double c, const double *x, double *F)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i)
        F[i] = x[i] - 1.0 / (1.0 - hsum(N, c, x, i));
}

/* Analytic Jacobian F'(x) in double precision (Sections 1.1 and 3: the paper
   uses the analytic Jacobian).  With r_i = (1 - t_i)^{-1},
     dF_i/dx_j = delta_ij - r_i^2 * c/(2N) * mu_i/(mu_j + mu_i).            */
void orc_jacobian(int64_t N, double c, const double *x, double *J)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double ri = 1.0 / (1.0 - hsum(N, c, x, i));
        double mi = mu_node(i, N);
        for (int64_t j = 0; j < N; ++j) {
            double d = ri * ri * (c / (2.0 * (double)N)) * (mi / (mu_node(j, N) + mi));
            J[i * N + j] = (i == j ? 1.0 : 0.0) - d;
        }
    }
}

/* Optional scaling of the Jacobian into the binary16 range before the
   down-cast (Section 2.3 warns that rounding to half precision can underflow;
   the paper scales vectors, this scales the rows of J).  Row i of J is
   bounded by B_i = 1 + c/(2N) r_i^2, since |J_ij| <= delta_ij + c/(2N) r_i^2
   mu_i/(mu_i + mu_j) and mu_i/(mu_i + mu_j) < 1.  The row factor is the power
   of two 2^k_i with k_i the largest integer such that 2^k_i B_i <= 2^13
   (three bits of headroom below the binary16 maximum 65504 for growth in the
   elimination): k_i = 13 - ceil(log2 B_i), found exactly from frexp.
   Multiplying a binary32 entry by 2^k_i is exact, so J_h = I_s^h(R J32)
   differs from I_s^h(J32) only in its rounding to binary16. */
void orc_row_scales(int64_t N, double c, const double *x, double *rs)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double ri = 1.0 / (1.0 - hsum(N, c, x, i));
        double B = 1.0 + (c / (2.0 * (double)N)) * ri * ri;
        int e;
        double m = frexp(B, &e); /* B = m 2^e, m in [0.5, 1) */
        int ceil_log2 = (m == 0.5) ? e - 1 : e;
        rs[i] = ldexp(1.0, 13 - ceil_log2);
    }
}

double orc_norm2(int64_t n, const double *v)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i)
        s += v[i] * v[i];
    return sqrt(s);
}

static double norm2_f(int64_t n, const float *v)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i)
        s += (double)v[i] * (double)v[i];
    return sqrt(s);
}

/* ------------------------------------------------------------------------ */
/* Gaussian elimination with partial pivoting (Section 1.3: J = L U by an    */
/* LU factorisation; Section 2: J_h factored in half precision).             */
/* Unblocked, right-looking.  At step k the pivot is the first row i >= k   */
/* (in current order) of largest |a_ik|; rows k and p are swapped across the */
/* whole width; ipiv[k] = p (0-based, LAPACK convention).  L is unit lower  */
/* and stored below the diagonal, U on and above it.  A zero pivot leaves   */
/* the column unscaled and is reported as info = k+1 for the first such k.  */
/* ------------------------------------------------------------------------ */

static void swap_rows_d(double *A, int64_t N, int64_t r1, int64_t r2)
{
    if (r1 == r2)
        return;
    for (int64_t j = 0; j < N; ++j) {
        double t = A[r1 * N + j];
        A[r1 * N + j] = A[r2 * N + j];
        A[r2 * N + j] = t;
    }
}

static int64_t pivot_row_d(const double *A, int64_t N, int64_t k)
{
    int64_t p = k;
    double best = fabs(A[k * N + k]);
    for (int64_t i = k + 1; i < N; ++i) {
        double v = fabs(A[i * N + k]);
        if (v > best) {
            best = v;
            p = i;
        }
    }
    return p;
}

/* FP64 arithmetic (the F64 column of Tables 2 and 3). */
int orc_lu64(int64_t N, double *A, int32_t *ipiv)
{
    int info = 0;
    for (int64_t k = 0; k < N; ++k) {
        int64_t p = pivot_row_d(A, N, k);
        ipiv[k] = (int32_t)p;
        swap_rows_d(A, N, k, p);
        double akk = A[k * N + k];
        if (akk == 0.0) {
            if (!info)
                info = (int)k + 1;
            continue;
        }
#pragma omp parallel for schedule(static)
        for (int64_t i = k + 1; i < N; ++i) {
            double l = A[i * N + k] / akk;
            A[i * N + k] = l;
            for (int64_t j = k + 1; j < N; ++j)
                A[i * N + j] = A[i * N + j] - l * A[k * N + j];
        }
    }
    return info;
}

/* FP32 arithmetic: every operation rounded to single (the F32 column). */
int orc_lu32(int64_t N, float *A, int32_t *ipiv)
{
    int info = 0;
    for (int64_t k = 0; k < N; ++k) {
        int64_t p = k;
        float best = fabsf(A[k * N + k]);
        for (int64_t i = k + 1; i < N; ++i)
            if (fabsf(A[i * N + k]) > best) {
                best = fabsf(A[i * N + k]);
                p = i;
            }
        ipiv[k] = (int32_t)p;
        if (p != k)
            for (int64_t j = 0; j < N; ++j) {
                float t = A[k * N + j];
                A[k * N + j] = A[p * N + j];
                A[p * N + j] = t;
            }
        float akk = A[k * N + k];
        if (akk == 0.0f) {
            if (!info)
                info = (int)k + 1;
            continue;
        }
#pragma omp parallel for schedule(static)
        for (int64_t i = k + 1; i < N; ++i) {
            float l = A[i * N + k] / akk;
            A[i * N + k] = l;
            for (int64_t j = k + 1; j < N; ++j) {
                float prod = l * A[k * N + j];
                A[i * N + j] = A[i * N + j] - prod;
            }
        }
    }
    return info;
}

/* FP16 arithmetic (Section 2: "factor J_h in half precision"; Section 3.1:
   the half-precision computations of the paper).  A holds binary16 values
   (as doubles).  Every arithmetic result is rounded to binary16:
     l_ik = fl16(a_ik / a_kk),   a_ij = fl16(a_ij - fl16(l_ik * a_kj)).
   The quotient, product and difference are first formed in double; for
   binary16 operands that double is exact (product, difference) or rounds
   to the same binary16 value as the exact quotient, so each step is one
   correctly rounded binary16 operation.  Returns info; sets *overflow when a
   result overflowed to infinity. */
static int lu16_impl(int64_t N, double *A, int32_t *ipiv, int *overflow, int recip)
{
    int info = 0, ovf = 0;
    for (int64_t k = 0; k < N; ++k) {
        int64_t p = pivot_row_d(A, N, k);
        ipiv[k] = (int32_t)p;
        swap_rows_d(A, N, k, p);
        double akk = A[k * N + k];
        if (akk == 0.0) {
            if (!info)
                info = (int)k + 1;
            continue;
        }
        const double rk = orc_fl16(1.0 / akk); /* recip: the rounded reciprocal of the pivot */
#pragma omp parallel for schedule(static) reduction(| : ovf)
        for (int64_t i = k + 1; i < N; ++i) {
            double l = recip ? orc_fl16(A[i * N + k] * rk) : orc_fl16(A[i * N + k] / akk);
            A[i * N + k] = l;
            for (int64_t j = k + 1; j < N; ++j) {
                double v = orc_fl16(A[i * N + j] - orc_fl16(l * A[k * N + j]));
                if (isinf(v))
                    ovf = 1;
                A[i * N + j] = v;
            }
        }
    }
    if (overflow)
        *overflow = ovf;
    return info;
}

int orc_lu16(int64_t N, double *A, int32_t *ipiv, int *overflow)
{
    return lu16_impl(N, A, ipiv, overflow, 0);
}

/* The same elimination with the column scaled by the reciprocal of the pivot,
   as unblocked LAPACK-style codes do (xGETF2 multiplies the column below the
   pivot by 1/a_kk): r = fl16(1/a_kk), l_ik = fl16(a_ik * r), then
   a_ij = fl16(a_ij - fl16(l_ik * a_kj)).  r carries one more rounding than
   the quotient, so every multiplier of column k shares r's relative error. */
int orc_lu16_recip(int64_t N, double *A, int32_t *ipiv, int *overflow)
{
    return lu16_impl(N, A, ipiv, overflow, 1);
}

/* Half-precision factorisation with binary16 storage and binary32
   arithmetic (the arithmetic model of the GPU factorisation; the paper does
   not fix one, Section 2 only says the factorisation of J_h is done in half
   precision).  Gaussian elimination with partial pivoting in which
     - the pivot row's entries u_kj (j >= k) and the multipliers
       l_ik = fl16(a_ik / u_kk) are rounded to binary16 when they are formed;
     - the entries not yet eliminated are carried in binary32 and updated
       a_ij <- a_ij - l_ik u_kj (the product of two binary16 numbers is exact
       in binary32, so this is one binary32 rounding);
     - after every nb elimination steps (k+1 a multiple of nb) the
       not-yet-eliminated submatrix is rounded to binary16.
   A holds binary16 values (as doubles) on entry and the binary16 factors on
   exit.  The pivot is the first row of largest binary32 |a_ik|.
   Returns info (first zero pivot, 1-based) and sets *overflow on an
   infinite entry. */
int orc_lu16_dev(int64_t N, int64_t nb, double *A, int32_t *ipiv, int *overflow)
{
    size_t NN = (size_t)N * (size_t)N;
    float *W = (float *)malloc(sizeof(float) * NN);
    for (size_t q = 0; q < NN; ++q)
        W[q] = (float)A[q];
    int info = 0, ovf = 0;
    if (nb < 1)
        nb = 1;
    for (int64_t k = 0; k < N; ++k) {
        int64_t p = k;
        float best = fabsf(W[k * N + k]);
        for (int64_t i = k + 1; i < N; ++i)
            if (fabsf(W[i * N + k]) > best) {
                best = fabsf(W[i * N + k]);
                p = i;
            }
        ipiv[k] = (int32_t)p;
        if (p != k)
            for (int64_t j = 0; j < N; ++j) {
                float t = W[k * N + j];
                W[k * N + j] = W[p * N + j];
                W[p * N + j] = t;
            }
        for (int64_t j = k; j < N; ++j)
            W[k * N + j] = (float)orc_fl16((double)W[k * N + j]);
        float ukk = W[k * N + k];
        if (ukk == 0.0f) {
            if (!info)
                info = (int)k + 1;
        } else {
#pragma omp parallel for schedule(static)
            for (int64_t i = k + 1; i < N; ++i) {
                float l = (float)orc_fl16((double)(W[i * N + k] / ukk));
                W[i * N + k] = l;
                for (int64_t j = k + 1; j < N; ++j) {
                    float prod = l * W[k * N + j];
                    W[i * N + j] = W[i * N + j] - prod;
                }
            }
        }
        if ((k + 1) % nb == 0 || k == N - 1) {
#pragma omp parallel for schedule(static) reduction(| : ovf)
            for (int64_t i = k + 1; i < N; ++i)
                for (int64_t j = k + 1; j < N; ++j) {
                    float v = (float)orc_fl16((double)W[i * N + j]);
                    if (isinf(v))
                        ovf = 1;
                    W[i * N + j] = v;
                }
        }
    }
    for (size_t q = 0; q < NN; ++q) {
        A[q] = (double)W[q];
        if (isinf(A[q]))
            ovf = 1;
    }
    free(W);
    if (overflow)
        *overflow = ovf;
    return info;
}

/* Apply the row interchanges ipiv[0..N-1] in order to a vector. */
static void apply_pivots_d(int64_t N, const int32_t *ipiv, double *b)
{
    for (int64_t k = 0; k < N; ++k) {
        int64_t p = ipiv[k];
        if (p != k) {
            double t = b[k];
            b[k] = b[p];
            b[p] = t;
        }
    }
}
static void apply_pivots_f(int64_t N, const int32_t *ipiv, float *b)
{
    for (int64_t k = 0; k < N; ++k) {
        int64_t p = ipiv[k];
        if (p != k) {
            float t = b[k];
            b[k] = b[p];
            b[p] = t;
        }
    }
}

/* Solve (L U) z = P b in double, in place (forward then back substitution). */
void orc_lusolve64(int64_t N, const double *LU, const int32_t *ipiv, double *b)
{
    apply_pivots_d(N, ipiv, b);
    for (int64_t i = 0; i < N; ++i) {
        double s = b[i];
        for (int64_t t = 0; t < i; ++t)
            s = s - LU[i * N + t] * b[t];
        b[i] = s;
    }
    for (int64_t i = N - 1; i >= 0; --i) {
        double s = b[i];
        for (int64_t t = i + 1; t < N; ++t)
            s = s - LU[i * N + t] * b[t];
        b[i] = s / LU[i * N + i];
    }
}

/* Single-precision solve with single-precision factors (F32 column). */
void orc_lusolve32(int64_t N, const float *LU, const int32_t *ipiv, float *b)
{
    apply_pivots_f(N, ipiv, b);
    for (int64_t i = 0; i < N; ++i) {
        float s = b[i];
        for (int64_t t = 0; t < i; ++t) {
            float prod = LU[i * N + t] * b[t];
            s = s - prod;
        }
        b[i] = s;
    }
    for (int64_t i = N - 1; i >= 0; --i) {
        float s = b[i];
        for (int64_t t = i + 1; t < N; ++t) {
            float prod = LU[i * N + t] * b[t];
            s = s - prod;
        }
        b[i] = s / LU[i * N + i];
    }
}

/* Eq. (2.16) [fly], "interprecision transfer on the fly": the half-precision
   factors (binary16 values held as doubles) are promoted to single precision
   element by element and both triangular solves run in single-precision
   arithmetic.  b is single precision, in place. */
void orc_lusolve_fly(int64_t N, const double *LU16, const int32_t *ipiv, float *b)
{
    apply_pivots_f(N, ipiv, b);
    for (int64_t i = 0; i < N; ++i) {
        float s = b[i];
        for (int64_t t = 0; t < i; ++t) {
            float prod = (float)LU16[i * N + t] * b[t];
            s = s - prod;
        }
        b[i] = s;
    }
    for (int64_t i = N - 1; i >= 0; --i) {
        float s = b[i];
        for (int64_t t = i + 1; t < N; ++t) {
            float prod = (float)LU16[i * N + t] * b[t];
            s = s - prod;
        }
        b[i] = s / (float)LU16[i * N + i];
    }
}

/* Both triangular solves entirely in binary16 arithmetic (the inner solve of
   eq. (2.17) [nofly] and of eq. (2.19) [cheapir], and the step of the F16
   column, Section 1.3).  b holds binary16 values (as doubles), in place.
   The paper fixes the precision of every operation, not the order of each
   row's terms: the forward solve takes row i's terms in increasing t, the
   backward solve in decreasing t (from the last column towards the
   diagonal), the order of a column-oriented back substitution. */
void orc_lusolve16(int64_t N, const double *LU16, const int32_t *ipiv, double *b)
{
    apply_pivots_d(N, ipiv, b);
    for (int64_t i = 0; i < N; ++i) {
        double s = b[i];
        for (int64_t t = 0; t < i; ++t)
            s = orc_fl16(s - orc_fl16(LU16[i * N + t] * b[t]));
        b[i] = s;
    }
    for (int64_t i = N - 1; i >= 0; --i) {
        double s = b[i];
        for (int64_t t = N - 1; t > i; --t)
            s = orc_fl16(s - orc_fl16(LU16[i * N + t] * b[t]));
        b[i] = orc_fl16(s / LU16[i * N + i]);
    }
}

/* ------------------------------------------------------------------------ */
/* Linear iterations for the Newton step (Section 2.2).                      */
/* ------------------------------------------------------------------------ */

/* r = b - A u for the single-precision system A = J (Algorithm IR, first and
   last lines): each entry is accumulated in double in column order and
   rounded once to single. */
static void residual32(int64_t N, const float *A, const float *b, const float *u, float *r)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double s = (double)b[i];
        for (int64_t j = 0; j < N; ++j)
            s -= (double)A[i * N + j] * (double)u[j];
        r[i] = (float)s;
    }
}

/* z = (L U)^{-1} P v with the on-the-fly single-precision solve, in double
   vectors (the preconditioner-vector product of GMRES-IR, Section 2.2: "two
   triangular solves", done in single precision per Section 2.3). */
static void precond_apply(int64_t N, const double *LU16, const int32_t *ipiv, const double *rs,
                          const double *v, double *z, float *tmp)
{
    for (int64_t i = 0; i < N; ++i)
        tmp[i] = (float)v[i];
    if (rs) /* factors of R J: (R J)^{-1} R v = J^{-1} v; times 2^k is exact */
        for (int64_t i = 0; i < N; ++i)
            tmp[i] = tmp[i] * (float)rs[i];
    orc_lusolve_fly(N, LU16, ipiv, tmp);
    for (int64_t i = 0; i < N; ++i)
        z[i] = (double)tmp[i];
}

/* w = A v with A single precision, v double; double arithmetic. */
static void matvec32(int64_t N, const float *A, const double *v, double *w)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < N; ++j)
            s += (double)A[i * N + j] * v[j];
        w[i] = s;
    }
}

typedef struct {
    int iters;    /* linear iterations: IR corrections, or GMRES Arnoldi steps */
    int outer;    /* IR / GMRES-IR outer corrections */
    int failed;   /* IR failure rule fired (residual increased) */
    int converged;/* relative residual <= eta reached */
    double relres;/* final ||b - A u|| / ||b|| */
} orc_linstat;

/* Restarted, left-preconditioned GMRES(m) for M^{-1} A d = M^{-1} r with
   M = L U from the half-precision factorisation (Section 2.2, GMRES-IR).
   d0 = 0, modified Gram-Schmidt Arnoldi, Givens rotations, double
   arithmetic apart from the single-precision preconditioner solve.
   Stops when the preconditioned residual estimate is <= tol times the
   initial preconditioned residual norm, or after maxcycles restarts.
   Returns the number of Arnoldi steps. */
static int gmres_impl(int64_t N, const float *A, const double *LU16, const int32_t *ipiv, const double *rs,
                      const double *r, double *d, int m, double tol, int maxcycles)
{
    double *V = (double *)malloc(sizeof(double) * (size_t)N * (size_t)(m + 1));
    double *H = (double *)calloc((size_t)(m + 1) * (size_t)m, sizeof(double));
    double *cs = (double *)malloc(sizeof(double) * (size_t)m);
    double *sn = (double *)malloc(sizeof(double) * (size_t)m);
    double *g = (double *)malloc(sizeof(double) * (size_t)(m + 1));
    double *y = (double *)malloc(sizeof(double) * (size_t)m);
    double *w = (double *)malloc(sizeof(double) * (size_t)N);
    double *t = (double *)malloc(sizeof(double) * (size_t)N);
    float *tmp = (float *)malloc(sizeof(float) * (size_t)N);
    int steps = 0;
    double beta0 = -1.0;
    for (int64_t i = 0; i < N; ++i)
        d[i] = 0.0;
    for (int cycle = 0; cycle < maxcycles; ++cycle) {
        /* preconditioned residual of the current d: M^{-1}(r - A d) */
        matvec32(N, A, d, w);
        for (int64_t i = 0; i < N; ++i)
            t[i] = r[i] - w[i];
        precond_apply(N, LU16, ipiv, rs, t, w, tmp);
        double beta = orc_norm2(N, w);
        if (beta0 < 0.0)
            beta0 = beta;
        if (beta == 0.0 || beta <= tol * beta0)
            break;
        for (int64_t i = 0; i < N; ++i)
            V[i] = w[i] / beta;
        for (int k = 0; k <= m; ++k)
            g[k] = 0.0;
        g[0] = beta;
        int j, done = 0;
        for (j = 0; j < m; ++j) {
            /* w = M^{-1} A v_j */
            matvec32(N, A, V + (size_t)j * N, t);
            precond_apply(N, LU16, ipiv, rs, t, w, tmp);
            ++steps;
            /* modified Gram-Schmidt against v_0..v_j */
            for (int i = 0; i <= j; ++i) {
                const double *vi = V + (size_t)i * N;
                double h = 0.0;
                for (int64_t q = 0; q < N; ++q)
                    h += w[q] * vi[q];
                H[i * m + j] = h;
                for (int64_t q = 0; q < N; ++q)
                    w[q] -= h * vi[q];
            }
            double hn = orc_norm2(N, w);
            H[(j + 1) * m + j] = hn;
            if (hn != 0.0)
                for (int64_t q = 0; q < N; ++q)
                    V[(size_t)(j + 1) * N + q] = w[q] / hn;
            /* previous rotations on the new column, then a new rotation */
            for (int i = 0; i < j; ++i) {
                double a = H[i * m + j], b = H[(i + 1) * m + j];
                H[i * m + j] = cs[i] * a + sn[i] * b;
                H[(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
            }
            double a = H[j * m + j], b = H[(j + 1) * m + j];
            double rho = hypot(a, b);
            cs[j] = (rho == 0.0) ? 1.0 : a / rho;
            sn[j] = (rho == 0.0) ? 0.0 : b / rho;
            H[j * m + j] = rho;
            H[(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            if (fabs(g[j + 1]) <= tol * beta0 || hn == 0.0) {
                done = 1;
                ++j;
                break;
            }
        }
        /* y = R^{-1} g (upper triangular j x j), d += V y */
        for (int i = j - 1; i >= 0; --i) {
            double s = g[i];
            for (int k = i + 1; k < j; ++k)
                s -= H[i * m + k] * y[k];
            y[i] = s / H[i * m + i];
        }
        for (int i = 0; i < j; ++i)
            for (int64_t q = 0; q < N; ++q)
                d[q] += y[i] * V[(size_t)i * N + q];
        if (done)
            break;
    }
    free(V);
    free(H);
    free(cs);
    free(sn);
    free(g);
    free(y);
    free(w);
    free(t);
    free(tmp);
    return steps;
}

int orc_gmres(int64_t N, const float *A, const double *LU16, const int32_t *ipiv, const double *r,
              double *d, int m, double tol, int maxcycles)
{
    return gmres_impl(N, A, LU16, ipiv, NULL, r, d, m, tol, maxcycles);
}

/* Iterative refinement (Algorithm IR, Section 2.2) and GMRES-IR for
   A u = b with A single precision and a half-precision factorisation.
   u0 = 0.  Stops with success when ||b - A u|| <= eta ||b|| (Section 3.1),
   declares failure when the residual norm increases and then returns the
   iterate with the smallest residual (Section 3.1), and otherwise stops
   after maxit corrections.
   solver: 0 = IR with the on-the-fly correction d = U^{-1} L^{-1} r
               (eq. (2.16) applied to IR, Section 2.3);
           1 = IR with the scaled half-precision correction of eq. (2.19);
           2 = GMRES-IR (defect from GMRES(m) on M^{-1} A d = M^{-1} r). */
/* rs (may be NULL): the row factors of a scaled factorisation LU = P R A
   (orc_row_scales); every solve with the factors is applied to R times its
   right-hand side, so that it solves with A. */
void orc_linsolve_scaled(int64_t N, const float *A, const double *LU16, const int32_t *ipiv, const double *rs,
                         const float *b, float *u, double eta, int maxit, int solver, int m, double gtol,
                         int gcycles, orc_linstat *st)
{
    float *r = (float *)malloc(sizeof(float) * (size_t)N);
    float *ubest = (float *)malloc(sizeof(float) * (size_t)N);
    float *dv = (float *)malloc(sizeof(float) * (size_t)N);
    double *rd = (double *)malloc(sizeof(double) * (size_t)N);
    double *dd = (double *)malloc(sizeof(double) * (size_t)N);
    double *h16 = (double *)malloc(sizeof(double) * (size_t)N);
    memset(st, 0, sizeof(*st));
    for (int64_t i = 0; i < N; ++i)
        u[i] = 0.0f;
    double nb = norm2_f(N, b);
    residual32(N, A, b, u, r);
    double nr = norm2_f(N, r), best = nr, prev = nr;
    memcpy(ubest, u, sizeof(float) * (size_t)N);
    for (;;) {
        if (nr <= eta * nb) {
            st->converged = 1;
            break;
        }
        if (st->outer >= maxit)
            break;
        if (solver == 0) {
            memcpy(dv, r, sizeof(float) * (size_t)N);
            if (rs)
                for (int64_t i = 0; i < N; ++i)
                    dv[i] = dv[i] * (float)rs[i];
            orc_lusolve_fly(N, LU16, ipiv, dv);
            st->iters++;
        } else if (solver == 1) {
            /* eq. (2.19): d = ||r|| I_h^s( U^{-1} L^{-1} I_s^h(r/||r||) ) */
            float rn = (float)nr;
            for (int64_t i = 0; i < N; ++i)
                h16[i] = orc_fl16((double)(r[i] / rn) * (rs ? rs[i] : 1.0));
            orc_lusolve16(N, LU16, ipiv, h16);
            for (int64_t i = 0; i < N; ++i)
                dv[i] = rn * (float)h16[i];
            st->iters++;
        } else {
            for (int64_t i = 0; i < N; ++i)
                rd[i] = (double)r[i];
            st->iters += gmres_impl(N, A, LU16, ipiv, rs, rd, dd, m, gtol, gcycles);
            for (int64_t i = 0; i < N; ++i)
                dv[i] = (float)dd[i];
        }
        for (int64_t i = 0; i < N; ++i)
            u[i] = u[i] + dv[i];
        st->outer++;
        residual32(N, A, b, u, r);
        nr = norm2_f(N, r);
        if (nr > prev) {
            st->failed = 1;
            memcpy(u, ubest, sizeof(float) * (size_t)N);
            nr = best;
            break;
        }
        prev = nr;
        if (nr < best) {
            best = nr;
            memcpy(ubest, u, sizeof(float) * (size_t)N);
        }
    }
    st->relres = (nb > 0.0) ? nr / nb : 0.0;
    free(r);
    free(ubest);
    free(dv);
    free(rd);
    free(dd);
    free(h16);
}

void orc_linsolve(int64_t N, const float *A, const double *LU16, const int32_t *ipiv, const float *b,
                  float *u, double eta, int maxit, int solver, int m, double gtol, int gcycles,
                  orc_linstat *st)
{
    orc_linsolve_scaled(N, A, LU16, ipiv, NULL, b, u, eta, maxit, solver, m, gtol, gcycles, st);
}

/* ------------------------------------------------------------------------ */
/* Newton drivers: Algorithm 1.1 [newton] and Algorithm 2.1 [newton3p].      */
/* ------------------------------------------------------------------------ */

enum { ORC_FP64LU = 0, ORC_IR16 = 1, ORC_GMRESIR16 = 2, ORC_F32 = 3, ORC_F16 = 4, ORC_IR16GM = 5 };

typedef struct {
    double eta;         /* eta_J of eq. (2.3) [inexactJ] */
    int ir_maxit;       /* cap on IR / GMRES-IR outer corrections */
    int gmres_m;        /* GMRES restart length */
    double gmres_tol;   /* GMRES relative tolerance on the preconditioned residual */
    int gmres_cycles;   /* GMRES restart cycles */
    int newton_maxit;   /* cap on Newton steps */
    double tau_a;       /* absolute tolerance of Algorithm 1.1 */
    int ir_variant;     /* 0: on-the-fly correction (eq. 2.16), 1: scaled fp16 (eq. 2.19) */
    int lu_nb;          /* 0: binary16 arithmetic LU (orc_lu16); -1: the same with the
                           multipliers scaled by the rounded reciprocal of the pivot
                           (orc_lu16_recip); >0: binary16 storage, binary32 arithmetic,
                           rounding period lu_nb (orc_lu16_dev) */
    int scale_fp16;     /* 1: J_h = I_s^h(R J32) with the row factors of orc_row_scales, the
                           solves applied to R times their right-hand side (three-precision
                           modes) */
} orc_params;

typedef struct {
    int status;         /* 0 converged, 1 not converged after newton_maxit, 2 numeric (NaN/Inf), 3 fp16 overflow */
    int newton_iters;
    double hist[128];   /* ||F(x_n)||_2 / ||F(x_0)||_2, n = 0..newton_iters */
    int lin_iters[128];
    int lin_outer[128];
    int lin_failed[128];
    double lin_relres[128];
    int lu_info[128];
} orc_result;

/* Newton's method from x0 until ||F|| <= tau_r ||F(x0)|| + tau_a.
   The step solves J s = -F with the scaled right-hand side of eqs. (2.17)
   [nofly] and (2.18) [noflystep] (Section 2.3):  the unit vector
   -F/||F|| is rounded to the working precision of the solve, the solve
   returns u, and s = ||F|| u (promoted to double).
   mode ORC_FP64LU: J stored and factored in double (Algorithm 1.1, F64).
   mode ORC_IR16 / ORC_GMRESIR16: J stored in single, J_h = I_s^h(J) factored
     in half, and J u = b solved to ||J u - b|| <= eta ||b|| by IR or
     GMRES-IR (Algorithm 2.1).
   mode ORC_F32 / ORC_F16: two-precision Newton of Section 1.3: J stored and
     factored in single / half and the step computed with one solve in that
     precision (columns F32 / F16 of Tables 2 and 3).  F16 factors
     J_h = I_s^h(J) as the three-precision modes do (p->lu_nb selects the
     arithmetic model) and solves in binary16 arithmetic.
   mode ORC_IR16GM: as ORC_IR16 until the first step whose IR does not meet
     eta (the failure rule of Section 3.1 or the iteration cap); that step is
     solved again by GMRES-IR from u0 = 0, as are all later steps. */
int orc_newton(int64_t N, double c, int mode, const double *x0, double tau_r, const orc_params *p,
               double *x, orc_result *res)
{
    memset(res, 0, sizeof(*res));
    size_t NN = (size_t)N * (size_t)N;
    double *F = (double *)malloc(sizeof(double) * (size_t)N);
    double *J = (double *)malloc(sizeof(double) * NN);
    float *J32 = (mode == ORC_FP64LU || mode == ORC_F16) ? NULL : (float *)malloc(sizeof(float) * NN);
    float *LU32 = (mode == ORC_F32) ? (float *)malloc(sizeof(float) * NN) : NULL;
    int32_t *ipiv = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    float *b32 = (float *)malloc(sizeof(float) * (size_t)N);
    float *u32 = (float *)malloc(sizeof(float) * (size_t)N);
    double *bd = (double *)malloc(sizeof(double) * (size_t)N);
    double *rs = p->scale_fp16 ? (double *)malloc(sizeof(double) * (size_t)N) : NULL;
    double *xbest = (double *)malloc(sizeof(double) * (size_t)N);

    for (int64_t i = 0; i < N; ++i)
        x[i] = x0 ? x0[i] : 1.0;
    orc_F(N, c, x, F);
    double f0 = orc_norm2(N, F), fn = f0;
    double tau = tau_r * f0 + p->tau_a;
    /* the iterate with the smallest ||F||, returned when the iteration does
       not meet the tolerance (the convention of the C interface) */
    double fbest = f0;
    memcpy(xbest, x, sizeof(double) * (size_t)N);
    res->hist[0] = 1.0;
    int n = 0, gm_sticky = 0;
    res->status = 1;
    while (!(fn <= tau)) {
        if (!isfinite(fn)) {
            res->status = 2;
            break;
        }
        if (n >= p->newton_maxit || n >= 127)
            break;
        orc_jacobian(N, c, x, J);
        if (mode == ORC_FP64LU) {
            res->lu_info[n] = orc_lu64(N, J, ipiv);
            for (int64_t i = 0; i < N; ++i)
                bd[i] = -F[i] / fn;
            orc_lusolve64(N, J, ipiv, bd);
            for (int64_t i = 0; i < N; ++i)
                x[i] = x[i] + fn * bd[i];
        } else if (mode == ORC_F32) {
            for (size_t q = 0; q < NN; ++q)
                LU32[q] = (float)J[q];
            res->lu_info[n] = orc_lu32(N, LU32, ipiv);
            for (int64_t i = 0; i < N; ++i)
                b32[i] = (float)(-F[i] / fn);
            orc_lusolve32(N, LU32, ipiv, b32);
            for (int64_t i = 0; i < N; ++i)
                x[i] = x[i] + fn * (double)b32[i];
        } else if (mode == ORC_F16) {
            /* J_h = I_s^h(J) from the single-precision Jacobian and the same
               half-precision factorisation as the three-precision modes */
            int ovf = 0;
            for (size_t q = 0; q < NN; ++q)
                J[q] = orc_fl16((double)(float)J[q]);
            if (p->lu_nb > 0)
                res->lu_info[n] = orc_lu16_dev(N, p->lu_nb, J, ipiv, &ovf);
            else if (p->lu_nb == -1)
                res->lu_info[n] = orc_lu16_recip(N, J, ipiv, &ovf);
            else
                res->lu_info[n] = orc_lu16(N, J, ipiv, &ovf);
            if (ovf) {
                res->status = 3;
                break;
            }
            for (int64_t i = 0; i < N; ++i)
                bd[i] = orc_fl16(-F[i] / fn);
            orc_lusolve16(N, J, ipiv, bd);
            for (int64_t i = 0; i < N; ++i)
                x[i] = x[i] + fn * bd[i];
        } else {
            /* Algorithm 2.1: J in single, J_h = I_s^h(J) in half (of R J with
               the row factors R when scale_fp16 is set) */
            int ovf = 0;
            if (rs)
                orc_row_scales(N, c, x, rs);
            for (size_t q = 0; q < NN; ++q) {
                J32[q] = (float)J[q];
                J[q] = orc_fl16((double)J32[q] * (rs ? rs[q / (size_t)N] : 1.0));
            }
            if (p->lu_nb > 0)
                res->lu_info[n] = orc_lu16_dev(N, p->lu_nb, J, ipiv, &ovf);
            else if (p->lu_nb == -1)
                res->lu_info[n] = orc_lu16_recip(N, J, ipiv, &ovf);
            else
                res->lu_info[n] = orc_lu16(N, J, ipiv, &ovf);
            if (ovf) {
                res->status = 3;
                break;
            }
            for (int64_t i = 0; i < N; ++i)
                b32[i] = (float)(-F[i] / fn);
            orc_linstat st;
            int solver = (mode == ORC_GMRESIR16 || gm_sticky) ? 2 : p->ir_variant;
            orc_linsolve_scaled(N, J32, J, ipiv, rs, b32, u32, p->eta, p->ir_maxit, solver, p->gmres_m,
                                p->gmres_tol, p->gmres_cycles, &st);
            if (mode == ORC_IR16GM && !gm_sticky && !st.converged) {
                /* IR stalled (failure rule or cap without meeting eta): this
                   step's correction is recomputed by GMRES-IR (Section 2.2)
                   from u0 = 0, and GMRES-IR serves every later step. */
                orc_linstat sg;
                gm_sticky = 1;
                orc_linsolve_scaled(N, J32, J, ipiv, rs, b32, u32, p->eta, p->ir_maxit, 2, p->gmres_m,
                                    p->gmres_tol, p->gmres_cycles, &sg);
                sg.iters += st.iters;
                sg.outer += st.outer;
                sg.failed = 1;
                st = sg;
            }
            res->lin_iters[n] = st.iters;
            res->lin_outer[n] = st.outer;
            res->lin_failed[n] = st.failed;
            res->lin_relres[n] = st.relres;
            for (int64_t i = 0; i < N; ++i)
                x[i] = x[i] + fn * (double)u32[i];
        }
        ++n;
        orc_F(N, c, x, F);
        fn = orc_norm2(N, F);
        res->hist[n] = (f0 > 0.0) ? fn / f0 : 0.0;
        if (fn < fbest) {
            fbest = fn;
            memcpy(xbest, x, sizeof(double) * (size_t)N);
        }
    }
    if (fn <= tau)
        res->status = 0;
    else if (fbest < fn || !isfinite(fn))
        memcpy(x, xbest, sizeof(double) * (size_t)N);
    res->newton_iters = n;
    free(F);
    free(J);
    free(J32);
    free(LU32);
    free(ipiv);
    free(b32);
    free(u32);
    free(bd);
    free(rs);
    free(xbest);
    return res->status;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
