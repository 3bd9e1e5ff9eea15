/*
 * perm_oracle.c -- the CPU oracle for matrix permanents.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
 * its Python binding) may link, load or call this file.  Only tests/, the smoke
 * check and the CPU-baseline leg of bench.py use it.  It shares no code, header,
 * table or helper with the CUDA path.
 *
 * What it computes (Su & Zheng, arXiv:1802.02779):
 *   - Eq. (1), Section 3.1: per(A) = sum over permutations s of prod_i a[i][s(i)].
 *     Written out literally (every permutation, every product) for n <= 10.
 *   - Eq. (4), Section 3.3: per(A) = (-1)^n sum_{S subset of columns} (-1)^{|S|}
 *     prod_i sum_{j in S} a[i][j].  Every one of the 2^n subsets is visited.
 *     The row sums of one subset reuse those of the previous subset, as the
 *     paper asks in Section 3.3 (it orders subsets by size; here the reuse comes
 *     from a binary-reflected Gray code, which visits the same 2^n subsets in a
 *     different order; the sum itself is unchanged).  Every 4096 subsets the row
 *     sums are recomputed from scratch so that no update chain is long.
 *
 * Arithmetic:
 *   - integer inputs: exact, modulo 2^256 (four 64-bit limbs, two's complement).
 *     For |per| < 2^255 this is the exact permanent.
 *   - complex inputs: double-double ("dd", an unevaluated sum hi+lo of two
 *     doubles, about 106 significant bits) built only from the error-free
 *     transforms TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and TwoProduct through a
 *     fused multiply-add (Ogita, Rump & Oishi, SIAM J. Sci. Comput. 26(6), 2005).
 *     Results come back as (re_hi, re_lo, im_hi, im_lo).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fopenmp -fPIC -shared.
 * -ffp-contract=off matters: TwoSum is only error-free if no step is fused.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_MAX_N 64

/* ORACLE_PLANT selects a deliberately wrong variant, built only by the test
   that checks that the pins catch such mistakes (tests/test_oracle_plants.py).
   The normal build leaves it at 0. */
#ifndef ORACLE_PLANT
#define ORACLE_PLANT 0
#endif
#define ORACLE_OK 0
#define ORACLE_EINVAL 1

/* ------------------------------------------------------------------ */
/* double-double                                                       */
/* ------------------------------------------------------------------ */
typedef struct { double hi, lo; } dd;
typedef struct { dd re, im; } cdd;

/* Knuth's TwoSum: s + e == a + b exactly. */
static inline dd two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    dd r = {s, e};
    return r;
}
/* Dekker's FastTwoSum, valid when |a| >= |b| (or a == 0). */
static inline dd fast_two_sum(double a, double b) {
    double s = a + b;
    double e = b - (s - a);
    dd r = {s, e};
    return r;
}
/* TwoProduct via fma: p + e == a * b exactly (barring underflow). */
static inline dd two_prod(double a, double b) {
    double p = a * b;
    double e = fma(a, b, -p);
    dd r = {p, e};
    return r;
}
static inline dd dd_from(double a) { dd r = {a, 0.0}; return r; }
/* Accurate dd addition (both components summed with TwoSum). */
static inline dd dd_add(dd a, dd b) {
#if ORACLE_PLANT == 4
    b.lo = 0.0;                      /* planted: drop the low word */
#endif
    dd s = two_sum(a.hi, b.hi);
    dd t = two_sum(a.lo, b.lo);
    double e = s.lo + t.hi;
    dd u = fast_two_sum(s.hi, e);
    e = u.lo + t.lo;
    return fast_two_sum(u.hi, e);
}
static inline dd dd_neg(dd a) { dd r = {-a.hi, -a.lo}; return r; }
static inline dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
static inline dd dd_mul(dd a, dd b) {
    dd p = two_prod(a.hi, b.hi);
    double e = p.lo + (a.hi * b.lo + a.lo * b.hi);
    return fast_two_sum(p.hi, e);
}
static inline cdd cdd_zero(void) { cdd z = {{0.0, 0.0}, {0.0, 0.0}}; return z; }
static inline cdd cdd_from(double re, double im) { cdd z = {dd_from(re), dd_from(im)}; return z; }
static inline cdd cdd_add(cdd a, cdd b) { cdd r = {dd_add(a.re, b.re), dd_add(a.im, b.im)}; return r; }
static inline cdd cdd_sub(cdd a, cdd b) { cdd r = {dd_sub(a.re, b.re), dd_sub(a.im, b.im)}; return r; }
static inline cdd cdd_mul(cdd a, cdd b) {
    cdd r;
    r.re = dd_sub(dd_mul(a.re, b.re), dd_mul(a.im, b.im));
#if ORACLE_PLANT == 5
    r.im = dd_sub(dd_mul(a.re, b.im), dd_mul(a.im, b.re));   /* planted: sign */
#else
    r.im = dd_add(dd_mul(a.re, b.im), dd_mul(a.im, b.re));
#endif
    return r;
}
static void cdd_store(cdd z, double *out) {
    out[0] = z.re.hi; out[1] = z.re.lo; out[2] = z.im.hi; out[3] = z.im.lo;
}

/* Exposed so that tests can check the dd primitives against exact rationals. */
void oracle_dd_add(const double *a, const double *b, double *out) {
    dd x = {a[0], a[1]}, y = {b[0], b[1]};
    dd r = dd_add(x, y);
    out[0] = r.hi; out[1] = r.lo;
}
void oracle_dd_mul(const double *a, const double *b, double *out) {
    dd x = {a[0], a[1]}, y = {b[0], b[1]};
    dd r = dd_mul(x, y);
    out[0] = r.hi; out[1] = r.lo;
}

/* ------------------------------------------------------------------ */
/* 256-bit integers modulo 2^256 (little-endian 64-bit limbs)          */
/* ------------------------------------------------------------------ */
typedef struct { uint64_t w[4]; } u256;

static inline u256 u256_from_i64(int64_t v) {
    u256 r;
    uint64_t fill = v < 0 ? ~(uint64_t)0 : 0;
    r.w[0] = (uint64_t)v; r.w[1] = fill; r.w[2] = fill; r.w[3] = fill;
    return r;
}
static inline u256 u256_add(u256 a, u256 b) {
    u256 r;
    unsigned __int128 c = 0;
    for (int i = 0; i < 4; i++) {
        c += (unsigned __int128)a.w[i] + b.w[i];
        r.w[i] = (uint64_t)c;
        c >>= 64;
    }
    return r;
}
static inline u256 u256_neg(u256 a) {
    u256 r;
    for (int i = 0; i < 4; i++) r.w[i] = ~a.w[i];
    u256 one = u256_from_i64(1);
    return u256_add(r, one);
}
static inline u256 u256_sub(u256 a, u256 b) { return u256_add(a, u256_neg(b)); }
/* (a * v) mod 2^256 for a signed 64-bit v. */
static inline u256 u256_mul_i64(u256 a, int64_t v) {
    int neg = v < 0;
    uint64_t m = neg ? (uint64_t)0 - (uint64_t)v : (uint64_t)v;
    u256 r;
    unsigned __int128 c = 0;
    for (int i = 0; i < 4; i++) {
        c += (unsigned __int128)a.w[i] * m;
        r.w[i] = (uint64_t)c;
        c >>= 64;
    }
    return neg ? u256_neg(r) : r;
}
static void u256_store(u256 a, uint64_t *out) { for (int i = 0; i < 4; i++) out[i] = a.w[i]; }

/* ------------------------------------------------------------------ */
/* Eq. (1): brute force over the symmetric group                       */
/* ------------------------------------------------------------------ */
/* Advance perm[0..n-1] to the next permutation in lexicographic order;
   returns 0 after the last one.  (Textbook next-permutation.) */
static int next_permutation(int *p, int n) {
    int i = n - 2;
    while (i >= 0 && p[i] >= p[i + 1]) i--;
    if (i < 0) return 0;
    int j = n - 1;
    while (p[j] <= p[i]) j--;
    int t = p[i]; p[i] = p[j]; p[j] = t;
    for (int a = i + 1, b = n - 1; a < b; a++, b--) { t = p[a]; p[a] = p[b]; p[b] = t; }
    return 1;
}

/* a: n*n complex entries, row-major, interleaved (re, im).
   out: re_hi, re_lo, im_hi, im_lo.  n = 0 gives 1 (empty product). */
int oracle_per_brute_c128(int n, const double *a, double *out) {
    if (n < 0 || n > 10 || (!a && n > 0) || !out) return ORACLE_EINVAL;
    int p[10];
    for (int i = 0; i < n; i++) p[i] = i;
    cdd total = cdd_zero();
    do {
        cdd prod = cdd_from(1.0, 0.0);
        for (int i = 0; i < n; i++) {
            const double *e = a + 2 * (i * n + p[i]);
            prod = cdd_mul(prod, cdd_from(e[0], e[1]));
        }
        total = cdd_add(total, prod);
    } while (n > 0 && next_permutation(p, n));
    cdd_store(total, out);
    return ORACLE_OK;
}

/* a: n*n int64 entries, row-major.  out: 4 limbs of per(A) mod 2^256. */
int oracle_per_brute_i64(int n, const int64_t *a, uint64_t *out) {
    if (n < 0 || n > 10 || (!a && n > 0) || !out) return ORACLE_EINVAL;
    int p[10];
    for (int i = 0; i < n; i++) p[i] = i;
    u256 total = u256_from_i64(0);
    do {
        u256 prod = u256_from_i64(1);
#if ORACLE_PLANT == 3
        for (int i = 0; i < n; i++) prod = u256_mul_i64(prod, a[i * n + p[0]]);  /* planted: index */
#else
        for (int i = 0; i < n; i++) prod = u256_mul_i64(prod, a[i * n + p[i]]);
#endif
        total = u256_add(total, prod);
    } while (n > 0 && next_permutation(p, n));
    u256_store(total, out);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------ */
/* Eq. (4): Ryser's inclusion-exclusion over all 2^n column subsets    */
/* ------------------------------------------------------------------ */
#define RYSER_REFRESH 4096u   /* row sums recomputed from scratch this often */

/* The subset visited at step g is the binary-reflected Gray code g ^ (g >> 1).
   Bit j set <=> column j is in S. */
static inline uint64_t gray(uint64_t g) { return g ^ (g >> 1); }

static int popcount64(uint64_t x) { int c = 0; while (x) { x &= x - 1; c++; } return c; }

int oracle_per_ryser_i64(int n, const int64_t *a, uint64_t *out, int nthreads) {
    if (n < 0 || n > 40 || (!a && n > 0) || !out) return ORACLE_EINVAL;
    if (n == 0) { u256_store(u256_from_i64(1), out); return ORACLE_OK; }
    const uint64_t total_codes = (uint64_t)1 << n;
    const uint64_t nchunks = (total_codes + RYSER_REFRESH - 1) / RYSER_REFRESH;
    u256 *partial = (u256 *)calloc(nchunks, sizeof(u256));
    if (!partial) return ORACLE_EINVAL;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t c = 0; c < (int64_t)nchunks; c++) {
        uint64_t g0 = (uint64_t)c * RYSER_REFRESH;
        uint64_t g1 = g0 + RYSER_REFRESH < total_codes ? g0 + RYSER_REFRESH : total_codes;
        int64_t rs[64];
        /* row sums of the first subset of the chunk, from scratch */
        uint64_t S = gray(g0);
        for (int i = 0; i < n; i++) {
            int64_t s = 0;
            for (int j = 0; j < n; j++) if ((S >> j) & 1u) s += a[i * n + j];
            rs[i] = s;
        }
        u256 acc = u256_from_i64(0);
        for (uint64_t g = g0; g < g1; g++) {
            if (g > g0) {
                /* step from gray(g-1) to gray(g): exactly one column flips */
                uint64_t Snew = gray(g);
                uint64_t diff = Snew ^ S;
                int j = 0;
                while (!((diff >> j) & 1u)) j++;
                int added = (Snew >> j) & 1u;
                for (int i = 0; i < n; i++) rs[i] += added ? a[i * n + j] : -a[i * n + j];
                S = Snew;
            }
            u256 prod = u256_from_i64(1);
            for (int i = 0; i < n; i++) prod = u256_mul_i64(prod, rs[i]);
#if ORACLE_PLANT == 2
            if (S == total_codes - 1) prod = u256_from_i64(0);   /* planted: dropped term */
#endif
            /* sign (-1)^(n - |S|) */
#if ORACLE_PLANT == 1
            if (popcount64(S) & 1) acc = u256_sub(acc, prod);   /* planted: sign */
#else
            if ((n - popcount64(S)) & 1) acc = u256_sub(acc, prod);
#endif
            else acc = u256_add(acc, prod);
        }
        partial[c] = acc;
    }
    u256 total = u256_from_i64(0);
    for (uint64_t c = 0; c < nchunks; c++) total = u256_add(total, partial[c]);
    free(partial);
    u256_store(total, out);
    return ORACLE_OK;
}

/* a: n*n complex entries, row-major interleaved (re, im).  out: re_hi, re_lo, im_hi, im_lo.
   Row sums, products and the accumulator are all double-double. */
int oracle_per_ryser_c128(int n, const double *a, double *out, int nthreads) {
    if (n < 0 || n > 40 || (!a && n > 0) || !out) return ORACLE_EINVAL;
    if (n == 0) { cdd_store(cdd_from(1.0, 0.0), out); return ORACLE_OK; }
    const uint64_t total_codes = (uint64_t)1 << n;
    const uint64_t nchunks = (total_codes + RYSER_REFRESH - 1) / RYSER_REFRESH;
    cdd *partial = (cdd *)calloc(nchunks, sizeof(cdd));
    if (!partial) return ORACLE_EINVAL;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t c = 0; c < (int64_t)nchunks; c++) {
        uint64_t g0 = (uint64_t)c * RYSER_REFRESH;
        uint64_t g1 = g0 + RYSER_REFRESH < total_codes ? g0 + RYSER_REFRESH : total_codes;
        cdd rs[64];
        uint64_t S = gray(g0);
        for (int i = 0; i < n; i++) {
            cdd s = cdd_zero();
            for (int j = 0; j < n; j++)
                if ((S >> j) & 1u) s = cdd_add(s, cdd_from(a[2 * (i * n + j)], a[2 * (i * n + j) + 1]));
            rs[i] = s;
        }
        cdd acc = cdd_zero();
        for (uint64_t g = g0; g < g1; g++) {
            if (g > g0) {
                uint64_t Snew = gray(g);
                uint64_t diff = Snew ^ S;
                int j = 0;
                while (!((diff >> j) & 1u)) j++;
                int added = (Snew >> j) & 1u;
                for (int i = 0; i < n; i++) {
                    cdd e = cdd_from(a[2 * (i * n + j)], a[2 * (i * n + j) + 1]);
                    rs[i] = added ? cdd_add(rs[i], e) : cdd_sub(rs[i], e);
                }
                S = Snew;
            }
            cdd prod = rs[0];
            for (int i = 1; i < n; i++) prod = cdd_mul(prod, rs[i]);
            if ((n - popcount64(S)) & 1) acc = cdd_sub(acc, prod);
            else acc = cdd_add(acc, prod);
        }
        partial[c] = acc;
    }
    cdd total = cdd_zero();
    for (uint64_t c = 0; c < nchunks; c++) total = cdd_add(total, partial[c]);
    free(partial);
    cdd_store(total, out);
    return ORACLE_OK;
}

/* Number of OpenMP threads a parallel region would use (1 without OpenMP). */
int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
