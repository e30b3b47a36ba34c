/*
 * exact.c -- exact fixed-point superaccumulator.  TEST INFRASTRUCTURE ONLY.
 *
 * This is the plain definition of what twofold summation approximates: the
 * exact real S = sum x_i (or sum x_i*y_i with unrounded products), the target
 * that *value* + *error* estimates (Overview; Accuracy section).  It is
 * computed without any floating-point arithmetic:
 *
 *   every finite binary32/binary64 number is (-1)^s * m * 2^k with an integer
 *   significand m; a product of two such numbers is (-1)^(s1+s2) * (m1*m2) *
 *   2^(k1+k2) with m1*m2 formed exactly in 128-bit integers.  Each term is
 *   added at bit offset k into an array of 32-bit digits held in signed 64-bit
 *   words (so up to 2^31 terms can be added between carry propagations).  The
 *   digit array spans 2^-2208 .. 2^2272, which holds every binary64 product
 *   (lowest bit 2^-2148) and the sum of up to 2^64 of them.
 *
 * Rounding to binary32/binary64 happens once, at the end, to nearest even
 * with gradual underflow.  Partial accumulators of different threads are
 * added digit by digit, so the result does not depend on the thread count.
 */
#include "oracle.h"
#include "orc_internal.h"
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ACC_LSB  (-2208)
#define ACC_NDIG 140
#define ACC_RENORM (1LL << 30)

typedef struct {
    int64_t d[ACC_NDIG];
    int64_t pending;
    int nan, pinf, ninf;
} acc_t;

static void acc_init(acc_t* a) { memset(a, 0, sizeof(*a)); }

static void acc_normalize(acc_t* a) {
    int64_t carry = 0;
    for (int i = 0; i < ACC_NDIG - 1; ++i) {
        int64_t v = a->d[i] + carry;
        carry = v >> 32;                       /* floor division by 2^32 */
        a->d[i] = v - (carry * ((int64_t)1 << 32));
    }
    a->d[ACC_NDIG - 1] += carry;
    a->pending = 0;
}

/* add (-1)^neg * M * 2^K, M < 2^107 */
static inline void acc_add(acc_t* a, u128 M, int K, int neg) {
    int shift = K - ACC_LSB;
    int i = shift >> 5, r = shift & 31;
    u128 lo = M << r;
    uint64_t hi = r ? (uint64_t)(M >> (128 - r)) : 0;
    int64_t d0 = (int64_t)(uint32_t)lo;
    int64_t d1 = (int64_t)(uint32_t)(lo >> 32);
    int64_t d2 = (int64_t)(uint32_t)(lo >> 64);
    int64_t d3 = (int64_t)(uint32_t)(lo >> 96);
    int64_t d4 = (int64_t)hi;
    if (neg) { a->d[i] -= d0; a->d[i+1] -= d1; a->d[i+2] -= d2; a->d[i+3] -= d3; a->d[i+4] -= d4; }
    else     { a->d[i] += d0; a->d[i+1] += d1; a->d[i+2] += d2; a->d[i+3] += d3; a->d[i+4] += d4; }
    if (++a->pending >= ACC_RENORM) acc_normalize(a);
}

static void acc_merge(acc_t* dst, acc_t* src) {
    acc_normalize(dst); acc_normalize(src);
    for (int i = 0; i < ACC_NDIG; ++i) dst->d[i] += src->d[i];
    dst->nan |= src->nan; dst->pinf |= src->pinf; dst->ninf |= src->ninf;
    acc_normalize(dst);
}

static int acc_class(const acc_t* a) {
    if (a->nan || (a->pinf && a->ninf)) return 1;
    if (a->pinf) return 2;
    if (a->ninf) return 3;
    return 0;
}

static void acc_add_double(acc_t* a, double x) {
    int neg, k, cls; uint64_t m;
    orc_decompose_f64(x, &neg, &m, &k, &cls);
    if (cls == 1) { a->nan = 1; return; }
    if (cls == 2) { if (neg) a->ninf = 1; else a->pinf = 1; return; }
    if (m) acc_add(a, (u128)m, k, neg);
}

/* bit at absolute exponent e of the non-negative normalized magnitude */
static int mag_bit(const int64_t* d, int e) {
    int off = e - ACC_LSB;
    if (off < 0) return 0;
    int i = off >> 5, b = off & 31;
    if (i >= ACC_NDIG) return 0;
    return (int)((d[i] >> b) & 1);
}

static int mag_any_below(const int64_t* d, int e) {  /* any bit at exponent < e */
    int off = e - ACC_LSB;
    if (off <= 0) return 0;
    int i = off >> 5, b = off & 31;
    for (int j = 0; j < i && j < ACC_NDIG; ++j) if (d[j]) return 1;
    if (i < ACC_NDIG && b && (d[i] & (((int64_t)1 << b) - 1))) return 1;
    return 0;
}

/* Round the accumulated value once to `prec` bits with quantum >= 2^emin_lsb.
   Returns the rounded value as a double (Inf when out of the double range;
   callers narrow binary32 results, which are exact or overflow to Inf). */
static double acc_round(const acc_t* src, int prec, int emin_lsb) {
    int cls = acc_class(src);
    if (cls == 1) return NAN;
    if (cls == 2) return INFINITY;
    if (cls == 3) return -INFINITY;
    acc_t a = *src;
    acc_normalize(&a);
    int neg = a.d[ACC_NDIG - 1] < 0;
    if (neg) {
        for (int i = 0; i < ACC_NDIG; ++i) a.d[i] = -a.d[i];
        acc_normalize(&a);
    }
    int h = ACC_NDIG - 1;
    while (h >= 0 && a.d[h] == 0) --h;
    if (h < 0) return 0.0;
    int b = 63; while (!((a.d[h] >> b) & 1)) --b;
    int top = ACC_LSB + 32 * h + b;
    int r = top - prec + 1;
    if (r < emin_lsb) r = emin_lsb;
    uint64_t q = 0;
    for (int e = top; e >= r; --e) q = (q << 1) | (uint64_t)mag_bit(a.d, e);
    int half = mag_bit(a.d, r - 1);
    int sticky = mag_any_below(a.d, r - 1);
    if (half && (sticky || (q & 1))) q += 1;
    double v = ldexp((double)q, r);
    return neg ? -v : v;
}

/* ---------------------------------------------------------- term loops */

typedef struct {
    int dtype;
    const void* x; const void* y;
    int64_t lo, hi;
    int want_abs;
    acc_t acc, aabs;
} job_t;

static void add_term_sum_f64(acc_t* a, acc_t* aa, double x, int want_abs) {
    int neg, k, cls; uint64_t m;
    orc_decompose_f64(x, &neg, &m, &k, &cls);
    if (cls) {
        if (cls == 1) a->nan = 1; else if (neg) a->ninf = 1; else a->pinf = 1;
        return;
    }
    if (!m) return;
    acc_add(a, (u128)m, k, neg);
    if (want_abs) acc_add(aa, (u128)m, k, 0);
}

static void add_term_sum_f32(acc_t* a, acc_t* aa, float x, int want_abs) {
    int neg, k, cls; uint64_t m;
    orc_decompose_f32(x, &neg, &m, &k, &cls);
    if (cls) {
        if (cls == 1) a->nan = 1; else if (neg) a->ninf = 1; else a->pinf = 1;
        return;
    }
    if (!m) return;
    acc_add(a, (u128)m, k, neg);
    if (want_abs) acc_add(aa, (u128)m, k, 0);
}

static void add_term_prod(acc_t* a, acc_t* aa, int n1, uint64_t m1, int k1, int c1,
                          int n2, uint64_t m2, int k2, int c2, int want_abs) {
    int neg = n1 ^ n2;
    if (c1 || c2) {
        /* IEEE: NaN if either is NaN or Inf*0; otherwise a signed infinity */
        if (c1 == 1 || c2 == 1 || (c1 == 2 && c2 == 0 && m2 == 0) ||
            (c2 == 2 && c1 == 0 && m1 == 0)) a->nan = 1;
        else if (neg) a->ninf = 1; else a->pinf = 1;
        return;
    }
    if (!m1 || !m2) return;
    u128 M = (u128)m1 * (u128)m2;
    acc_add(a, M, k1 + k2, neg);
    if (want_abs) acc_add(aa, M, k1 + k2, 0);
}

static void run_range(job_t* j) {
    int64_t i;
    if (j->dtype == ORC_F64) {
        const double* x = (const double*)j->x; const double* y = (const double*)j->y;
        if (!y) {
            for (i = j->lo; i < j->hi; ++i) add_term_sum_f64(&j->acc, &j->aabs, x[i], j->want_abs);
        } else {
            for (i = j->lo; i < j->hi; ++i) {
                int n1, k1, c1, n2, k2, c2; uint64_t m1, m2;
                orc_decompose_f64(x[i], &n1, &m1, &k1, &c1);
                orc_decompose_f64(y[i], &n2, &m2, &k2, &c2);
                add_term_prod(&j->acc, &j->aabs, n1, m1, k1, c1, n2, m2, k2, c2, j->want_abs);
            }
        }
    } else {
        const float* x = (const float*)j->x; const float* y = (const float*)j->y;
        if (!y) {
            for (i = j->lo; i < j->hi; ++i) add_term_sum_f32(&j->acc, &j->aabs, x[i], j->want_abs);
        } else {
            for (i = j->lo; i < j->hi; ++i) {
                int n1, k1, c1, n2, k2, c2; uint64_t m1, m2;
                orc_decompose_f32(x[i], &n1, &m1, &k1, &c1);
                orc_decompose_f32(y[i], &n2, &m2, &k2, &c2);
                add_term_prod(&j->acc, &j->aabs, n1, m1, k1, c1, n2, m2, k2, c2, j->want_abs);
            }
        }
    }
}

static void* run_range_thread(void* p) { run_range((job_t*)p); return NULL; }

int orc_default_threads(void) {
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

static void fill_result(const acc_t* acc, const acc_t* aabs, double v, double e, orc_exact_t* out) {
    out->cls = acc_class(acc);
    out->s = acc_round(acc, 53, -1074);
    out->s32 = (float)acc_round(acc, 24, -149);
    out->sabs = acc_round(aabs, 53, -1074);
    acc_t t = *acc;
    acc_add_double(&t, -out->s);
    out->s_lo = acc_round(&t, 53, -1074);
    t = *acc;
    acc_add_double(&t, -v);
    out->rv = acc_round(&t, 53, -1074);
    acc_add_double(&t, -e);
    out->r = acc_round(&t, 53, -1074);
}

int orc_exact(int dtype, const void* x, const void* y, int64_t n,
              double v, double e, int nthreads, orc_exact_t* out) {
    if ((dtype != ORC_F32 && dtype != ORC_F64) || n < 0 || !out || (n > 0 && !x)) return -1;
    if (nthreads <= 0) nthreads = orc_default_threads();
    if (n < 65536) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    job_t* jobs = (job_t*)calloc((size_t)nthreads, sizeof(job_t));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return -1; }
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].dtype = dtype; jobs[t].x = x; jobs[t].y = y; jobs[t].want_abs = 1;
        jobs[t].lo = n * t / nthreads; jobs[t].hi = n * (t + 1) / nthreads;
        acc_init(&jobs[t].acc); acc_init(&jobs[t].aabs);
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, run_range_thread, &jobs[t]);
    run_range(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        acc_merge(&jobs[0].acc, &jobs[t].acc);
        acc_merge(&jobs[0].aabs, &jobs[t].aabs);
    }
    fill_result(&jobs[0].acc, &jobs[0].aabs, v, e, out);
    free(jobs); free(th);
    return 0;
}

/* ------------------------------------------------------------- batched */

typedef struct {
    int dtype; const void* x; const void* y; const int64_t* off; int64_t nseg;
    const double* v; const double* e; orc_exact_t* out;
    int64_t* next;
} bjob_t;

static void* run_batched(void* p) {
    bjob_t* b = (bjob_t*)p;
    job_t* j = (job_t*)malloc(sizeof(job_t));
    for (;;) {
        int64_t s = __atomic_fetch_add(b->next, 1, __ATOMIC_RELAXED);
        if (s >= b->nseg) break;
        j->dtype = b->dtype; j->x = b->x; j->y = b->y; j->want_abs = 1;
        j->lo = b->off[s]; j->hi = b->off[s + 1];
        acc_init(&j->acc); acc_init(&j->aabs);
        run_range(j);
        fill_result(&j->acc, &j->aabs, b->v ? b->v[s] : 0.0, b->e ? b->e[s] : 0.0, &b->out[s]);
    }
    free(j);
    return NULL;
}

int orc_exact_batched(int dtype, const void* x, const void* y, const int64_t* off,
                      int64_t nseg, const double* v, const double* e, int nthreads,
                      orc_exact_t* out) {
    if ((dtype != ORC_F32 && dtype != ORC_F64) || nseg < 0 || !off || !out) return -1;
    for (int64_t s = 0; s < nseg; ++s) if (off[s + 1] < off[s] || off[s] < 0) return -1;
    if (nthreads <= 0) nthreads = orc_default_threads();
    if (nthreads > 256) nthreads = 256;
    int64_t next = 0;
    bjob_t b = { dtype, x, y, off, nseg, v, e, out, &next };
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!th) return -1;
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, run_batched, &b);
    run_batched(&b);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    return 0;
}

double orc_exact_add_doubles(const double* t, int k) {
    acc_t a; acc_init(&a);
    for (int i = 0; i < k; ++i) acc_add_double(&a, t[i]);
    return acc_round(&a, 53, -1074);
}
