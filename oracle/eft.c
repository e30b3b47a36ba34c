/*
 * eft.c -- error-free transforms, written from their statements.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * FAST-TWO-SUM: Theorem 1 (Dekker), section "Algorithms".  Exact when |a|>=|b|.
 * TWO-SUM:      Theorem 2 (Knuth), section "Algorithms".  Exact for all finite
 *               a, b whose sum does not overflow.
 * TwoProduct:   not in the paper; its definition p = RN(a*b), e = RN(a*b - p).
 *               Here the exact product is formed from the integer significands
 *               (no fused multiply-add is used), then rounded twice by
 *               round-to-nearest-even.
 */
#include "oracle.h"
#include "orc_internal.h"
#include <math.h>
#include <string.h>

#define DEF_SUM_ARRAYS(T, SUF)                                               \
void orc_fast_two_sum_##SUF(const T* a, const T* b, int64_t n, T* x, T* y) { \
    for (int64_t i = 0; i < n; ++i) orc_fts_##SUF(a[i], b[i], &x[i], &y[i]); \
}                                                                            \
void orc_two_sum_##SUF(const T* a, const T* b, int64_t n, T* x, T* y) {      \
    for (int64_t i = 0; i < n; ++i) orc_ts_##SUF(a[i], b[i], &x[i], &y[i]);  \
}
DEF_SUM_ARRAYS(float, f32)
DEF_SUM_ARRAYS(double, f64)

/* ---- TwoProduct from the definition --------------------------------- */

static int bitlen128(u128 m) {
    int n = 0;
    uint64_t hi = (uint64_t)(m >> 64);
    if (hi) { n = 64; m = hi; }
    uint64_t lo = (uint64_t)m;
    while (lo) { ++n; lo >>= 1; }
    return n;
}

/* Round +M*2^K to `prec` significant bits, round-to-nearest-even, with the
   quantum never below 2^emin_lsb (gradual underflow).  Returns the value as a
   double (exact: the result has at most prec <= 53 bits); overflow beyond
   the double range gives +Inf, and callers narrow to float where needed. */
double orc_round_mk(u128 M, int K, int prec, int emin_lsb, u128* Mr, int* R) {
    if (M == 0) { if (Mr) *Mr = 0; if (R) *R = K; return 0.0; }
    int nb = bitlen128(M);
    int top = K + nb - 1;                 /* exponent of the leading bit */
    int r = top - prec + 1;
    if (r < emin_lsb) r = emin_lsb;
    u128 q;
    if (r <= K) {                         /* representable as is */
        q = M; r = K;
    } else {
        int sh = r - K;                   /* number of dropped bits, >= 1 */
        if (sh > 128) {
            q = 0;                        /* below half of the quantum */
        } else {
            q = (sh == 128) ? 0 : (M >> sh);
            u128 rem = (sh == 128) ? M : (M - (q << sh));
            u128 half = (u128)1 << (sh - 1);
            if (rem > half || (rem == half && (q & 1))) q += 1;
        }
    }
    if (Mr) *Mr = q;
    if (R) *R = r;
    return ldexp((double)q, r);           /* q <= 2^prec: exact conversion */
}

/* one TwoProduct in a binary format with `prec` bits, lowest quantum
   2^emin_lsb and largest finite < 2^(emax+1) */
static void two_product_exact(int na, uint64_t ma, int ka, int nb_, uint64_t mb, int kb,
                              int prec, int emin_lsb, int emax, double* p, double* e) {
    int neg = na ^ nb_;
    u128 M = (u128)ma * (u128)mb;
    int K = ka + kb;
    if (M == 0) { *p = neg ? -0.0 : 0.0; *e = 0.0; return; }
    u128 Mp; int Rp;
    double pv = orc_round_mk(M, K, prec, emin_lsb, &Mp, &Rp);
    if (ldexp(1.0, emax + 1) <= pv) {     /* RN overflows to infinity */
        *p = neg ? -INFINITY : INFINITY;
        *e = neg ? INFINITY : -INFINITY;  /* a*b - p, with p infinite */
        return;
    }
    /* exact residual M*2^K - Mp*2^Rp; Rp >= K whenever rounding happened */
    *p = neg ? -pv : pv;
    *e = 0.0;                             /* exact product: +0 residual */
    if (Rp > K) {
        /* Mp*2^Rp lies within one quantum of M*2^K, so the shift fits unless
           Mp == 0 (total underflow), where the shift amount is unbounded */
        u128 Ms = (Mp == 0) ? 0 : (Mp << (Rp - K));
        u128 D; int eneg;
        if (M >= Ms) { D = M - Ms; eneg = 0; } else { D = Ms - M; eneg = 1; }
        if (D != 0) {
            double ev = orc_round_mk(D, K, prec, emin_lsb, NULL, NULL);
            /* a nonzero residual keeps its sign even when it rounds to zero */
            *e = (neg ^ eneg) ? -ev : ev;
        }
    }
}

void orc_two_product_f32(const float* a, const float* b, int64_t n, float* p, float* e) {
    for (int64_t i = 0; i < n; ++i) {
        int na, nb_, ca, cb, ka, kb; uint64_t ma, mb;
        orc_decompose_f32(a[i], &na, &ma, &ka, &ca);
        orc_decompose_f32(b[i], &nb_, &mb, &kb, &cb);
        if (ca || cb) {                   /* IEEE special operands */
            float pi = a[i] * b[i];
            p[i] = pi; e[i] = pi - pi;    /* NaN for Inf/NaN products */
            continue;
        }
        double pv, ev;
        two_product_exact(na, ma, ka, nb_, mb, kb, 24, -149, 127, &pv, &ev);
        p[i] = (float)pv; e[i] = (float)ev;   /* both exact narrowings */
    }
}

void orc_two_product_f64(const double* a, const double* b, int64_t n, double* p, double* e) {
    for (int64_t i = 0; i < n; ++i) {
        int na, nb_, ca, cb, ka, kb; uint64_t ma, mb;
        orc_decompose_f64(a[i], &na, &ma, &ka, &ca);
        orc_decompose_f64(b[i], &nb_, &mb, &kb, &cb);
        if (ca || cb) {
            double pi = a[i] * b[i];
            p[i] = pi; e[i] = pi - pi;
            continue;
        }
        two_product_exact(na, ma, ka, nb_, mb, kb, 53, -1074, 1023, &p[i], &e[i]);
    }
}
