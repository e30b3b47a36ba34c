/*
 * loops.c -- the paper's sequential summation loops, one element at a time,
 * in the paper's order and notation.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 *   sumtf  twofold fast summation ........ Example 1 (Dekker based)
 *   sumk   Kahan compensated summation ... Example 2 (returns the sum and,
 *                                          as a second output, -c: the
 *                                          compensation not yet applied)
 *   sumt   twofold rigorous summation .... Example 3 (Knuth based, as fixed
 *                                          in the 31-Dec-2013 revision)
 *   sum    direct summation .............. Example 3
 *   sumd   double accumulator, float data  listing after Example 3
 *   sumq   binary128 accumulator for double data: the paper's __float128
 *          comparison (Performance section, "sumd" for double)
 *   dot*   "multiplication like a[i]*b[i] in place of data[i]" (end of the
 *          Algorithms section): the product is rounded to the data type.
 *   dottf2, dott2: the same loops with TwoProduct: p = RN(a*b) feeds the sum
 *          and its exact rounding error ep joins the error term,
 *          e <- e + (q + ep) where q is the sum step's own error.
 *   dotd   double accumulator; the product of two binary32 numbers is formed
 *          in binary64, where it is exact.
 *
 * All operations are plain IEEE + - * in the data type (no contraction).
 */
#include "oracle.h"
#include "orc_internal.h"

/* ------------------------------------------------------------------ sums */
#define DEF_SUMS(T, SUF)                                                      \
void orc_sum_##SUF(int64_t m, const T* data, T out[2]) {                      \
    T s = 0;                                                                  \
    for (int64_t i = 0; i < m; i++)                                           \
        s += data[i];                                                         \
    out[0] = s; out[1] = 0;                                                   \
}                                                                             \
void orc_sumk_##SUF(int64_t m, const T* data, T out[2]) {                     \
    T s = 0, c = 0;                                                           \
    for (int64_t i = 0; i < m; i++) {                                         \
        T y, t;                                                               \
        y = data[i] - c;                                                      \
        t = s + y;                                                            \
        c = (t - s) - y;                                                      \
        s = t;                                                                \
    }                                                                         \
    out[0] = s; out[1] = 0 - c;  /* the sum, and the compensation still owed */ \
}                                                                             \
void orc_sumtf_##SUF(int64_t m, const T* data, T out[2]) {                    \
    T s = 0, e = 0;                                                           \
    for (int64_t i = 0; i < m; i++) {                                         \
        T y, t, c;                                                            \
        y = data[i];                                                          \
        t = s + y;                                                            \
        c = (t - s) - y;                                                      \
        e = e - c;                                                            \
        s = t;                                                                \
    }                                                                         \
    out[0] = s; out[1] = e;                                                   \
}                                                                             \
void orc_sumt_##SUF(int64_t m, const T* data, T out[2]) {                     \
    T s = 0, e = 0;                                                           \
    for (int64_t i = 0; i < m; i++) {                                         \
        T t, y, yt, dy, ds;                                                   \
        y = data[i];                                                          \
        t = s + y;                                                            \
        yt = t - s;                                                           \
        dy = y - yt;                                                          \
        ds = s - (t - yt);                                                    \
        e += ds + dy;                                                         \
        s = t;                                                                \
    }                                                                         \
    out[0] = s; out[1] = e;                                                   \
}
DEF_SUMS(float, f32)
DEF_SUMS(double, f64)

double orc_sumd_f32(int64_t m, const float* data) {
    double s = 0;
    for (int64_t i = 0; i < m; i++)
        s += data[i];
    return s;
}

void orc_sumq_f64(int64_t m, const double* data, double out[2]) {
    _Float128 s = 0;
    for (int64_t i = 0; i < m; i++)
        s += data[i];
    double hi = (double)s;
    out[0] = hi;
    out[1] = (double)(s - (_Float128)hi);
}

/* ------------------------------------------------- dots, rounded product */
#define DEF_DOTS(T, SUF)                                                      \
void orc_dot_##SUF(int64_t m, const T* a, const T* b, T out[2]) {             \
    T s = 0;                                                                  \
    for (int64_t i = 0; i < m; i++) {                                         \
        T y = a[i] * b[i];                                                    \
        s += y;                                                               \
    }                                                                         \
    out[0] = s; out[1] = 0;                                                   \
}                                                                             \
void orc_dotk_##SUF(int64_t m, const T* a, const T* b, T out[2]) {            \
    T s = 0, c = 0;                                                           \
    for (int64_t i = 0; i < m; i++) {                                         \
        T y, t;                                                               \
        T ab = a[i] * b[i];                                                   \
        y = ab - c;                                                           \
        t = s + y;                                                            \
        c = (t - s) - y;                                                      \
        s = t;                                                                \
    }                                                                         \
    out[0] = s; out[1] = 0 - c;                                               \
}                                                                             \
void orc_dottf_##SUF(int64_t m, const T* a, const T* b, T out[2]) {           \
    T s = 0, e = 0;                                                           \
    for (int64_t i = 0; i < m; i++) {                                         \
        T y, t, c;                                                            \
        y = a[i] * b[i];                                                      \
        t = s + y;                                                            \
        c = (t - s) - y;                                                      \
        e = e - c;                                                            \
        s = t;                                                                \
    }                                                                         \
    out[0] = s; out[1] = e;                                                   \
}                                                                             \
void orc_dott_##SUF(int64_t m, const T* a, const T* b, T out[2]) {            \
    T s = 0, e = 0;                                                           \
    for (int64_t i = 0; i < m; i++) {                                         \
        T t, y, yt, dy, ds;                                                   \
        y = a[i] * b[i];                                                      \
        t = s + y;                                                            \
        yt = t - s;                                                           \
        dy = y - yt;                                                          \
        ds = s - (t - yt);                                                    \
        e += ds + dy;                                                         \
        s = t;                                                                \
    }                                                                         \
    out[0] = s; out[1] = e;                                                   \
}                                                                             \
void orc_dottf2_##SUF(int64_t m, const T* a, const T* b, T out[2]) {          \
    T s = 0, e = 0;                                                           \
    for (int64_t i = 0; i < m; i++) {                                         \
        T y, ep, t, c;                                                        \
        orc_two_product_##SUF(&a[i], &b[i], 1, &y, &ep);                      \
        t = s + y;                                                            \
        c = (t - s) - y;                                                      \
        e = e + (ep - c);        /* q = -c is the sum step's error */         \
        s = t;                                                                \
    }                                                                         \
    out[0] = s; out[1] = e;                                                   \
}                                                                             \
void orc_dott2_##SUF(int64_t m, const T* a, const T* b, T out[2]) {           \
    T s = 0, e = 0;                                                           \
    for (int64_t i = 0; i < m; i++) {                                         \
        T t, y, ep, yt, dy, ds;                                               \
        orc_two_product_##SUF(&a[i], &b[i], 1, &y, &ep);                      \
        t = s + y;                                                            \
        yt = t - s;                                                           \
        dy = y - yt;                                                          \
        ds = s - (t - yt);                                                    \
        e += (ds + dy) + ep;                                                  \
        s = t;                                                                \
    }                                                                         \
    out[0] = s; out[1] = e;                                                   \
}
DEF_DOTS(float, f32)
DEF_DOTS(double, f64)

double orc_dotd_f32(int64_t m, const float* a, const float* b) {
    double s = 0;
    for (int64_t i = 0; i < m; i++)
        s += (double)a[i] * (double)b[i];
    return s;
}
