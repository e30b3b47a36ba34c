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
 *   dot*   the same loops with the product of the i-th elements as the item
 *          (end of the Algorithms section), rounded to the data type.
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
/* One item y of each loop, on the state (s, e).  The twofold steps are the
   error-free transforms the paper bases them on: Example 1 moves s by
   FAST-TWO-SUM (Theorem 1) and collects the transform's error term in e (the
   paper writes the correction as c = -term and subtracts it; the two agree
   bit for bit because e is never -0); Example 3 does the same with TWO-SUM
   (Theorem 2), whose error term is the paper's ds + dy.  Kahan's step
   (Example 2) carries the correction c into the next item. */
#define DEF_STEPS(T, SUF)                                                     \
static inline void fast_item_##SUF(T* s, T* e, T y, T ep, int with_ep) {      \
    T t, term;                                                                \
    orc_fts_##SUF(*s, y, &t, &term);                                          \
    *e = with_ep ? *e + (ep + term) : *e + term;                              \
    *s = t;                                                                   \
}                                                                             \
static inline void rigorous_item_##SUF(T* s, T* e, T y, T ep, int with_ep) {  \
    T t, term;                                                                \
    orc_ts_##SUF(*s, y, &t, &term);                                           \
    *e = with_ep ? *e + (term + ep) : *e + term;                              \
    *s = t;                                                                   \
}                                                                             \
static inline void kahan_item_##SUF(T* s, T* c, T y) {                        \
    const T corrected = y - *c;          /* the item with last step's loss */ \
    const T t = *s + corrected;                                               \
    *c = (t - *s) - corrected;           /* what t failed to absorb */        \
    *s = t;                                                                   \
}
DEF_STEPS(float, f32)
DEF_STEPS(double, f64)

#define DEF_SUMS(T, SUF)                                                      \
void orc_sum_##SUF(int64_t m, const T* data, T out[2]) {                      \
    T acc = 0;                                                                \
    for (int64_t i = 0; i < m; i++) acc = acc + data[i];                      \
    out[0] = acc; out[1] = 0;                                                 \
}                                                                             \
void orc_sumk_##SUF(int64_t m, const T* data, T out[2]) {                     \
    T s = 0, c = 0;                                                           \
    for (int64_t i = 0; i < m; i++) kahan_item_##SUF(&s, &c, data[i]);        \
    out[0] = s; out[1] = 0 - c;  /* the sum, and the compensation still owed */ \
}                                                                             \
void orc_sumtf_##SUF(int64_t m, const T* data, T out[2]) {                    \
    T s = 0, e = 0;                                                           \
    for (int64_t i = 0; i < m; i++) fast_item_##SUF(&s, &e, data[i], 0, 0);     \
    out[0] = s; out[1] = e;                                                   \
}                                                                             \
void orc_sumt_##SUF(int64_t m, const T* data, T out[2]) {                     \
    T s = 0, e = 0;                                                           \
    for (int64_t i = 0; i < m; i++) rigorous_item_##SUF(&s, &e, data[i], 0, 0); \
    out[0] = s; out[1] = e;                                                   \
}
DEF_SUMS(float, f32)
DEF_SUMS(double, f64)

/* the wider accumulators: each binary32 item widens exactly to binary64
   (each binary64 item to binary128) before the one rounded add */
double orc_sumd_f32(int64_t m, const float* data) {
    double acc = 0.0;
    for (int64_t i = 0; i < m; i++) acc = acc + (double)data[i];
    return acc;
}

void orc_sumq_f64(int64_t m, const double* data, double out[2]) {
    _Float128 acc = 0;
    for (int64_t i = 0; i < m; i++) acc = acc + (_Float128)data[i];
    const double hi = (double)acc;
    out[0] = hi;
    out[1] = (double)(acc - (_Float128)hi);
}

/* ------------------------------------------------------------------ dots */
/* The dot loops take the product of the i-th elements as the loop's item
   (the paper's remark at the end of the Algorithms section): rounded to the
   data type (dot, dotk, dottf, dott), or split by TwoProduct into p and its
   exact error ep, p feeding the step and ep joining the error term as
   e <- e + (term + ep) (dottf2, dott2). */
#define DEF_DOTS(T, SUF)                                                      \
void orc_dot_##SUF(int64_t m, const T* a, const T* b, T out[2]) {             \
    T acc = 0;                                                                \
    for (int64_t i = 0; i < m; i++) { const T p = a[i] * b[i]; acc = acc + p; } \
    out[0] = acc; out[1] = 0;                                                 \
}                                                                             \
void orc_dotk_##SUF(int64_t m, const T* a, const T* b, T out[2]) {            \
    T s = 0, c = 0;                                                           \
    for (int64_t i = 0; i < m; i++) kahan_item_##SUF(&s, &c, a[i] * b[i]);    \
    out[0] = s; out[1] = 0 - c;                                               \
}                                                                             \
void orc_dottf_##SUF(int64_t m, const T* a, const T* b, T out[2]) {           \
    T s = 0, e = 0;                                                           \
    for (int64_t i = 0; i < m; i++) fast_item_##SUF(&s, &e, a[i] * b[i], 0, 0);  \
    out[0] = s; out[1] = e;                                                   \
}                                                                             \
void orc_dott_##SUF(int64_t m, const T* a, const T* b, T out[2]) {            \
    T s = 0, e = 0;                                                           \
    for (int64_t i = 0; i < m; i++) rigorous_item_##SUF(&s, &e, a[i] * b[i], 0, 0); \
    out[0] = s; out[1] = e;                                                   \
}                                                                             \
void orc_dottf2_##SUF(int64_t m, const T* a, const T* b, T out[2]) {          \
    T s = 0, e = 0;                                                           \
    for (int64_t i = 0; i < m; i++) {                                         \
        T p, ep;                                                              \
        orc_two_product_##SUF(&a[i], &b[i], 1, &p, &ep);                      \
        fast_item_##SUF(&s, &e, p, ep, 1);                                       \
    }                                                                         \
    out[0] = s; out[1] = e;                                                   \
}                                                                             \
void orc_dott2_##SUF(int64_t m, const T* a, const T* b, T out[2]) {           \
    T s = 0, e = 0;                                                           \
    for (int64_t i = 0; i < m; i++) {                                         \
        T p, ep;                                                              \
        orc_two_product_##SUF(&a[i], &b[i], 1, &p, &ep);                      \
        rigorous_item_##SUF(&s, &e, p, ep, 1);                                \
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
