/*
 * oracle.h -- CPU oracle for twofold summation (E. Latkin, "Twofold fast
 * summation", 2013).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this code; only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or constant with
 * the CUDA path.
 *
 * Contents
 *   1. Error-free transforms (Thm 1 Dekker FAST-TWO-SUM, Thm 2 Knuth TWO-SUM,
 *      and TwoProduct written from its definition p = RN(ab), e = RN(ab - p)
 *      with the exact product formed in integer arithmetic).
 *   2. The paper's sequential loops: sum, sumd, sumk, sumtf, sumt (Examples
 *      1-3 and the double-accumulator listing in section "Algorithms") and the
 *      dot-product forms (the product of the i-th elements as the item),
 *      plus the TwoProduct dot forms.
 *   3. An exact fixed-point superaccumulator: the plain definition S = sum x_i
 *      (or sum x_i*y_i with unrounded products) as an exact real, rounded once.
 *   4. An order replay ("emulator") of the kernels' documented reduction order,
 *      built from the same per-item steps as section 2 and the TwoSum merge.
 *
 * Floating point: compiled with -ffp-contract=off -fno-fast-math so that every
 * + - * is one IEEE-754 binary32/binary64 operation rounded to nearest even.
 */
#ifndef TWOFOLD_ORACLE_H
#define TWOFOLD_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* dtype codes */
#define ORC_F32 0
#define ORC_F64 1

/* ---- 1. primitives, elementwise over arrays --------------------------- */
void orc_fast_two_sum_f32(const float* a, const float* b, int64_t n, float* x, float* y);
void orc_fast_two_sum_f64(const double* a, const double* b, int64_t n, double* x, double* y);
void orc_two_sum_f32(const float* a, const float* b, int64_t n, float* x, float* y);
void orc_two_sum_f64(const double* a, const double* b, int64_t n, double* x, double* y);
void orc_two_product_f32(const float* a, const float* b, int64_t n, float* p, float* e);
void orc_two_product_f64(const double* a, const double* b, int64_t n, double* p, double* e);

/* ---- 2. the paper's sequential loops ---------------------------------- */
/* out[0] = value, out[1] = error (0 for single-output methods) */
void orc_sum_f32(int64_t m, const float* d, float out[2]);
void orc_sumk_f32(int64_t m, const float* d, float out[2]);
void orc_sumtf_f32(int64_t m, const float* d, float out[2]);
void orc_sumt_f32(int64_t m, const float* d, float out[2]);
double orc_sumd_f32(int64_t m, const float* d);
void orc_sum_f64(int64_t m, const double* d, double out[2]);
void orc_sumk_f64(int64_t m, const double* d, double out[2]);
void orc_sumtf_f64(int64_t m, const double* d, double out[2]);
void orc_sumt_f64(int64_t m, const double* d, double out[2]);
/* binary128 accumulator for double data (the paper's __float128 'sumd');
   returns the accumulator rounded to double, and its residual. */
void orc_sumq_f64(int64_t m, const double* d, double out[2]);

/* dot forms with the rounded product a[i]*b[i] (paper, literal) */
void orc_dot_f32(int64_t m, const float* a, const float* b, float out[2]);
void orc_dotk_f32(int64_t m, const float* a, const float* b, float out[2]);
void orc_dottf_f32(int64_t m, const float* a, const float* b, float out[2]);
void orc_dott_f32(int64_t m, const float* a, const float* b, float out[2]);
void orc_dot_f64(int64_t m, const double* a, const double* b, double out[2]);
void orc_dotk_f64(int64_t m, const double* a, const double* b, double out[2]);
void orc_dottf_f64(int64_t m, const double* a, const double* b, double out[2]);
void orc_dott_f64(int64_t m, const double* a, const double* b, double out[2]);
/* double accumulator, product formed in double (exact for binary32 operands) */
double orc_dotd_f32(int64_t m, const float* a, const float* b);
/* TwoProduct forms: the product's rounding error joins the error term */
void orc_dottf2_f32(int64_t m, const float* a, const float* b, float out[2]);
void orc_dott2_f32(int64_t m, const float* a, const float* b, float out[2]);
void orc_dottf2_f64(int64_t m, const double* a, const double* b, double out[2]);
void orc_dott2_f64(int64_t m, const double* a, const double* b, double out[2]);

/* ---- 3. exact superaccumulator ----------------------------------------- */
typedef struct {
    double s;      /* RN64(S)                                   */
    double s_lo;   /* RN64(S - RN64(S))                          */
    double sabs;   /* RN64(sum of |terms|)                       */
    double rv;     /* RN64(S - v)                                */
    double r;      /* RN64(S - v - e)                            */
    float  s32;    /* RN32(S), one rounding                      */
    int32_t cls;   /* 0 finite, 1 NaN, 2 +Inf, 3 -Inf            */
} orc_exact_t;

/* y == NULL -> sum of x; else sum of x[i]*y[i] with exact products.
   v, e: the pair whose residuals are reported (pass 0, 0 if none).
   nthreads <= 0 -> all online cores.  Returns 0, or -1 on bad arguments. */
int orc_exact(int dtype, const void* x, const void* y, int64_t n,
              double v, double e, int nthreads, orc_exact_t* out);
/* per CSR segment [off[s], off[s+1]); v, e may be NULL */
int orc_exact_batched(int dtype, const void* x, const void* y, const int64_t* off,
                      int64_t nseg, const double* v, const double* e, int nthreads,
                      orc_exact_t* out);
/* round an exact sum of the doubles t[0..k) once (used to form v+e exactly) */
double orc_exact_add_doubles(const double* t, int k);

/* ---- 4. replay of the kernels' reduction order ------------------------- */
/* op: 0 sum, 1 dot.  variant: 0 plain, 1 fast ('tf'), 2 rigorous ('t'),
   3 wide ('d', binary32 data with binary64 accumulation), 4 kahan ('k',
   Example 2), 5 fast and 6 rigorous dots with the paper's rounded product
   (no TwoProduct term).
   out_f64 != 0 returns the binary64 grid-fold pair for binary32 data.
   out: two values of the output type (float or double). */
int orc_replay_flat(int dtype, int op, int variant, const void* x, const void* y,
                    int64_t n, int block, int unroll, int64_t grid, int out_f64,
                    void* out);
int orc_replay_csr(int dtype, int op, int variant, const void* x, const void* y,
                   const int64_t* off, int64_t nseg, int unroll, int64_t tile,
                   int out_f64, int nthreads, void* out);
/* merge of G shard pairs (binary64 (V, E) each) in rank order, output as the
   reductions write theirs (see replay.c) */
int orc_merge_pairs(int dtype, int variant, const double* pairs, int64_t G, int out_f64,
                    void* out);

#ifdef __cplusplus
}
#endif
#endif
