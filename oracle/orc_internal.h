/* orc_internal.h -- helpers private to the oracle (test infrastructure only). */
#ifndef TWOFOLD_ORC_INTERNAL_H
#define TWOFOLD_ORC_INTERNAL_H
#include <stdint.h>
#include <string.h>

typedef unsigned __int128 u128;

double orc_round_mk(u128 M, int K, int prec, int emin_lsb, u128* Mr, int* R);
int orc_default_threads(void);

/* sign, integer significand, exponent of the last significand bit, and class
   (0 finite, 1 NaN, 2 infinite) of a binary32 / binary64 number */
static inline void orc_decompose_f32(float a, int* neg, uint64_t* m, int* k, int* cls) {
    uint32_t u; memcpy(&u, &a, 4);
    *neg = (int)(u >> 31);
    int be = (int)((u >> 23) & 0xff);
    uint32_t f = u & 0x7fffffu;
    if (be == 0xff) { *cls = f ? 1 : 2; *m = 0; *k = 0; return; }
    *cls = 0;
    if (be == 0) { *m = f; *k = -149; }
    else { *m = f | 0x800000u; *k = be - 150; }
}

static inline void orc_decompose_f64(double a, int* neg, uint64_t* m, int* k, int* cls) {
    uint64_t u; memcpy(&u, &a, 8);
    *neg = (int)(u >> 63);
    int be = (int)((u >> 52) & 0x7ff);
    uint64_t f = u & 0xfffffffffffffull;
    if (be == 0x7ff) { *cls = f ? 1 : 2; *m = 0; *k = 0; return; }
    *cls = 0;
    if (be == 0) { *m = f; *k = -1074; }
    else { *m = f | (1ull << 52); *k = be - 1075; }
}

/* The two sum transforms on one pair, written from the theorems (section
   "Algorithms"): Dekker's FAST-TWO-SUM (Theorem 1) and Knuth's TWO-SUM
   (Theorem 2); the exported array forms in eft.c and the sequential loops in
   loops.c both use them. */
#define ORC_DEF_SUM_EFTS(T, SUF)                                              \
static inline void orc_fts_##SUF(T a, T b, T* x, T* y) {                      \
    const T xi = a + b;                  /* x  <- a (+) b  */                 \
    const T bv = xi - a;                 /* b' <- x (-) a  */                 \
    *x = xi;                                                                  \
    *y = b - bv;                         /* y  <- b (-) b' */                 \
}                                                                             \
static inline void orc_ts_##SUF(T a, T b, T* x, T* y) {                       \
    const T xi = a + b;                  /* 1. x  <- a (+) b   */             \
    const T bv = xi - a;                 /* 2. b' <- x (-) a   */             \
    const T av = xi - bv;                /* 3. a' <- x (-) b'  */             \
    const T bs = b - bv;                 /* 4. b# <- b (-) b'  */             \
    const T as = a - av;                 /* 5. a# <- a (-) a'  */             \
    *x = xi;                                                                  \
    *y = as + bs;                        /* 6. y  <- a# (+) b# */             \
}
ORC_DEF_SUM_EFTS(float, f32)
ORC_DEF_SUM_EFTS(double, f64)

#endif
