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



#endif
