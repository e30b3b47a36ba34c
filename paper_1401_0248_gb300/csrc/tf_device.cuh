// tf_device.cuh -- device building blocks of the twofold kernels (sm_103a).
//
// Every floating-point operation below is an explicit round-to-nearest-even
// intrinsic (__fadd_rn, __dsub_rn, __fma_rn, ...), which the compiler never
// contracts or reassociates; the library is also built with --fmad=false and
// without fast-math or flush-to-zero.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tf {

// KAHAN is Example 2; FAST_LIT and RIG_LIT are the fast and rigorous dots with
// the paper's rounded product alone (no TwoProduct term).
enum Variant : int { PLAIN = 0, FAST = 1, RIGOROUS = 2, WIDE = 3, KAHAN = 4, FAST_LIT = 5,
                     RIG_LIT = 6 };

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------- rounding
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// ---------------------------------------------------- error-free transforms
// Theorem 1 (Dekker): x = a (+) b, y = b (-) (x (-) a); exact when |a| >= |b|.
template <typename T>
__device__ __forceinline__ void fast_two_sum(T a, T b, T& x, T& y) {
    x = add_rn(a, b);
    T bv = sub_rn(x, a);
    y = sub_rn(b, bv);
}

// Theorem 2 (Knuth): six operations, exact for any a, b without overflow.
template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T& x, T& y) {
    x = add_rn(a, b);
    T bv = sub_rn(x, a);
    T av = sub_rn(x, bv);
    T bs = sub_rn(b, bv);
    T as = sub_rn(a, av);
    y = add_rn(as, bs);
}

// Exact binary32 -> binary64 widening on the integer pipe (GB300's binary64
// conversion shares the slow binary64 rate): sign, exponent + 896, significand
// shifted by 29.  False for subnormal, infinite or NaN inputs (callers then
// convert with the hardware); same bits either way.
__device__ __forceinline__ bool widen_i(float a, double& r) {
    const unsigned int u = __float_as_uint(a);
    const unsigned int e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    if (e == 0u) {
        if (m != 0u) return false;
        r = __hiloint2double((int)(u & 0x80000000u), 0);
        return true;
    }
    if (e == 0xffu) return false;
    r = __hiloint2double((int)((u & 0x80000000u) | ((e + 896u) << 20) | (m >> 3)), (int)(m << 29));
    return true;
}

// The exact binary64 product of two binary32 numbers on the integer pipe: the
// 48-bit product of the significands (one wide multiply) normalised into a
// binary64 significand; the exponent stays in the normal binary64 range for
// normal inputs.  False for subnormal, infinite or NaN inputs.
__device__ __forceinline__ bool wide_product_i(float a, float b, double& r) {
    const unsigned int ua = __float_as_uint(a), ub = __float_as_uint(b);
    const unsigned int ea = (ua >> 23) & 0xffu, eb = (ub >> 23) & 0xffu;
    const unsigned int sg = (ua ^ ub) & 0x80000000u;
    if (((ua << 1) == 0u && eb != 0xffu) || ((ub << 1) == 0u && ea != 0xffu)) {
        r = __hiloint2double((int)sg, 0);          // a zero times a finite number
        return true;
    }
    if (ea == 0u || eb == 0u || ea == 0xffu || eb == 0xffu) return false;
    const unsigned long long P = (unsigned long long)((ua & 0x7fffffu) | 0x800000u) *
                                 (unsigned long long)((ub & 0x7fffffu) | 0x800000u);
    const unsigned int top = (unsigned int)(P >> 47);          // 1: P in [2^47, 2^48)
    const unsigned long long mant = (P << (5 + (top ^ 1u))) & 0x000fffffffffffffull;
    const unsigned int ex = ea + eb + 769u + top;             // biased binary64 exponent
    r = __longlong_as_double((long long)(((unsigned long long)(sg | (ex << 20)) << 32) | mant));
    return true;
}

// TwoProduct: p = RN(ab), e = RN(ab - p) by one fused multiply-add.
template <typename T>
__device__ __forceinline__ void two_product(T a, T b, T& p, T& e) {
    p = mul_rn(a, b);
    e = fma_rn(a, b, -p);
}

// ---- hybrid binary64 transforms: x from one binary64 add, the error on the
// integer pipe.  A TWO-SUM done wholly in integers (rounding included) is
// limited by GB300's integer ALU pipe; this split keeps both pipes busy.
//
// The error of x = RN(a + b) in units of 2^(emin - 1075), emin the smaller
// exponent field: r = ma*2^(ea-emin) +- mb*2^(eb-emin) -+ mx*2^(ex-emin).
// |a + b - x| <= min(|a|, |b|), so |r| < 2^53 and r is exact when the terms
// are added modulo 2^64 (a shift by 64 or more leaves 0 there, as the
// mathematical term does modulo 2^64).  If ex < emin the sum is exact.
__device__ __forceinline__ unsigned long long shl_sat(unsigned long long v, unsigned int s) {
    unsigned long long r;
    asm("shl.b64 %0, %1, %2;" : "=l"(r) : "l"(v), "r"(s));   // s >= 64 gives 0
    return r;
}

__device__ __forceinline__ double sum_error_h64(unsigned long long A, unsigned long long B,
                                                int ea, int eb, int emin, double x) {
    const unsigned long long M52 = 0x000fffffffffffffull, H = 1ull << 52;
    const unsigned long long X = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((X >> 52) & 0x7ff);
    if (ex < emin) return 0.0;
    unsigned long long ta = shl_sat((A & M52) | H, (unsigned)(ea - emin));
    unsigned long long tb = shl_sat((B & M52) | H, (unsigned)(eb - emin));
    const unsigned long long tx = shl_sat((X & M52) | H, (unsigned)(ex - emin));
    if ((A ^ X) >> 63) ta = 0ull - ta;          // terms signed relative to x
    if ((B ^ X) >> 63) tb = 0ull - tb;
    const unsigned long long r = ta + tb - tx;
    if (r == 0ull) return 0.0;
    const unsigned long long neg = r >> 63;
    const unsigned long long mag = neg ? (0ull - r) : r;
    const int pr = 63 - __clzll((long long)mag);               // <= 52
    const unsigned long long sy = (X >> 63) ^ neg;
    return __longlong_as_double((long long)((sy << 63) |
                                            ((unsigned long long)(emin + pr - 52) << 52) |
                                            ((mag << (52 - pr)) & M52)));
}

// A binary64 add issued as a fused multiply-add by `one` == 1.0: RN(a*1 + b)
// = RN(a + b) for every input, signed zeros included (-0*1 + +0 = +0,
// -0*1 + -0 = -0).  GB300 issues DFMA at 626 G/s against DADD's 528 G/s, so
// the per-item steps on binary64 add this way (the merges keep DADD); `one`
// must be a value the compiler cannot see (a load of g_one), since a known
// 1.0 is folded back into a DADD.
static __device__ double g_one = 1.0;   // never written: read once per kernel as `one`

template <bool FMA>
__device__ __forceinline__ double dadd(double a, double b, double one) {
    if constexpr (FMA) return __fma_rn(a, one, b);
    else return __dadd_rn(a, b);
}

// TWO-SUM(a, b): x = RN(a + b), y = a + b - x.  False (x, y untouched) unless
// both exponent fields lie in [54, 2044]; then the caller uses two_sum.
template <bool FMA = false>
__device__ __forceinline__ bool two_sum_h64(double a, double b, double& x, double& y,
                                            double one = 1.0) {
    const unsigned long long A = (unsigned long long)__double_as_longlong(a);
    const unsigned long long B = (unsigned long long)__double_as_longlong(b);
    const int ea = (int)((A >> 52) & 0x7ff), eb = (int)((B >> 52) & 0x7ff);
    const int emin = min(ea, eb);
    if (emin < 54 || max(ea, eb) > 2044) return false;
    x = dadd<FMA>(a, b, one);
    y = sum_error_h64(A, B, ea, eb, emin, x);
    return true;
}

// FAST-TWO-SUM(a, b) as written (x = a + b, y = b - (x - a)), for either order
// of magnitudes.  If ea >= eb (exponent fields) it is error-free (Dekker's
// condition) and y is the exact error.  Otherwise x - a = b - err exactly
// (err = a + b - x), so y = b - RN(b - err); as |err| <= ulp(b), RN(b - err)
// is b moved by 0 or one ulp(b) (0, 1 or 2 half-ulps below a power of two),
// chosen by comparing |err| with ulp/2 (ulp/4 and 3ulp/4 below a power of
// two), ties to even.
template <bool FMA = false>
__device__ __forceinline__ bool fast_two_sum_h64(double a, double b, double& x, double& y,
                                                 double one = 1.0) {
    const unsigned long long A = (unsigned long long)__double_as_longlong(a);
    const unsigned long long B = (unsigned long long)__double_as_longlong(b);
    const int ea = (int)((A >> 52) & 0x7ff), eb = (int)((B >> 52) & 0x7ff);
    const int emin = min(ea, eb);
    if (emin < 54 || max(ea, eb) > 2044) return false;
    x = dadd<FMA>(a, b, one);
    const double err = sum_error_h64(A, B, ea, eb, emin, x);
    if (ea >= eb) { y = err; return true; }
    const unsigned long long E = (unsigned long long)__double_as_longlong(err);
    const unsigned long long M52 = 0x000fffffffffffffull;
    const int Eu = eb - 52;                               // exponent field of ulp(b)
    const int eE = (int)((E >> 52) & 0x7ff);
    // |err| < ulp(b)/4 (err = 0 included: its field is 0 < Eu - 2): b - err
    // rounds back to b in every case below, so y = 0
    if (eE < Eu - 2) { y = 0.0; return true; }
    const unsigned long long mE = E & M52, mB = B & M52;
    const unsigned long long sb = B >> 63;
    const bool wpos = ((E >> 63) != sb);                 // b - err moves away from zero
    int ey;                                              // exponent field of |y| (0: y = 0)
    unsigned long long sy = sb;
    if (wpos || mB != 0ull) {                            // neighbours one ulp(b) apart
        const bool move = (eE > Eu - 1) || (eE == Eu - 1 && (mE != 0ull || (mB & 1ull)));
        ey = move ? Eu : 0;
        if (wpos) sy ^= 1ull;
    } else {                                             // b a power of two, moving down
        int j;
        if (eE < Eu - 2 || (eE == Eu - 2 && mE == 0ull)) j = 0;
        else if (eE == Eu - 2) j = 1;
        else if (eE == Eu - 1) j = mE < (1ull << 51) ? 1 : 2;
        else j = 2;
        ey = j == 0 ? 0 : (j == 1 ? Eu - 1 : Eu);
    }
    y = ey ? __longlong_as_double((long long)((sy << 63) | ((unsigned long long)ey << 52))) : 0.0;
    return true;
}

// Out-of-line binary64 forms for the excluded operand ranges, kept as real
// branches so that the common path never issues them.
static __device__ __noinline__ double widen_slow(float a) { return (double)a; }
static __device__ __noinline__ double wide_product_slow(float a, float b) {
    return __dmul_rn((double)a, (double)b);
}
static __device__ __noinline__ double2 two_sum_slow(double a, double b) {
    double x, y;
    two_sum(a, b, x, y);
    return make_double2(x, y);
}
static __device__ __noinline__ double2 fast_two_sum_slow(double a, double b) {
    double x, y;
    fast_two_sum(a, b, x, y);
    return make_double2(x, y);
}
static __device__ __noinline__ double2 two_product_slow(double a, double b) {
    double p, e;
    two_product(a, b, p, e);
    return make_double2(p, e);
}

// TwoProduct of two binary64 numbers on the integer pipe: the 106-bit
// product of the significands, rounded to 53 bits to nearest even, gives p;
// the signed remainder is e = ab - p, exact here (the cases where ab - p
// underflows are excluded).  Returns false, leaving p and e untouched, for
// zero, subnormal or non-finite operands and for exponent sums where p or e
// would leave the normal range; callers then use the FMA form.  Same bits.
// A product below 2^105 is doubled first (a multiply by 2, on the FMA pipe),
// so the rounding point is always bit 53 and every shift is a constant one.
__device__ __forceinline__ bool two_product_i64(double a, double b, double& p, double& e) {
    const unsigned long long A = (unsigned long long)__double_as_longlong(a);
    const unsigned long long B = (unsigned long long)__double_as_longlong(b);
    const unsigned long long M52 = 0x000fffffffffffffull;
    const int ea = (int)((A >> 52) & 0x7ff), eb = (int)((B >> 52) & 0x7ff);
    const int es = ea + eb;
    // ea, eb in [1, 2046] (normal, finite) and es in [1128, 3067]
    if ((unsigned)(ea - 1) >= 2046u || (unsigned)(eb - 1) >= 2046u || (unsigned)(es - 1128) > 1939u)
        return false;
    const unsigned long long ma = (A & M52) | (1ull << 52);
    const unsigned long long mb = (B & M52) | (1ull << 52);
    unsigned long long lo = ma * mb;
    unsigned long long hi = __umul64hi(ma, mb);          // product in [2^104, 2^106)
    const unsigned int top = (unsigned int)(hi >> 41) & 1u;   // product >= 2^105
    const unsigned int m = 2u - top;
    hi = hi * m + ((lo >> 63) & (unsigned long long)(1u - top));
    lo = lo * m;                                           // now in [2^105, 2^106)
    const unsigned long long q = (hi << 11) | (lo >> 53);     // [2^52, 2^53)
    const unsigned long long rem = lo & ((1ull << 53) - 1ull);
    // round to nearest even by a carry: q rounds up exactly when
    // rem + 2^52 - 1 + (q & 1) reaches 2^53; then ab - p = rem - 2^53
    const unsigned long long c = (rem + ((1ull << 52) - 1ull) + (q & 1ull)) >> 53;
    const unsigned long long sg = (A ^ B) >> 63;
    // exponent field es - 1023 + top; q + c = 2^53 carries into it
    p = __longlong_as_double((long long)((sg << 63) |
                                         (((unsigned long long)(es - 1024 + (int)top) << 52) + q + c)));
    const unsigned long long rmag = c ? ((1ull << 53) - rem) : rem;
    if (rmag == 0ull) {
        e = 0.0;
    } else {
        // rmag counts units of 2^(es - 2151 + top)
        const int pr = 63 - __clzll((long long)rmag);          // <= 52
        const unsigned long long se = sg ^ c;
        e = __longlong_as_double((long long)((se << 63) |
                                             ((unsigned long long)(es + pr - 1128 + (int)top) << 52) |
                                             ((rmag << (52 - pr)) & M52)));
    }
    return true;
}

// ---------------------------------------------------------------- binary128
// IEEE binary128 in integer arithmetic: the wide ('d') accumulator for
// binary64 data, the paper's __float128 comparison.  Bits as IEEE stores
// them: hi = sign | 15-bit exponent (bias 16383) | top 48 fraction bits.
// Sums of binary64 numbers and products of two never reach the binary128
// subnormal or overflow ranges, so only zeros, normals, infinities and NaN
// occur.
struct q128 {
    unsigned long long lo, hi;
    __device__ __forceinline__ q128() : lo(0ull), hi(0ull) {}
    __device__ __forceinline__ q128(unsigned long long l, unsigned long long h) : lo(l), hi(h) {}
    __device__ __forceinline__ explicit q128(int) : lo(0ull), hi(0ull) {}   // +0
    __device__ explicit q128(double x);                                       // exact widening
};
typedef unsigned __int128 u128;
constexpr unsigned long long kQFrac = 0x0000ffffffffffffull;

__device__ __forceinline__ q128 q_pack(unsigned long long sign, int be, u128 m) {
    // m holds the implicit bit at 112 for normals
    return q128((unsigned long long)m,
                (sign << 63) | ((unsigned long long)be << 48) | ((unsigned long long)(m >> 64) & kQFrac));
}

__device__ __forceinline__ q128::q128(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned long long sign = u >> 63;
    const int e = (int)((u >> 52) & 0x7ff);
    unsigned long long f = u & 0x000fffffffffffffull;
    if (e == 0x7ff) {                                   // Inf / NaN (keep a quiet NaN)
        hi = (sign << 63) | (0x7fffull << 48) | (f ? (1ull << 47) : 0ull);
        lo = 0ull;
    } else if (e == 0) {
        if (f == 0ull) { hi = sign << 63; lo = 0ull; return; }
        const int lz = __clzll((long long)f) - 11;        // subnormal binary64: normalise
        f <<= lz;                                         // leading one at bit 52
        const q128 r = q_pack(sign, 15361 - lz, (u128)f << 60);      // 2^(-1022 - lz)
        lo = r.lo; hi = r.hi;
    } else {
        const q128 r = q_pack(sign, e + 15360, (u128)(f | (1ull << 52)) << 60);
        lo = r.lo; hi = r.hi;
    }
}

// the exact binary128 product of two binary64 numbers (106-bit significand)
__device__ __forceinline__ q128 q_mul_exact(double a, double b) {
    const unsigned long long A = (unsigned long long)__double_as_longlong(a);
    const unsigned long long B = (unsigned long long)__double_as_longlong(b);
    const int ea = (int)((A >> 52) & 0x7ff), eb = (int)((B >> 52) & 0x7ff);
    const unsigned long long sign = (A ^ B) >> 63;
    if (ea == 0x7ff || eb == 0x7ff || ea == 0 || eb == 0) {
        // specials, zeros and subnormals: widen both exactly and multiply the
        // normalised significands the same way below
        const q128 qa(a), qb(b);
        const int xa = (int)((qa.hi >> 48) & 0x7fff), xb = (int)((qb.hi >> 48) & 0x7fff);
        if (xa == 0x7fff || xb == 0x7fff) {
            const bool nan = (xa == 0x7fff && ((qa.hi & kQFrac) | qa.lo)) ||
                             (xb == 0x7fff && ((qb.hi & kQFrac) | qb.lo)) ||
                             (xa == 0 && xb == 0x7fff) || (xb == 0 && xa == 0x7fff);
            return nan ? q128(0ull, (0x7fffull << 48) | (1ull << 47))
                       : q128(0ull, (sign << 63) | (0x7fffull << 48));
        }
        if (xa == 0 || xb == 0) return q128(0ull, sign << 63);
        const u128 ma = ((u128)(qa.hi & kQFrac) << 64 | qa.lo) | ((u128)1 << 112);
        const u128 mb = ((u128)(qb.hi & kQFrac) << 64 | qb.lo) | ((u128)1 << 112);
        // both significands are 53-bit values shifted left by 60
        const u128 P = (ma >> 60) * (mb >> 60);                  // in [2^104, 2^106)
        const int top = (int)(P >> 105);                         // 1 if bit 105 set
        return q_pack(sign, xa + xb - 16383 + top, P << (8 - top));
    }
    const u128 P = (u128)((A & 0x000fffffffffffffull) | (1ull << 52)) *
                   (u128)((B & 0x000fffffffffffffull) | (1ull << 52));
    const int top = (int)(P >> 105);
    return q_pack(sign, ea + eb - 2046 + 16383 + top, P << (8 - top));
}

__device__ __forceinline__ int q_clz(u128 m) {
    const unsigned long long h = (unsigned long long)(m >> 64);
    return h ? __clzll((long long)h) : 64 + __clzll((long long)(unsigned long long)m);
}

// a + b rounded to nearest even (three guard bits, sticky folded into the last)
__device__ __forceinline__ q128 q_add(q128 a, q128 b) {
    int ea = (int)((a.hi >> 48) & 0x7fff), eb = (int)((b.hi >> 48) & 0x7fff);
    unsigned long long sa = a.hi >> 63, sb = b.hi >> 63;
    if (ea == 0x7fff || eb == 0x7fff) {
        const bool na = ea == 0x7fff && ((a.hi & kQFrac) | a.lo);
        const bool nb = eb == 0x7fff && ((b.hi & kQFrac) | b.lo);
        const q128 qnan(0ull, (0x7fffull << 48) | (1ull << 47));
        if (na || nb) return qnan;
        if (ea == 0x7fff && eb == 0x7fff) return sa == sb ? a : qnan;
        return ea == 0x7fff ? a : b;
    }
    if (ea == 0) {                                       // a = +-0 (no subnormals occur)
        if (eb == 0) return q128(0ull, (sa & sb) << 63);  // -0 only for -0 + -0
        return b;
    }
    if (eb == 0) return a;
    u128 ma = ((u128)(a.hi & kQFrac) << 64 | a.lo) | ((u128)1 << 112);
    u128 mb = ((u128)(b.hi & kQFrac) << 64 | b.lo) | ((u128)1 << 112);
    if (ea < eb || (ea == eb && ma < mb)) {             // |a| >= |b|
        u128 tm = ma; ma = mb; mb = tm;
        int te = ea; ea = eb; eb = te;
        unsigned long long ts = sa; sa = sb; sb = ts;
    }
    const int d = ea - eb;
    ma <<= 3;
    mb <<= 3;
    if (d > 0) {
        if (d >= 120) {
            mb = 1;                                      // sticky only
        } else {
            const u128 lost = mb & (((u128)1 << d) - 1);
            mb = (mb >> d) | (lost ? (u128)1 : (u128)0);
        }
    }
    int e = ea;
    u128 m;
    if (sa == sb) {
        m = ma + mb;
        if (m >> 116) { m = (m >> 1) | (m & 1); e += 1; }
    } else {
        m = ma - mb;
        if (m == 0) return q128(0ull, 0ull);             // exact cancellation: +0
        const int lz = q_clz(m) - 12;                    // leading one back to bit 115
        m <<= lz;
        e -= lz;
    }
    const unsigned int g = (unsigned int)m & 7u;
    m >>= 3;
    if (g > 4u || (g == 4u && (m & 1))) {
        m += 1;
        if (m >> 113) { m >>= 1; e += 1; }
    }
    return q_pack(sa, e, m);
}

// RN64 of a binary128 value, with gradual underflow and overflow to Inf
__device__ __forceinline__ double q_to_double(q128 a) {
    const int e = (int)((a.hi >> 48) & 0x7fff);
    const unsigned long long sign = a.hi >> 63;
    if (e == 0x7fff) {
        const bool nan = (a.hi & kQFrac) | a.lo;
        return __longlong_as_double((long long)((sign << 63) | (0x7ffull << 52) | (nan ? (1ull << 51) : 0ull)));
    }
    if (e == 0) return __longlong_as_double((long long)(sign << 63));
    const u128 m = ((u128)(a.hi & kQFrac) << 64 | a.lo) | ((u128)1 << 112);
    const int E = e - 16383;                              // unbiased exponent
    int sh = 60 + (E < -1022 ? (-1022 - E) : 0);
    if (sh > 126) return __longlong_as_double((long long)(sign << 63));
    unsigned long long q = (unsigned long long)(m >> sh);
    const u128 rem = m & (((u128)1 << sh) - 1);
    const u128 half = (u128)1 << (sh - 1);
    if (rem > half || (rem == half && (q & 1ull))) q += 1;
    unsigned long long bits;
    if (E < -1022) bits = q;                              // subnormal (2^52 is the least normal)
    else if (E > 1023) bits = 0x7ffull << 52;             // overflow
    else bits = ((unsigned long long)(E + 1022) << 52) + q;   // carries into the exponent
    if (bits >= (0x7ffull << 52)) bits = 0x7ffull << 52;
    return __longlong_as_double((long long)((sign << 63) | bits));
}

__device__ __forceinline__ q128 q_neg(q128 a) { return q128(a.lo, a.hi ^ (1ull << 63)); }

// ------------------------------------------------------ accumulation types
// Chains of the wide variant accumulate binary32 data in binary64; all other
// variants accumulate in the data type.  Cross-block merges of binary32 data
// run in binary64 except for the plain variant.
template <typename T, int VAR> struct Acc { using type = T; };
template <> struct Acc<float, WIDE> { using type = double; };
template <> struct Acc<double, WIDE> { using type = q128; };
template <typename T, int VAR> struct GridAcc { using type = double; };
template <> struct GridAcc<float, PLAIN> { using type = float; };
template <> struct GridAcc<double, WIDE> { using type = q128; };

__device__ __forceinline__ q128 add_rn(q128 a, q128 b) { return q_add(a, b); }

// Shared-memory storage of a value type: the type itself, or for q128 (whose
// constructor a __shared__ variable may not run) a plain struct of its layout.
template <typename A> struct SmemOf { using type = A; };
struct q128_raw { unsigned long long lo, hi; };
template <> struct SmemOf<q128> { using type = q128_raw; };

template <int VAR> constexpr bool twofold_v = (VAR != PLAIN && VAR != WIDE);
// the per-item step after the product: literal dots step like the sums
template <int VAR> constexpr int step_v = VAR == FAST_LIT ? FAST : (VAR == RIG_LIT ? RIGOROUS : VAR);

// One item into one chain (s, e).  Sums: the item is x.  Dots: the item is
// RN(x*y) and, for the twofold variants, ep is its TwoProduct error.
//   fast (Example 1):     the chain value and the item go through FAST-TWO-SUM
//                         (Theorem 1); the sum becomes the chain value and the
//                         transform's error is added to e (dots: the error and
//                         ep are added together first, then to e)
//   rigorous (Example 3): the same with TWO-SUM (Theorem 2)
//   plain:                the item is added to the chain value
//   wide:                 the item is added to a binary64 accumulator
//                         (binary32 products are exact in binary64)
// `one` is a runtime 1.0 (see dadd): the binary64 sums and twofold dots and
// the binary64 accumulator of binary32 data ('wide') issue their adds as DFMA
// (the plain binary64 dot rounds its product first, by a multiply).
template <int VAR, bool DOT, typename T, typename A>
__device__ __forceinline__ void feed(A& s, A& e, T a, T b, double one = 1.0) {
    constexpr int STEP = step_v<VAR>;
    constexpr bool TPROD = DOT && (VAR == FAST || VAR == RIGOROUS);   // TwoProduct error kept
    constexpr bool FMA = sizeof(T) == 8 && (!DOT || VAR != PLAIN);
    if constexpr (VAR == WIDE && sizeof(T) == 8) {
        // binary64 data: binary128 accumulator, products exact in binary128
        s = q_add(s, DOT ? q_mul_exact(a, b) : q128(a));
    } else if constexpr (VAR == WIDE) {
        double p;
        if constexpr (DOT) {
            if (!wide_product_i(a, b, p)) p = wide_product_slow(a, b);
        } else {
            if (!widen_i(a, p)) p = widen_slow(a);
        }
        s = dadd<true>(s, p, one);      // the widened item (or exact product) by DFMA
    } else if constexpr (VAR == PLAIN) {
        if constexpr (FMA) {
            s = dadd<true>(s, a, one);
        } else {
            T p = DOT ? mul_rn(a, b) : a;
            s = add_rn(s, p);
        }
    } else if constexpr (sizeof(T) == 8) {
        // binary64: the error-free transforms take one binary64 add (or none
        // for the product) plus integer work; the bits are those of the
        // binary64 operation sequences of Examples 1-3.  The fast step is
        // FAST-TWO-SUM of the chain value and the item, its error added to e
        // (Example 1's compensation term is that error negated); Kahan's step
        // is FAST-TWO-SUM of the chain value and the item plus e, whose error
        // becomes the new e.
        double p, ep = 0.0;
        if constexpr (TPROD) {
            if (!two_product_i64(a, b, p, ep)) { const double2 r = two_product_slow(a, b); p = r.x; ep = r.y; }
        } else if constexpr (DOT) {
            double unused;
            if (!two_product_i64(a, b, p, unused)) p = two_product_slow(a, b).x;
        } else {
            p = a;
        }
        double t, y;
        if constexpr (STEP == KAHAN) {
            const double yk = dadd<FMA>(p, e, one);
            if (!fast_two_sum_h64<FMA>(s, yk, t, y, one)) { const double2 r = fast_two_sum_slow(s, yk); t = r.x; y = r.y; }
            e = y;
        } else {
            if constexpr (STEP == FAST) {
                if (!fast_two_sum_h64<FMA>(s, p, t, y, one)) { const double2 r = fast_two_sum_slow(s, p); t = r.x; y = r.y; }
            } else {
                if (!two_sum_h64<FMA>(s, p, t, y, one)) { const double2 r = two_sum_slow(s, p); t = r.x; y = r.y; }
            }
            if constexpr (TPROD) e = dadd<FMA>(e, dadd<FMA>(y, ep, one), one); else e = dadd<FMA>(e, y, one);
        }
        s = t;
    } else {
        T p, ep = T(0);
        if constexpr (TPROD) two_product(a, b, p, ep); else p = DOT ? mul_rn(a, b) : a;
        if constexpr (STEP == KAHAN) {
            // Example 2 with e holding the negated compensation term: the item
            // plus e joins the chain value, and the new e is what that sum lost
            const T yk = add_rn(p, e);
            const T t = add_rn(s, yk);
            e = sub_rn(yk, sub_rn(t, s));
            s = t;
        } else if constexpr (STEP == FAST) {
            T t = add_rn(s, p);
            T c = sub_rn(sub_rn(t, s), p);
            if constexpr (TPROD) e = add_rn(e, sub_rn(ep, c)); else e = sub_rn(e, c);
            s = t;
        } else {
            // Example 3: TWO-SUM (Theorem 2) of s and the item, its error to e
            T t, q;
            two_sum(s, p, t, q);
            if constexpr (TPROD) e = add_rn(e, add_rn(q, ep)); else e = add_rn(e, q);
            s = t;
        }
    }
}

// Merge (v2, e2) into (v, e): (v, q) = TWO-SUM(v, v2); e = (e + e2) + q.
// Plain and wide merge by one addition.
template <bool TW, typename A>
__device__ __forceinline__ void merge(A& v, A& e, A v2, A e2) {
    if constexpr (!TW) {
        v = add_rn(v, v2);
    } else {
        A x, q;
        if constexpr (sizeof(A) == 8) {
            if (!two_sum_h64(v, v2, x, q)) { const double2 r = two_sum_slow(v, v2); x = r.x; q = r.y; }
        } else {
            two_sum(v, v2, x, q);
        }
        e = add_rn(add_rn(e, e2), q);
        v = x;
    }
}

template <typename A>
__device__ __forceinline__ A shfl_xor(A v, int o) { return __shfl_xor_sync(FULL, v, o); }
__device__ __forceinline__ q128 shfl_xor(q128 v, int o) {
    return q128(__shfl_xor_sync(FULL, v.lo, o), __shfl_xor_sync(FULL, v.hi, o));
}

template <typename A>
__device__ __forceinline__ A shfl_down(A v, int o) { return __shfl_down_sync(FULL, v, o); }
__device__ __forceinline__ q128 shfl_down(q128 v, int o) {
    return q128(__shfl_down_sync(FULL, v.lo, o), __shfl_down_sync(FULL, v.hi, o));
}

// xor butterfly over the lanes of a warp for offsets o = W/2 ... 1; every
// lane holds lane (lane ^ o)'s previous pair as second operand.
template <bool TW, typename A>
__device__ __forceinline__ void warp_fold(A& v, A& e, int W = 32) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        if (o < W) {
            A v2 = shfl_xor(v, o);
            A e2 = shfl_xor(e, o);
            merge<TW>(v, e, v2, e2);
        }
    }
}

// Block fold: warp butterflies, then warp 0 folds the W = blockDim/32 warp
// pairs by the butterfly over W lanes.  Thread 0 returns the block pair.
// smem must hold 2 * 32 values of A.  Ends with the block synchronized.
template <bool TW, typename A>
__device__ __forceinline__ void block_fold(A& v, A& e, A* smem) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    warp_fold<TW>(v, e);
    if (lane == 0) { smem[warp] = v; smem[32 + warp] = e; }
    __syncthreads();
    if (warp == 0) {
        v = lane < W ? smem[lane] : A(0);
        e = lane < W ? smem[32 + lane] : A(0);
        warp_fold<TW>(v, e, W);
    }
    __syncthreads();
}

// Block fold as a tree over the block's threads: pair t <- merge(pair t,
// pair t + w) for w = B/2, B/4, ..., 1 and threads t < w (the order of the
// per-thread chain tree), through shared memory while w >= 32 and by
// shuffles inside warp 0 below; each merge runs once, in one lane, so a fold
// issues about a fifth of the binary64 instructions of a butterfly in which
// every lane runs every merge.  Thread 0 returns the block pair; sv, se hold
// blockDim.x values of A.  Ends with the block synchronized.
template <bool TW, typename A>
__device__ __forceinline__ void block_tree(A& v, A& e, A* sv, A* se) {
    const int t = threadIdx.x, B = blockDim.x;
    if (B > 32) {
        sv[t] = v;
        se[t] = e;
        __syncthreads();
        for (int w = B / 2; w >= 32; w >>= 1) {
            if (t < w) {
                A a = sv[t], ae = se[t];
                merge<TW>(a, ae, sv[t + w], se[t + w]);
                sv[t] = a;
                se[t] = ae;
            }
            __syncthreads();
        }
        if (t < 32) { v = sv[t]; e = se[t]; }
    }
    if (t < 32) {
#pragma unroll
        for (int w = 16; w >= 1; w >>= 1) {
            const A v2 = shfl_down(v, w), e2 = shfl_down(e, w);
            if (t < w) merge<TW>(v, e, v2, e2);
        }
    }
    __syncthreads();
}

// ------------------------------------------------------------------ loads
// 128-bit streaming loads: read-only path, no L1 allocation (the data is read
// once), 256-byte L2 prefetch granule.
__device__ __forceinline__ void ld_stream(const float* p, float (&r)[4]) {
    asm("ld.global.nc.L1::no_allocate.L2::256B.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]) : "l"(p));
}
__device__ __forceinline__ void ld_stream(const double* p, double (&r)[2]) {
    asm("ld.global.nc.L1::no_allocate.L2::256B.v2.f64 {%0,%1}, [%2];"
                 : "=d"(r[0]), "=d"(r[1]) : "l"(p));
}
template <typename T, int V>
__device__ __forceinline__ void ld_vec(const T* p, bool aligned, T (&r)[V]) {
    if (aligned) {
        ld_stream(p, r);
    } else {
#pragma unroll
        for (int l = 0; l < V; ++l) r[l] = __ldg(p + l);
    }
}

// coherent load of a pair written by another block (bypasses L1)
template <typename A>
__device__ __forceinline__ void ld_pair_cg(const A* p, A& v, A& e) {
    v = __ldcg(p);
    e = __ldcg(p + 1);
}
__device__ __forceinline__ void ld_pair_cg(const q128* p, q128& v, q128& e) {
    const unsigned long long* u = reinterpret_cast<const unsigned long long*>(p);
    v = q128(__ldcg(u), __ldcg(u + 1));
    e = q128(__ldcg(u + 2), __ldcg(u + 3));
}

// ------------------------------------------------------------- workspace
// Workspace header; per-block / per-piece data start at byte 256.
struct WsHeader {
    unsigned int ticket;     // single vector: blocks done (reset by the last)
    int error;               // device error word, sticky until the host reads it
    int call_bad;            // batched: offsets of the current call are invalid (cleared by csr_merge)
    unsigned int reserved;
    double stage[2];         // host-buffer calls: the output pair
    unsigned long long tile_next;   // batched: next tile to claim (cleared by csr_merge)
};
constexpr size_t kWsHeader = 256;

// Output of a pair (V, E) from the cross-block precision to the caller:
// binary64 data or TF_OUT_F64: (V, E); binary32 plain: (v, e) as is;
// binary32 twofold / wide: v = RN32(V), e = RN32((V - v) + E).
template <typename T, int VAR, typename G>
__device__ __forceinline__ void write_out(void* out, int64_t idx, G V, G E, bool out_f64) {
    if constexpr (sizeof(G) == 16) {
        // binary128 accumulator: (RN64(S), RN64(S - RN64(S)))
        double* o = (double*)out;
        const double hi = q_to_double(V);
        o[2 * idx] = hi;
        o[2 * idx + 1] = q_to_double(q_add(V, q_neg(q128(hi))));
    } else if constexpr (sizeof(T) == 8) {
        double* o = (double*)out;
        o[2 * idx] = V; o[2 * idx + 1] = E;
    } else {
        if (out_f64) {
            double* o = (double*)out;
            o[2 * idx] = (double)V; o[2 * idx + 1] = (double)E;
        } else if constexpr (VAR == PLAIN) {
            float* o = (float*)out;
            o[2 * idx] = (float)V; o[2 * idx + 1] = (float)E;
        } else {
            float* o = (float*)out;
            float v = __double2float_rn((double)V);
            double d = __dadd_rn(__dsub_rn((double)V, (double)v), (double)E);
            o[2 * idx] = v; o[2 * idx + 1] = __double2float_rn(d);
        }
    }
}

}  // namespace tf
