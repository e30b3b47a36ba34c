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

enum Variant : int { PLAIN = 0, FAST = 1, RIGOROUS = 2, WIDE = 3 };

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

// TwoProduct: p = RN(ab), e = RN(ab - p) by one fused multiply-add.
template <typename T>
__device__ __forceinline__ void two_product(T a, T b, T& p, T& e) {
    p = mul_rn(a, b);
    e = fma_rn(a, b, -p);
}

// ------------------------------------------------------ accumulation types
// Chains of the wide variant accumulate binary32 data in binary64; all other
// variants accumulate in the data type.  Cross-block merges of binary32 data
// run in binary64 except for the plain variant.
template <typename T, int VAR> struct Acc { using type = T; };
template <> struct Acc<float, WIDE> { using type = double; };
template <typename T, int VAR> struct GridAcc { using type = double; };
template <> struct GridAcc<float, PLAIN> { using type = float; };

template <int VAR> constexpr bool twofold_v = (VAR == FAST || VAR == RIGOROUS);

// One item into one chain (s, e).  Sums: y = x.  Dots: y = RN(x*y) and, for
// the twofold variants, ep = its TwoProduct error.
//   fast (Example 1):     t = s + y; c = (t - s) - y; e = e - c; s = t
//                         dot: e = e + (ep - c)
//   rigorous (Example 3): t = s + y; yt = t - s; dy = y - yt;
//                         ds = s - (t - yt); e = e + (ds + dy); s = t
//                         dot: e = e + ((ds + dy) + ep)
//   plain:                s = s + y
//   wide:                 S = S + y in binary64 (binary32 products are exact
//                         in binary64)
template <int VAR, bool DOT, typename T, typename A>
__device__ __forceinline__ void feed(A& s, A& e, T a, T b) {
    if constexpr (VAR == WIDE) {
        double p = DOT ? __dmul_rn((double)a, (double)b) : (double)a;
        s = __dadd_rn(s, p);
    } else if constexpr (VAR == PLAIN) {
        T p = DOT ? mul_rn(a, b) : a;
        s = add_rn(s, p);
    } else {
        T p, ep = T(0);
        if constexpr (DOT) two_product(a, b, p, ep); else p = a;
        if constexpr (VAR == FAST) {
            T t = add_rn(s, p);
            T c = sub_rn(sub_rn(t, s), p);
            if constexpr (DOT) e = add_rn(e, sub_rn(ep, c)); else e = sub_rn(e, c);
            s = t;
        } else {
            T t = add_rn(s, p);
            T yt = sub_rn(t, s);
            T dy = sub_rn(p, yt);
            T ds = sub_rn(s, sub_rn(t, yt));
            T q = add_rn(ds, dy);
            if constexpr (DOT) e = add_rn(e, add_rn(q, ep)); else e = add_rn(e, q);
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
        two_sum(v, v2, x, q);
        e = add_rn(add_rn(e, e2), q);
        v = x;
    }
}

// xor butterfly over the lanes of a warp for offsets o = W/2 ... 1; every
// lane holds lane (lane ^ o)'s previous pair as second operand.
template <bool TW, typename A>
__device__ __forceinline__ void warp_fold(A& v, A& e, int W = 32) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        if (o < W) {
            A v2 = __shfl_xor_sync(FULL, v, o);
            A e2 = __shfl_xor_sync(FULL, e, o);
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

// coherent 16-byte load of a pair written by another block (bypasses L1)
template <typename A>
__device__ __forceinline__ void ld_pair_cg(const A* p, A& v, A& e) {
    v = __ldcg(p);
    e = __ldcg(p + 1);
}

// ------------------------------------------------------------- workspace
// Workspace header; per-block / per-piece data start at byte 256.
struct WsHeader {
    unsigned int ticket;     // single vector: blocks done (reset by the last)
    int error;               // device error word, sticky until the host reads it
    int call_bad;            // batched: offsets of the current call are invalid
    unsigned int ticket2;    // batched: blocks done (reset by the last)
    double stage[2];         // host-buffer calls: the output pair
};
constexpr size_t kWsHeader = 256;

// Output of a pair (V, E) from the cross-block precision to the caller:
// binary64 data or TF_OUT_F64: (V, E); binary32 plain: (v, e) as is;
// binary32 twofold / wide: v = RN32(V), e = RN32((V - v) + E).
template <typename T, int VAR, typename G>
__device__ __forceinline__ void write_out(void* out, int64_t idx, G V, G E, bool out_f64) {
    if constexpr (sizeof(T) == 8) {
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
