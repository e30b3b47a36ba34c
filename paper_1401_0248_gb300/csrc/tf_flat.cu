// tf_flat.cu -- twofold sum / dot of one vector in one launch (sm_103a).
//
// Grid-stride streaming with 128-bit loads: thread g of P threads takes the
// 16-byte vectors j = g + P*m and feeds element l of vector j to its chain
// (m mod U)*V + l, U vectors in flight per step.  The U*V chains hide the
// dependency of each chain's additions (the latency chain the paper breaks
// with independent accumulators in its h-functions).  A thread's chains fold
// by a tree; the block's threads by the same tree (binary64 twofold kernels)
// or by warp butterflies and a butterfly over the warp pairs (the others);
// the last block to finish (a ticket in the workspace, no waiting) folds the
// block pairs the same way and writes the result.
#include "tf_device.cuh"
#include "tf_internal.h"

namespace tf {

template <typename T, int VAR, bool DOT, int U>
__global__ void __launch_bounds__(512)
flat_kernel(const T* __restrict__ x, const T* __restrict__ y, int64_t n,
            void* __restrict__ out, unsigned char* __restrict__ ws, int aligned, int out_f64) {
    using A = typename Acc<T, VAR>::type;
    using G = typename GridAcc<T, VAR>::type;
    constexpr bool TW = twofold_v<VAR>;
    constexpr int V = 16 / sizeof(T);
    constexpr int C = U * V;

    A s[C], e[C];
#pragma unroll
    for (int c = 0; c < C; ++c) { s[c] = A(0); e[c] = A(0); }
    double one = 1.0;                 // binary64 data, wide: a 1.0 the compiler cannot see
    if constexpr (sizeof(T) == 8 || VAR == WIDE) one = *reinterpret_cast<volatile double*>(&g_one);

    const int64_t nv = n / V;
    const int tail = (int)(n - nv * V);
    const int64_t P = (int64_t)gridDim.x * blockDim.x;
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;

    // steps of U full vectors: vector j + u*P is step m = kU + u, chain u*V + l
    auto load = [&](int64_t jj, T (&xv)[U][V], T (&yv)[U][V]) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            ld_vec<T, V>(x + (jj + u * P) * V, aligned, xv[u]);
            if constexpr (DOT) ld_vec<T, V>(y + (jj + u * P) * V, aligned, yv[u]);
        }
    };
    auto feed_all = [&](const T (&xv)[U][V], const T (&yv)[U][V]) {
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int l = 0; l < V; ++l)
                feed<VAR, DOT>(s[u * V + l], e[u * V + l], xv[u][l], DOT ? yv[u][l] : T(0), one);
    };
    // binary32 twofold dots and binary64 twofold sums and dots: the next
    // step's loads go out before this step's arithmetic (two steps of loads
    // in flight per thread; the binary64 plans keep one 16-byte load per
    // array per step, U = 1, so the extra registers leave occupancy intact)
    constexpr bool PREFETCH = (sizeof(T) == 4 && DOT && VAR != WIDE) ||
                              (sizeof(T) == 8 && (VAR == FAST || VAR == RIGOROUS));
    if constexpr (PREFETCH) {
        if (j + (U - 1) * P < nv) {
            T xv[U][V], yv[U][V];
            load(j, xv, yv);
            for (;;) {
                const int64_t jn = j + U * P;
                const bool more = jn + (U - 1) * P < nv;
                T xn[U][V], yn[U][V];
                if (more) load(jn, xn, yn);
                feed_all(xv, yv);
                j = jn;
                if (!more) break;
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int l = 0; l < V; ++l) {
                        xv[u][l] = xn[u][l];
                        yv[u][l] = yn[u][l];
                    }
            }
        }
    } else {
        for (; j + (U - 1) * P < nv; j += U * P) {
            T xv[U][V], yv[U][V];
            load(j, xv, yv);
            feed_all(xv, yv);
        }
    }
    // fewer than U full vectors left for this thread, and maybe the partial
    // vector n/V (owned by the thread with g = (n/V) mod P)
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t jj = j + u * P;
        if (jj < nv) {
            T xv[V], yv[V];
            ld_vec<T, V>(x + jj * V, aligned, xv);
            if constexpr (DOT) ld_vec<T, V>(y + jj * V, aligned, yv);
#pragma unroll
            for (int l = 0; l < V; ++l)
                feed<VAR, DOT>(s[u * V + l], e[u * V + l], xv[l], DOT ? yv[l] : T(0), one);
        } else if (jj == nv && tail > 0) {
#pragma unroll
            for (int l = 0; l < V; ++l)
                if (l < tail) {
                    T a = x[jj * V + l];
                    T b = DOT ? y[jj * V + l] : T(0);
                    feed<VAR, DOT>(s[u * V + l], e[u * V + l], a, b, one);
                }
        }
    }

    // thread fold: tree over the chains
#pragma unroll
    for (int w = C / 2; w >= 1; w >>= 1)
#pragma unroll
        for (int c = 0; c < w; ++c) merge<TW>(s[c], e[c], s[c + w], e[c + w]);
    A v = s[0], ev = e[0];

    // Binary64 twofold kernels fold blocks (and the grid) by the tree over the
    // block's threads, where each merge's three binary64 adds run in one lane;
    // the others keep the warp butterflies, whose merges are cheap there.
    constexpr bool TREE = sizeof(T) == 8 && TW;
    __shared__ __align__(16) double tree_buf[TREE ? 2 * 512 : 2];
    __shared__ typename SmemOf<A>::type smA[64];
    if constexpr (TREE) block_tree<TW>(v, ev, tree_buf, tree_buf + 512);
    else block_fold<TW>(v, ev, reinterpret_cast<A*>(smA));

    WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
    G* slots = reinterpret_cast<G*>(ws + kWsHeader);
    __shared__ int am_last;
    if (threadIdx.x == 0) {
        slots[2 * blockIdx.x] = (G)v;
        slots[2 * blockIdx.x + 1] = (G)ev;
        __threadfence();
        unsigned int t = atomicAdd(&hdr->ticket, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();

    // grid fold: thread t takes block pairs t, t + B, t + 2B, ... in turn
    G gv = G(0), ge = G(0);
    if (threadIdx.x < gridDim.x) {
        ld_pair_cg(slots + 2 * threadIdx.x, gv, ge);
        for (int64_t i = threadIdx.x + blockDim.x; i < gridDim.x; i += blockDim.x) {
            G v2, e2;
            ld_pair_cg(slots + 2 * i, v2, e2);
            merge<TW>(gv, ge, v2, e2);
        }
    }
    __shared__ typename SmemOf<G>::type smG[64];
    if constexpr (TREE) block_tree<TW>(gv, ge, tree_buf, tree_buf + 512);
    else block_fold<TW>(gv, ge, reinterpret_cast<G*>(smG));
    if (threadIdx.x == 0) {
        write_out<T, VAR, G>(out, 0, gv, ge, out_f64 != 0);
        hdr->ticket = 0u;           // ready for the next call / graph replay
    }
}

template <typename T, int VAR, bool DOT>
static cudaError_t launch_u(int unroll, const void* x, const void* y, int64_t n, void* out,
                            void* ws, int block, int64_t grid, int aligned, int out_f64,
                            cudaStream_t st) {
    const T* xp = static_cast<const T*>(x);
    const T* yp = static_cast<const T*>(y);
    unsigned char* w = static_cast<unsigned char*>(ws);
    switch (unroll) {
    case 1: flat_kernel<T, VAR, DOT, 1><<<(unsigned)grid, block, 0, st>>>(xp, yp, n, out, w, aligned, out_f64); break;
    case 2: flat_kernel<T, VAR, DOT, 2><<<(unsigned)grid, block, 0, st>>>(xp, yp, n, out, w, aligned, out_f64); break;
    case 4: flat_kernel<T, VAR, DOT, 4><<<(unsigned)grid, block, 0, st>>>(xp, yp, n, out, w, aligned, out_f64); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T, int VAR>
static cudaError_t launch_d(int dot, int unroll, const void* x, const void* y, int64_t n,
                            void* out, void* ws, int block, int64_t grid, int aligned,
                            int out_f64, cudaStream_t st) {
    return dot ? launch_u<T, VAR, true>(unroll, x, y, n, out, ws, block, grid, aligned, out_f64, st)
               : launch_u<T, VAR, false>(unroll, x, y, n, out, ws, block, grid, aligned, out_f64, st);
}

cudaError_t launch_flat(int dtype, int variant, int dot, int unroll, const void* x,
                        const void* y, int64_t n, void* out, void* ws, int block,
                        int64_t grid, int aligned, int out_f64, cudaStream_t st) {
    if (dtype == 0) {
        switch (variant) {
        case PLAIN: return launch_d<float, PLAIN>(dot, unroll, x, y, n, out, ws, block, grid, aligned, out_f64, st);
        case FAST: return launch_d<float, FAST>(dot, unroll, x, y, n, out, ws, block, grid, aligned, out_f64, st);
        case RIGOROUS: return launch_d<float, RIGOROUS>(dot, unroll, x, y, n, out, ws, block, grid, aligned, out_f64, st);
        case WIDE: return launch_d<float, WIDE>(dot, unroll, x, y, n, out, ws, block, grid, aligned, out_f64, st);
        case KAHAN: return launch_d<float, KAHAN>(dot, unroll, x, y, n, out, ws, block, grid, aligned, out_f64, st);
        case FAST_LIT: return dot ? launch_u<float, FAST_LIT, true>(unroll, x, y, n, out, ws, block, grid, aligned, out_f64, st) : cudaErrorInvalidValue;
        case RIG_LIT: return dot ? launch_u<float, RIG_LIT, true>(unroll, x, y, n, out, ws, block, grid, aligned, out_f64, st) : cudaErrorInvalidValue;
        }
    } else {
        switch (variant) {
        case PLAIN: return launch_d<double, PLAIN>(dot, unroll, x, y, n, out, ws, block, grid, aligned, out_f64, st);
        case FAST: return launch_d<double, FAST>(dot, unroll, x, y, n, out, ws, block, grid, aligned, out_f64, st);
        case RIGOROUS: return launch_d<double, RIGOROUS>(dot, unroll, x, y, n, out, ws, block, grid, aligned, out_f64, st);
        case WIDE: return launch_d<double, WIDE>(dot, unroll, x, y, n, out, ws, block, grid, aligned, out_f64, st);
        case KAHAN: return launch_d<double, KAHAN>(dot, unroll, x, y, n, out, ws, block, grid, aligned, out_f64, st);
        case FAST_LIT: return dot ? launch_u<double, FAST_LIT, true>(unroll, x, y, n, out, ws, block, grid, aligned, out_f64, st) : cudaErrorInvalidValue;
        case RIG_LIT: return dot ? launch_u<double, RIG_LIT, true>(unroll, x, y, n, out, ws, block, grid, aligned, out_f64, st) : cudaErrorInvalidValue;
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace tf
