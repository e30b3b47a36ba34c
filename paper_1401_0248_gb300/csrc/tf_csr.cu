// tf_csr.cu -- twofold sums / dots of many ragged CSR segments in one
// persistent launch (sm_103a).
//
// Load balance does not depend on the length mix: the concatenated vector is
// cut into equal tiles of `tile` elements, and each warp of the persistent
// grid takes a contiguous run of tiles.  Inside a tile the warp reduces each
// segment's piece: lane l takes the 16-byte vector slots l, l+32, ... of the
// tile, slot m-th for the lane feeding chains (m mod U)*V + (element mod V).
// Elements outside the piece are fed as +0, which leaves a twofold, plain or
// wide chain's bits unchanged (Kahan chains skip them), so the chain
// assignment is the documented one with no branches in the streaming loop.  A segment inside one tile is written directly; a
// segment over k tiles leaves k piece pairs in the workspace and the warp that
// completes the k-th piece (a per-segment ticket, no waiting) merges them in
// tile order.  A first small kernel checks the offsets, clears the tickets
// and writes the empty segments.
#include "tf_device.cuh"
#include "tf_internal.h"

namespace tf {

constexpr int kTfErrOffsets = 6;       // TF_ERR_OFFSETS

size_t csr_ws_bytes(int64_t n, int64_t nseg) {
    size_t cnt = ((size_t)(nseg > 0 ? nseg : 1) * 4 + 255) / 256 * 256;
    size_t ntiles = (size_t)((n + kMinTile - 1) / kMinTile) + 1;
    return kHeaderBytes + cnt + ntiles * 2 * kPairBytes;
}

template <typename T, int VAR>
__global__ void csr_prepare(const int64_t* __restrict__ off, int64_t nseg, int64_t n,
                            void* __restrict__ out, unsigned char* __restrict__ ws, int out_f64) {
    using G = typename GridAcc<T, VAR>::type;
    WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
    unsigned int* cnt = reinterpret_cast<unsigned int*>(ws + kWsHeader);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s <= nseg; s += stride) {
        const int64_t a = off[s];
        bad |= (a < 0) || (a > n) || (s == 0 && a != 0);
        if (s < nseg) {
            const int64_t b = off[s + 1];
            bad |= (b < a);
            cnt[s] = 0u;
            if (b == a) write_out<T, VAR, G>(out, s, G(0), G(0), out_f64 != 0);
        }
    }
    if (bad) {
        atomicExch(&hdr->call_bad, 1);
        atomicExch(&hdr->error, kTfErrOffsets);
    }
}

template <typename T, int VAR, bool DOT, int U>
__global__ void __launch_bounds__(512)
csr_kernel(const T* __restrict__ x, const T* __restrict__ y, const int64_t* __restrict__ off,
           int64_t nseg, void* __restrict__ out, unsigned char* __restrict__ ws,
           size_t cnt_bytes, int64_t tile, int aligned, int out_f64) {
    using A = typename Acc<T, VAR>::type;
    using G = typename GridAcc<T, VAR>::type;
    constexpr bool TW = twofold_v<VAR>;
    constexpr int V = 16 / sizeof(T);
    constexpr int C = U * V;

    WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
    unsigned int* cnt = reinterpret_cast<unsigned int*>(ws + kWsHeader);
    G* pieces = reinterpret_cast<G*>(ws + kWsHeader + cnt_bytes);
    const int lane = threadIdx.x & 31;

    const bool bad = *reinterpret_cast<volatile int*>(&hdr->call_bad) != 0;
    if (bad) {
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        const G qnan = G(__int_as_float(0x7fffffff));
        for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += stride)
            write_out<T, VAR, G>(out, s, qnan, qnan, out_f64 != 0);
    } else {
        const int64_t total = off[nseg];
        const int64_t ntiles = (total + tile - 1) / tile;
        const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
        const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
        const int64_t t0 = ntiles * gw / nw, t1 = ntiles * (gw + 1) / nw;
        if (t0 < t1) {
            // segment holding element t0*tile: the last s < nseg with off[s] <= pos
            int64_t s = 0;
            if (lane == 0) {
                const int64_t pos = t0 * tile;
                int64_t lo = 0, hi = nseg;
                while (hi - lo > 1) {
                    const int64_t mid = lo + (hi - lo) / 2;
                    if (off[mid] <= pos) lo = mid; else hi = mid;
                }
                s = lo;
            }
            s = __shfl_sync(FULL, s, 0);
            int64_t a = off[s], b = off[s + 1];
            for (int64_t t = t0; t < t1; ++t) {
                const int64_t tlo = t * tile;
                const int64_t thi = min(tlo + tile, total);
                for (;;) {
                    const int64_t pa = max(a, tlo), pb = min(b, thi);
                    if (pb > pa) {
                        // ---- the piece [pa, pb) of segment s in tile t
                        A cs[C], ce[C];
#pragma unroll
                        for (int c = 0; c < C; ++c) { cs[c] = A(0); ce[c] = A(0); }
                        const int64_t qa = (pa - tlo) / V, qb = (pb - 1 - tlo) / V;
                        const int64_t mlo = qa > lane ? (qa - lane + 31) / 32 : 0;
                        const int64_t mhi = qb >= lane ? (qb - lane) / 32 : -1;
                        for (int64_t mb = (mlo / U) * U; mb <= mhi; mb += U) {
                            T xv[U][V], yv[U][V];
                            // Kahan chains skip the slots outside the piece (a +0 item
                            // would apply their pending compensation); every other
                            // variant takes them as +0, which leaves its bits unchanged
                            unsigned int live = ~0u;
                            // slot addresses grow with m, so the step's U vectors all lie
                            // inside the piece iff its first and last ones do
                            const int64_t b0 = tlo + (lane + 32 * mb) * V;
                            const int64_t b1 = b0 + (int64_t)(32 * V) * (U - 1);
                            if (mb >= mlo && mb + (U - 1) <= mhi && b0 >= pa && b1 + V <= pb) {
#pragma unroll
                                for (int u = 0; u < U; ++u) {
                                    ld_vec<T, V>(x + b0 + (int64_t)(32 * V) * u, aligned, xv[u]);
                                    if constexpr (DOT) ld_vec<T, V>(y + b0 + (int64_t)(32 * V) * u, aligned, yv[u]);
                                }
                            } else {
#pragma unroll
                                for (int u = 0; u < U; ++u) {
                                    const int64_t m = mb + u;
                                    const int64_t base = b0 + (int64_t)(32 * V) * u;
                                    if (m >= mlo && m <= mhi && base >= pa && base + V <= pb) {
                                        ld_vec<T, V>(x + base, aligned, xv[u]);
                                        if constexpr (DOT) ld_vec<T, V>(y + base, aligned, yv[u]);
                                    } else {
#pragma unroll
                                        for (int l = 0; l < V; ++l) {
                                            const int64_t i = base + l;
                                            const bool in = m >= mlo && m <= mhi && i >= pa && i < pb;
                                            xv[u][l] = in ? x[i] : T(0);
                                            if constexpr (DOT) yv[u][l] = in ? y[i] : T(0);
                                            if (!in) live &= ~(1u << (u * V + l));
                                        }
                                    }
                                }
                            }
#pragma unroll
                            for (int u = 0; u < U; ++u)
#pragma unroll
                                for (int l = 0; l < V; ++l) {
                                    if (step_v<VAR> == KAHAN && !((live >> (u * V + l)) & 1u)) continue;
                                    feed<VAR, DOT>(cs[u * V + l], ce[u * V + l], xv[u][l],
                                                   DOT ? yv[u][l] : T(0));
                                }
                        }
#pragma unroll
                        for (int w = C / 2; w >= 1; w >>= 1)
#pragma unroll
                            for (int c = 0; c < w; ++c) merge<TW>(cs[c], ce[c], cs[c + w], ce[c + w]);
                        A pv = cs[0], pe = ce[0];
                        warp_fold<TW>(pv, pe);

                        if (a >= tlo && b <= thi) {
                            // the whole segment lies in this tile
                            if (lane == 0) write_out<T, VAR, G>(out, s, (G)pv, (G)pe, out_f64 != 0);
                        } else {
                            const int64_t w0 = a / tile, w1 = (b - 1) / tile;
                            const int64_t k = w1 - w0 + 1;
                            const int64_t slot = (a < tlo) ? 2 * t : 2 * t + 1;
                            unsigned int old = 0;
                            if (lane == 0) {
                                pieces[2 * slot] = (G)pv;
                                pieces[2 * slot + 1] = (G)pe;
                                __threadfence();
                                old = atomicAdd(&cnt[s], 1u);
                            }
                            old = __shfl_sync(FULL, old, 0);
                            if ((int64_t)old == k - 1) {
                                // last piece of the segment: merge the k pieces in tile order
                                __threadfence();
                                G gv = G(0), ge = G(0);
                                if (lane < k) {
                                    const int64_t s0 = (lane == 0) ? 2 * w0 + 1 : 2 * (w0 + lane);
                                    ld_pair_cg(pieces + 2 * s0, gv, ge);
                                    for (int64_t i = lane + 32; i < k; i += 32) {
                                        G v2, e2;
                                        ld_pair_cg(pieces + 2 * (2 * (w0 + i)), v2, e2);
                                        merge<TW>(gv, ge, v2, e2);
                                    }
                                }
                                warp_fold<TW>(gv, ge);
                                if (lane == 0) {
                                    write_out<T, VAR, G>(out, s, gv, ge, out_f64 != 0);
                                    cnt[s] = 0u;
                                }
                            }
                        }
                    }
                    if (b > thi) break;                 // segment continues in the next tile
                    if (++s >= nseg) break;
                    a = b;
                    b = off[s + 1];
                    if (a >= thi) break;                // next segment starts in a later tile
                }
            }
        }
    }

    // the last block to finish clears the per-call flag
    __syncthreads();
    __shared__ int am_last;
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int t = atomicAdd(&hdr->ticket2, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (am_last && threadIdx.x == 0) {
        hdr->call_bad = 0;
        hdr->ticket2 = 0u;
    }
}

template <typename T, int VAR, bool DOT>
static cudaError_t launch_u(int unroll, const void* x, const void* y, int64_t n,
                            const int64_t* off, int64_t nseg, void* out, void* ws,
                            size_t ws_bytes, int block, int64_t grid, int64_t tile, int aligned,
                            int out_f64, cudaStream_t st) {
    (void)ws_bytes;
    unsigned char* w = static_cast<unsigned char*>(ws);
    const size_t cnt_bytes = ((size_t)(nseg > 0 ? nseg : 1) * 4 + 255) / 256 * 256;
    const int pblocks = (int)std::min<int64_t>(1024, (nseg + 1 + 255) / 256);
    csr_prepare<T, VAR><<<pblocks, 256, 0, st>>>(off, nseg, n, out, w, out_f64);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    const T* xp = static_cast<const T*>(x);
    const T* yp = static_cast<const T*>(y);
    switch (unroll) {
    case 1: csr_kernel<T, VAR, DOT, 1><<<(unsigned)grid, block, 0, st>>>(xp, yp, off, nseg, out, w, cnt_bytes, tile, aligned, out_f64); break;
    case 2: csr_kernel<T, VAR, DOT, 2><<<(unsigned)grid, block, 0, st>>>(xp, yp, off, nseg, out, w, cnt_bytes, tile, aligned, out_f64); break;
    case 4: csr_kernel<T, VAR, DOT, 4><<<(unsigned)grid, block, 0, st>>>(xp, yp, off, nseg, out, w, cnt_bytes, tile, aligned, out_f64); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T, int VAR>
static cudaError_t launch_d(int dot, int unroll, const void* x, const void* y, int64_t n,
                            const int64_t* off, int64_t nseg, void* out, void* ws,
                            size_t ws_bytes, int block, int64_t grid, int64_t tile, int aligned,
                            int out_f64, cudaStream_t st) {
    return dot ? launch_u<T, VAR, true>(unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, out_f64, st)
               : launch_u<T, VAR, false>(unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, out_f64, st);
}

cudaError_t launch_csr(int dtype, int variant, int dot, int unroll, const void* x,
                       const void* y, int64_t n, const int64_t* off, int64_t nseg,
                       void* out, void* ws, size_t ws_bytes, int block, int64_t grid,
                       int64_t tile, int aligned, int out_f64, cudaStream_t st) {
    if (dtype == 0) {
        switch (variant) {
        case PLAIN: return launch_d<float, PLAIN>(dot, unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, out_f64, st);
        case FAST: return launch_d<float, FAST>(dot, unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, out_f64, st);
        case RIGOROUS: return launch_d<float, RIGOROUS>(dot, unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, out_f64, st);
        case WIDE: return launch_d<float, WIDE>(dot, unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, out_f64, st);
        case KAHAN: return launch_d<float, KAHAN>(dot, unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, out_f64, st);
        case FAST_LIT: return dot ? launch_u<float, FAST_LIT, true>(unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, out_f64, st) : cudaErrorInvalidValue;
        case RIG_LIT: return dot ? launch_u<float, RIG_LIT, true>(unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, out_f64, st) : cudaErrorInvalidValue;
        }
    } else {
        switch (variant) {
        case PLAIN: return launch_d<double, PLAIN>(dot, unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, out_f64, st);
        case FAST: return launch_d<double, FAST>(dot, unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, out_f64, st);
        case RIGOROUS: return launch_d<double, RIGOROUS>(dot, unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, out_f64, st);
        case WIDE: return launch_d<double, WIDE>(dot, unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, out_f64, st);
        case KAHAN: return launch_d<double, KAHAN>(dot, unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, out_f64, st);
        case FAST_LIT: return dot ? launch_u<double, FAST_LIT, true>(unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, out_f64, st) : cudaErrorInvalidValue;
        case RIG_LIT: return dot ? launch_u<double, RIG_LIT, true>(unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, out_f64, st) : cudaErrorInvalidValue;
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace tf
