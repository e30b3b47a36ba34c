// tf_csr.cu -- twofold sums / dots of many ragged CSR segments in one
// persistent launch (sm_103a).
//
// Load balance does not depend on the length mix: the concatenated vector is
// cut into equal tiles of `tile` elements, and the warps of the persistent
// grid take tiles from a per-call counter in increasing order (one atomic per
// tile), so all warps stream one moving window of the input and finish
// within one tile of each other.  Inside a tile the warp reduces each
// segment's piece: lane l takes the 16-byte vector slots l, l+32, ... of the
// tile, slot m feeding chains (m mod U)*V + (element mod V).  Elements
// outside the piece are fed as +0, which leaves a twofold, plain or wide
// chain's bits unchanged (Kahan chains skip them), so the chain assignment is
// the documented one.  A segment inside one tile is written directly.  The
// pieces of a segment over 2..32 tiles are stored, and a merge kernel
// launched after the reduction merges them (one thread per segment; its wait
// for the reduction grid to complete orders the stores before its loads: no
// atomics on the streaming warps); over more than 32 tiles they merge by a
// pairwise tree in tile order, each merge done by the warp that completes the
// second of its two children (arrival counters, no waiting).  Which warp
// reduces which tile never changes a bit.  A first small kernel checks the
// offsets, clears the counters, writes the empty segments and records the
// segment holding each tile's first element.
#include "tf_csr.cuh"

namespace tf {

constexpr int kTfErrOffsets = 6;       // TF_ERR_OFFSETS
constexpr int kMergeThreads = 256;     // csr_merge: one thread per tile

size_t csr_ws_bytes(int64_t n, int64_t nseg) {
    (void)nseg;
    const size_t ntiles = csr_max_tiles(n);
    return kHeaderBytes + csr_cnt_bytes(n) + ntiles * 2 * kPairBytes + ntiles * 8;
}

template <typename T, int VAR>
__global__ void csr_prepare(const int64_t* __restrict__ off, int64_t nseg, int64_t n,
                            int64_t tile, void* __restrict__ out, unsigned char* __restrict__ ws,
                            int64_t* __restrict__ tile_seg, int out_f64) {
    using G = typename GridAcc<T, VAR>::type;
    grid_dependents_go();
    WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
    unsigned int* cnt = reinterpret_cast<unsigned int*>(ws + kWsHeader);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t first = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    for (int64_t s = first; s <= nseg; s += stride) {
        const int64_t a = off[s];
        bad |= (a < 0) || (a > n) || (s == 0 && a != 0);
        if (s < nseg) {
            const int64_t b = off[s + 1];
            bad |= (b < a);
            if (b == a) write_out<T, VAR, G>(out, s, G(0), G(0), out_f64 != 0);
        }
    }
    // the segment holding element t*tile: the last s < nseg with off[s] <= t*tile
    // (indices stay in [0, nseg] whatever the offsets hold; with invalid
    // offsets the map is not used)
    const int64_t ntiles = (n + tile - 1) / tile;
    for (int64_t t = first; t < ntiles; t += stride) {
        cnt[2 * t] = 0u;                      // the arrival counters of the tile's two slots
        cnt[2 * t + 1] = 0u;
        const int64_t pos = t * tile;
        int64_t lo = 0, hi = nseg;
        while (hi - lo > 1) {
            const int64_t mid = lo + (hi - lo) / 2;
            if (off[mid] <= pos) lo = mid; else hi = mid;
        }
        tile_seg[t] = lo;
    }
    if (bad) {
        atomicExch(&hdr->call_bad, 1);
        atomicExch(&hdr->error, kTfErrOffsets);
    }
}

// binary64 data (not wide): registers for 3 blocks of 512 threads at U = 1
// (the occupancy of the single-vector kernel), 2 at U = 2; the integer-pipe
// arithmetic needs the warps, and the compiler fits these without spilling
template <typename T, int VAR, bool DOT, int U>
__global__ void __launch_bounds__(512, (sizeof(T) == 8 && VAR != WIDE) ? (U == 1 ? 3 : (U == 2 ? 2 : 1)) : 1)
csr_kernel(const T* __restrict__ x, const T* __restrict__ y, const int64_t* __restrict__ off,
           int64_t nseg, void* __restrict__ out, unsigned char* __restrict__ ws,
           size_t cnt_bytes, const int64_t* __restrict__ tile_seg, int64_t tile, int aligned,
           int out_f64) {
    using A = typename Acc<T, VAR>::type;
    using G = typename GridAcc<T, VAR>::type;
    constexpr int V = 16 / sizeof(T);
    constexpr int C = U * V;
    constexpr int SV = 32 * V;              // elements per warp-wide slot row
    // load the next full step while the current one is fed: binary32 data
    // (it streams at the memory's pace) and the binary64 twofold sums (their
    // arithmetic outlasts a load only with many warps per SM); the binary64
    // dots and the wide kernels keep the registers instead (measured)
    constexpr bool PREFETCH = (sizeof(T) == 4 && VAR != WIDE) ||
                              (sizeof(T) == 8 && !DOT && (VAR == FAST || VAR == RIGOROUS));

    grid_wait();                      // the offsets check has completed
    grid_dependents_go();
    WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
    unsigned int* cnt = reinterpret_cast<unsigned int*>(ws + kWsHeader);
    G* pieces = reinterpret_cast<G*>(ws + kWsHeader + cnt_bytes);
    const int lane = threadIdx.x & 31;
    double one = 1.0;                 // binary64 data, wide: a 1.0 the compiler cannot see
    if constexpr (sizeof(T) == 8 || VAR == WIDE) one = *reinterpret_cast<volatile double*>(&g_one);

    const bool bad = *reinterpret_cast<volatile int*>(&hdr->call_bad) != 0;
    if (bad) {
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        const G qnan = G(__int_as_float(0x7fffffff));
        for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += stride)
            write_out<T, VAR, G>(out, s, qnan, qnan, out_f64 != 0);
    } else {
        const int64_t total = off[nseg];
        const int64_t ntiles = (total + tile - 1) / tile;
        unsigned long long t = 0ull;
        if (lane == 0) t = atomicAdd(&hdr->tile_next, 1ull);
        t = __shfl_sync(FULL, t, 0);
        while ((int64_t)t < ntiles) {
            // claim the next tile now; the answer is needed only after this one
            unsigned long long tn = 0ull;
            if (lane == 0) tn = atomicAdd(&hdr->tile_next, 1ull);
            const int64_t tlo = (int64_t)t * tile;
            const int64_t thi = min(tlo + tile, total);
            int64_t s = __ldg(tile_seg + t);
            int64_t a = __ldg(off + s), b = __ldg(off + s + 1);
            int64_t bn = __ldg(off + min(s + 2, nseg));   // the next segment's end, loaded ahead
            for (;;) {
                const int64_t pa = max(a, tlo), pb = min(b, thi);
                if (pb > pa) {
                    // ---- the piece [pa, pb) of segment s in tile t
                    A cs[C], ce[C];
#pragma unroll
                    for (int c = 0; c < C; ++c) { cs[c] = A(0); ce[c] = A(0); }
                    // this lane's slots m touching the piece: [mlo, mhi]; lying
                    // wholly inside it: [mA, mB] (tile-relative, 32-bit: tile <= 2^22)
                    const int ra = (int)(pa - tlo), rb = (int)(pb - tlo);
                    const int qa = ra / V, qb = (rb - 1) / V;
                    const int mlo = qa > lane ? (qa - lane + 31) / 32 : 0;
                    const int mhi = qb >= lane ? (qb - lane) / 32 : -1;
                    const int da = ra - lane * V, db = rb - V - lane * V;
                    const int mA = da > 0 ? (da + SV - 1) / SV : 0;
                    const int mB = db >= 0 ? db / SV : -1;
                    const T* xl = x + tlo + lane * V;
                    const T* yl = DOT ? y + tlo + lane * V : nullptr;

                    auto feed_step = [&](const T (&xv)[U][V], const T (&yv)[U][V], unsigned int live) {
#pragma unroll
                        for (int u = 0; u < U; ++u)
#pragma unroll
                            for (int l = 0; l < V; ++l) {
                                if (step_v<VAR> == KAHAN && !((live >> (u * V + l)) & 1u)) continue;
                                feed<VAR, DOT>(cs[u * V + l], ce[u * V + l], xv[u][l],
                                               DOT ? yv[u][l] : T(0), one);
                            }
                    };
                    auto load_full = [&](int mb, T (&xv)[U][V], T (&yv)[U][V]) {
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            ld_vec<T, V>(xl + (mb + u) * SV, aligned, xv[u]);
                            if constexpr (DOT) ld_vec<T, V>(yl + (mb + u) * SV, aligned, yv[u]);
                        }
                    };
                    // a step with slots outside the piece: those elements are +0
                    // (Kahan chains skip them)
                    auto partial_step = [&](int mb) {
                        T xv[U][V], yv[U][V];
                        unsigned int live = ~0u;
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const int m = mb + u;
                            if (m >= mA && m <= mB) {
                                ld_vec<T, V>(xl + m * SV, aligned, xv[u]);
                                if constexpr (DOT) ld_vec<T, V>(yl + m * SV, aligned, yv[u]);
                            } else {
#pragma unroll
                                for (int l = 0; l < V; ++l) {
                                    const int r = m * SV + l;      // offset from xl
                                    const int i = r + lane * V;    // tile-relative index
                                    const bool in = m >= mlo && m <= mhi && i >= ra && i < rb;
                                    xv[u][l] = in ? xl[r] : T(0);
                                    if constexpr (DOT) yv[u][l] = in ? yl[r] : T(0);
                                    if (!in) live &= ~(1u << (u * V + l));
                                }
                            }
                        }
                        feed_step(xv, yv, live);
                    };

                    // steps mb = (mlo/U)*U, ... <= mhi, in order: partial ones,
                    // then those wholly inside the piece, then partial ones
                    const int full0 = (mA + U - 1) / U * U;
                    int mb = (mlo / U) * U;
                    for (; mb < full0 && mb <= mhi; mb += U) partial_step(mb);
                    if (mb + (U - 1) <= mB) {
                        if constexpr (PREFETCH) {
                            T xv[U][V], yv[U][V];
                            load_full(mb, xv, yv);
                            for (;;) {
                                const int mn = mb + U;
                                const bool more = mn + (U - 1) <= mB;
                                T xn[U][V], yn[U][V];
                                if (more) load_full(mn, xn, yn);
                                feed_step(xv, yv, ~0u);
                                mb = mn;
                                if (!more) break;
#pragma unroll
                                for (int u = 0; u < U; ++u)
#pragma unroll
                                    for (int l = 0; l < V; ++l) {
                                        xv[u][l] = xn[u][l];
                                        if constexpr (DOT) yv[u][l] = yn[u][l];
                                    }
                            }
                        } else {
                            for (; mb + (U - 1) <= mB; mb += U) {
                                T xv[U][V], yv[U][V];
                                load_full(mb, xv, yv);
                                feed_step(xv, yv, ~0u);
                            }
                        }
                    }
                    for (; mb <= mhi; mb += U) partial_step(mb);

                    piece_finish<T, VAR, C>(cs, ce, s, a, b, (int64_t)t, tlo, thi, tile, out, cnt,
                                            pieces, lane, out_f64);
                }
                if (b > thi) break;                 // segment continues in the next tile
                if (++s >= nseg) break;
                a = b;
                b = bn;
                bn = __ldg(off + min(s + 2, nseg));
                if (a >= thi) break;                // next segment starts in a later tile
            }
            t = __shfl_sync(FULL, tn, 0);
        }
    }
}

// The segments over 2..32 tiles, after the reduction kernel has stored their
// piece pairs: thread t reads k from the word of slot 2t + 1 (0 unless a
// segment over k >= 2 tiles starts in tile t; the offsets check cleared it)
// and merges that segment's k pieces in the butterfly order
// (butterfly_node); the segment is the one holding tile t + 1's first
// element.  The reduction kernel has finished, so thread 0 clears the
// per-call flag and the tile counter.
template <typename T, int VAR>
__global__ void __launch_bounds__(kMergeThreads)
csr_merge(void* __restrict__ out, unsigned char* __restrict__ ws, size_t cnt_bytes,
          const int64_t* __restrict__ tile_seg, int64_t ntiles, int out_f64) {
    using G = typename GridAcc<T, VAR>::type;
    constexpr bool TW = twofold_v<VAR>;
    grid_wait();                      // the reduction has completed
    const unsigned int* cnt = reinterpret_cast<const unsigned int*>(ws + kWsHeader);
    const G* pieces = reinterpret_cast<const G*>(ws + kWsHeader + cnt_bytes);
    const int64_t t = (int64_t)blockIdx.x * kMergeThreads + threadIdx.x;
    if (t == 0) {
        WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
        hdr->call_bad = 0;
        hdr->tile_next = 0ull;
    }
    if (t + 1 >= ntiles) return;
    const int k = (int)cnt[2 * t + 1];
    if (k < 2) return;
    const int64_t s = __ldg(tile_seg + t + 1);
    G v, e;
    if (k <= 2) butterfly_node<1, 2, TW>(pieces, t, k, 0, v, e);
    else if (k <= 4) butterfly_node<1, 4, TW>(pieces, t, k, 0, v, e);
    else if (k <= 8) butterfly_node<1, 8, TW>(pieces, t, k, 0, v, e);
    else if (k <= 16) butterfly_node<1, 16, TW>(pieces, t, k, 0, v, e);
    else butterfly_node<1, 32, TW>(pieces, t, k, 0, v, e);
    write_out<T, VAR, G>(out, s, v, e, out_f64 != 0);
}

template <typename T, int VAR, bool DOT>
static cudaError_t launch_u(int unroll, const void* x, const void* y, int64_t n,
                            const int64_t* off, int64_t nseg, void* out, void* ws,
                            size_t ws_bytes, int block, int64_t grid, int64_t tile, int aligned,
                            int staged, int out_f64, cudaStream_t st) {
    (void)ws_bytes;
    unsigned char* w = static_cast<unsigned char*>(ws);
    const size_t cnt_bytes = csr_cnt_bytes(n);
    int64_t* tile_seg = reinterpret_cast<int64_t*>(w + kHeaderBytes + cnt_bytes +
                                                   csr_max_tiles(n) * 2 * kPairBytes);
    const int64_t items = std::max<int64_t>(nseg + 1, (n + tile - 1) / tile);
    const int pblocks = (int)std::min<int64_t>(1024, (items + 255) / 256);
    csr_prepare<T, VAR><<<pblocks, 256, 0, st>>>(off, nseg, n, tile, out, w, tile_seg, out_f64);
    cudaError_t err = cudaGetLastError();
    const int64_t* ctile_seg = tile_seg;
    if (err != cudaSuccess) return err;
    if (aligned && staged && csr_tma_usable(sizeof(T) == 4 ? 0 : 1, DOT ? 1 : 0, block, tile)) {
        err = launch_csr_tma(sizeof(T) == 4 ? 0 : 1, VAR, DOT ? 1 : 0, unroll, x, y, off, nseg, out,
                             w, cnt_bytes, tile_seg, block, grid, tile, out_f64, st);
    } else {
        const T* xp = static_cast<const T*>(x);
        const T* yp = static_cast<const T*>(y);
        switch (unroll) {
        case 1: err = launch_dependent(csr_kernel<T, VAR, DOT, 1>, (unsigned)grid, (unsigned)block, 0, st, xp, yp, off, nseg, out, w, cnt_bytes, ctile_seg, tile, aligned, out_f64); break;
        case 2: err = launch_dependent(csr_kernel<T, VAR, DOT, 2>, (unsigned)grid, (unsigned)block, 0, st, xp, yp, off, nseg, out, w, cnt_bytes, ctile_seg, tile, aligned, out_f64); break;
        case 4: err = launch_dependent(csr_kernel<T, VAR, DOT, 4>, (unsigned)grid, (unsigned)block, 0, st, xp, yp, off, nseg, out, w, cnt_bytes, ctile_seg, tile, aligned, out_f64); break;
        default: return cudaErrorInvalidValue;
        }
    }
    if (err != cudaSuccess) return err;
    // one thread per tile of n elements (they cover those of offsets[nseg] <= n;
    // the words of tiles past offsets[nseg] stay 0)
    const int64_t ntiles = (n + tile - 1) / tile;
    const int64_t mblocks = std::max<int64_t>(1, (ntiles + kMergeThreads - 1) / kMergeThreads);
    return launch_dependent(csr_merge<T, VAR>, (unsigned)mblocks, (unsigned)kMergeThreads, 0, st,
                            out, w, cnt_bytes, ctile_seg, ntiles, out_f64);
}

template <typename T, int VAR>
static cudaError_t launch_d(int dot, int unroll, const void* x, const void* y, int64_t n,
                            const int64_t* off, int64_t nseg, void* out, void* ws,
                            size_t ws_bytes, int block, int64_t grid, int64_t tile, int aligned,
                            int staged, int out_f64, cudaStream_t st) {
    return dot ? launch_u<T, VAR, true>(unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, staged, out_f64, st)
               : launch_u<T, VAR, false>(unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, staged, out_f64, st);
}

cudaError_t launch_csr(int dtype, int variant, int dot, int unroll, const void* x,
                       const void* y, int64_t n, const int64_t* off, int64_t nseg,
                       void* out, void* ws, size_t ws_bytes, int block, int64_t grid,
                       int64_t tile, int aligned, int staged, int out_f64, cudaStream_t st) {
    if (dtype == 0) {
        switch (variant) {
        case PLAIN: return launch_d<float, PLAIN>(dot, unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, staged, out_f64, st);
        case FAST: return launch_d<float, FAST>(dot, unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, staged, out_f64, st);
        case RIGOROUS: return launch_d<float, RIGOROUS>(dot, unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, staged, out_f64, st);
        case WIDE: return launch_d<float, WIDE>(dot, unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, staged, out_f64, st);
        case KAHAN: return launch_d<float, KAHAN>(dot, unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, staged, out_f64, st);
        case FAST_LIT: return dot ? launch_u<float, FAST_LIT, true>(unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, staged, out_f64, st) : cudaErrorInvalidValue;
        case RIG_LIT: return dot ? launch_u<float, RIG_LIT, true>(unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, staged, out_f64, st) : cudaErrorInvalidValue;
        }
    } else {
        switch (variant) {
        case PLAIN: return launch_d<double, PLAIN>(dot, unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, staged, out_f64, st);
        case FAST: return launch_d<double, FAST>(dot, unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, staged, out_f64, st);
        case RIGOROUS: return launch_d<double, RIGOROUS>(dot, unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, staged, out_f64, st);
        case WIDE: return launch_d<double, WIDE>(dot, unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, staged, out_f64, st);
        case KAHAN: return launch_d<double, KAHAN>(dot, unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, staged, out_f64, st);
        case FAST_LIT: return dot ? launch_u<double, FAST_LIT, true>(unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, staged, out_f64, st) : cudaErrorInvalidValue;
        case RIG_LIT: return dot ? launch_u<double, RIG_LIT, true>(unroll, x, y, n, off, nseg, out, ws, ws_bytes, block, grid, tile, aligned, staged, out_f64, st) : cudaErrorInvalidValue;
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace tf
