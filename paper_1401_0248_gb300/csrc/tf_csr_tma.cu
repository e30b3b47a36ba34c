// tf_csr_tma.cu -- the batched kernel with its input staged through shared
// memory by bulk copies (sm_103a, cp.async.bulk + mbarrier).
//
// Same order, same bits as csr_kernel: tiles are claimed from the per-call
// counter, a tile's segment pieces are fed slot row by slot row (lane l
// takes the 16-byte vector l of each 32-vector row, row m feeding chains
// (m mod U)*V + l), and pieces end in piece_finish.  What differs is how the
// data arrive: each warp owns a ring of kStages chunks of kRows rows in
// shared memory; lane 0 keeps the ring full with one bulk copy per chunk per
// operand (completion counted in bytes on the stage's mbarrier), running up
// to kStages - 1 chunks ahead of the consumer, across the tile boundary into
// the next claimed tile.  The warp's loads are then no longer tied to its
// control flow: the copies in flight keep streaming while the warp folds a
// piece, writes a result or waits for the next tile's segment index.
//
// Elements beyond the last whole 16-byte vector of the input (fewer than
// 16/sizeof(T)) are read from global memory directly.  Every wait is bounded;
// a wait that gives up sets TF_ERR_TIMEOUT in the workspace's error word,
// waits (bounded again) for the warp's copies in flight and ends the warp's
// work; if that wait gives up as well the error word becomes
// TF_ERR_UNDRAINED (copies may land after the block exits).
#include "tf_async.cuh"
#include "tf_csr.cuh"

#include <atomic>

namespace tf {

namespace {

constexpr int kRows = 8;                       // slot rows per chunk
constexpr int kRowBytes = 32 * 16;             // one row: 32 lanes x 16 bytes
constexpr int kChunkBytes = kRows * kRowBytes;  // 4 KiB per operand
constexpr int kStages = 3;
constexpr int kMaxWarps = 16;
constexpr int kTfErrTimeout = 7;               // TF_ERR_TIMEOUT
constexpr int kTfErrUndrained = 9;             // TF_ERR_UNDRAINED
constexpr unsigned kWaitLimit = 1u << 20;      // try_wait rounds before giving up


}  // namespace

template <typename T, int VAR, bool DOT, int U>
__global__ void __launch_bounds__(512)
csr_tma_kernel(const T* __restrict__ x, const T* __restrict__ y, const int64_t* __restrict__ off,
               int64_t nseg, void* __restrict__ out, unsigned char* __restrict__ ws,
               size_t cnt_bytes, const int64_t* __restrict__ tile_seg, int64_t tile,
               int out_f64) {
    using A = typename Acc<T, VAR>::type;
    using G = typename GridAcc<T, VAR>::type;
    constexpr int V = 16 / sizeof(T);
    constexpr int C = U * V;
    constexpr int SV = 32 * V;                 // elements per row
    constexpr int CE = kRows * SV;             // elements per chunk
    constexpr int NOPS = DOT ? 2 : 1;
    constexpr int kStageBytes = kChunkBytes * NOPS;
    static_assert(kRows % U == 0, "a step of U rows stays inside one chunk");

    extern __shared__ __align__(128) unsigned char ring_all[];
    __shared__ __align__(8) unsigned long long bars[kMaxWarps * kStages];

    grid_wait();                      // the offsets check has completed
    grid_dependents_go();
    WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
    unsigned int* cnt = reinterpret_cast<unsigned int*>(ws + kWsHeader);
    G* pieces = reinterpret_cast<G*>(ws + kWsHeader + cnt_bytes);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    double one = 1.0;                 // binary64 data, wide: a 1.0 the compiler cannot see
    if constexpr (sizeof(T) == 8 || VAR == WIDE) one = *reinterpret_cast<volatile double*>(&g_one);

    const uint32_t ring = smem_u32(ring_all) + (uint32_t)(wib * kStages * kStageBytes);
    const uint32_t bar0 = smem_u32(&bars[wib * kStages]);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < kStages; ++i) mbar_init(bar0 + 8 * i, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();

    const bool bad = *reinterpret_cast<volatile int*>(&hdr->call_bad) != 0;
    if (bad) {
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        const G qnan = G(__int_as_float(0x7fffffff));
        for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += stride)
            write_out<T, VAR, G>(out, s, qnan, qnan, out_f64 != 0);
    } else {
        const int64_t total = off[nseg];
        const int64_t ntiles = (total + tile - 1) / tile;
        const int64_t vend = total - total % V;   // the bulk copies end at this element
        auto nchunks = [&](int64_t tt) { return (min(tt * tile + tile, total) - tt * tile + CE - 1) / CE; };

        // consumer: tile t, its chunk 0 is chunk number kbase of this warp's
        // sequence; producer: next chunk (pt, pc); chunks issued / freed
        unsigned long long t = 0ull, tn_raw = 0ull;
        if (lane == 0) t = atomicAdd(&hdr->tile_next, 1ull);
        t = __shfl_sync(FULL, t, 0);
        if (lane == 0) tn_raw = atomicAdd(&hdr->tile_next, 1ull);
        int64_t tn = -1;                          // the next tile, once read
        int64_t sn = -1;                          // its first segment, loaded when tn is read
        int64_t pt = (int64_t)t, pc = 0, pnc = (int64_t)t < ntiles ? nchunks((int64_t)t) : 0;
        uint32_t issued = 0, freed = 0, kbase = 0;
        bool failed = false;

        // lane 0 issues chunks while the ring has room: the rest of tile t,
        // then the next claimed tile (read from the claim only when needed)
        auto top_up = [&]() {
            while (issued < freed + kStages) {
                if (pc >= pnc) {
                    if (pt != (int64_t)t) break;            // one tile ahead at most
                    if (tn < 0) {
                        tn = (int64_t)__shfl_sync(FULL, tn_raw, 0);
                        if (tn < ntiles) sn = __ldg(tile_seg + tn);   // used at the tile's start
                    }
                    if (tn >= ntiles) break;
                    pt = tn;
                    pc = 0;
                    pnc = nchunks(pt);
                }
                if (lane == 0) {
                    const int64_t e0 = pt * tile + pc * CE;
                    const int64_t e1 = min(min(e0 + CE, pt * tile + tile), vend);
                    const uint32_t bytes = e1 > e0 ? (uint32_t)((e1 - e0) * (int64_t)sizeof(T)) : 0u;
                    const uint32_t st = issued % kStages;
                    const uint32_t bar = bar0 + 8 * st;
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_arrive_expect_tx(bar, bytes * NOPS);
                    if (bytes) {
                        bulk_load(ring + st * kStageBytes, x + e0, bytes, bar);
                        if constexpr (DOT) bulk_load(ring + st * kStageBytes + kChunkBytes, y + e0, bytes, bar);
                    }
                }
                ++issued;
                ++pc;
            }
        };

        while (!failed && (int64_t)t < ntiles) {
            const int64_t tlo = (int64_t)t * tile;
            const int64_t thi = min(tlo + tile, total);
            // tile-relative end of the bulk-copied data (elements past it are
            // read from global memory)
            const int vrel = (int)max((int64_t)0, min(vend - tlo, tile));
            top_up();
            int64_t s = sn >= 0 ? sn : __ldg(tile_seg + t);
            sn = -1;
            int64_t a = __ldg(off + s), b = __ldg(off + s + 1);
            int64_t bn = __ldg(off + min(s + 2, nseg));   // the next segment's end, loaded ahead
            int cur = -1;                          // chunk of the tile being read

            // chunks before ch are read: free them, refill the ring, wait for ch
            auto ensure = [&](int ch) {
                if (ch == cur) return;
                __syncwarp();
                freed = kbase + (uint32_t)ch;
                top_up();
                const uint32_t k = kbase + (uint32_t)ch;
                const bool ok = mbar_wait(bar0 + 8 * (k % kStages), (k / kStages) & 1u, kWaitLimit);
                failed = __any_sync(FULL, !ok);
                cur = ch;
            };
            auto row_addr = [&](int row) {
                return ring + ((kbase + (uint32_t)(row / kRows)) % kStages) * kStageBytes +
                       (uint32_t)(((row % kRows) * 32 + lane) * 16);
            };

            for (;;) {
                const int64_t pa = max(a, tlo), pb = min(b, thi);
                if (pb > pa) {
                    A cs[C], ce[C];
#pragma unroll
                    for (int c = 0; c < C; ++c) { cs[c] = A(0); ce[c] = A(0); }
                    // tile-relative piece [ra, rb); rows m0..m1 touch it; steps
                    // mb in [fs, fe] lie wholly inside [ra, min(rb, vrel))
                    const int ra = (int)(pa - tlo), rb = (int)(pb - tlo);
                    const int rbv = min(rb, vrel);
                    const int m0 = ra / SV, m1 = (rb - 1) / SV;
                    const int fs = ((ra + SV - 1) / SV + U - 1) / U * U;
                    const int fe = rbv / SV - U;

                    // a step with elements outside the piece (+0; Kahan skips
                    // them) or past the bulk copies (read from global memory)
                    auto step_masked = [&](int mb) {
                        T xv[U][V], yv[U][V];
                        unsigned int live = ~0u;
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const int row = mb + u;
                            const uint32_t sa = row_addr(row);
                            ld_shared(sa, xv[u]);
                            if constexpr (DOT) ld_shared(sa + kChunkBytes, yv[u]);
#pragma unroll
                            for (int l = 0; l < V; ++l) {
                                const int i = row * SV + lane * V + l;
                                const bool in = i >= ra && i < rb;
                                if (in && i >= vrel) {
                                    xv[u][l] = x[tlo + i];
                                    if constexpr (DOT) yv[u][l] = y[tlo + i];
                                }
                                if (!in) {
                                    xv[u][l] = T(0);
                                    if constexpr (DOT) yv[u][l] = T(0);
                                    live &= ~(1u << (u * V + l));
                                }
                            }
                        }
#pragma unroll
                        for (int u = 0; u < U; ++u)
#pragma unroll
                            for (int l = 0; l < V; ++l) {
                                if (step_v<VAR> == KAHAN && !((live >> (u * V + l)) & 1u)) continue;
                                feed<VAR, DOT>(cs[u * V + l], ce[u * V + l], xv[u][l],
                                               DOT ? yv[u][l] : T(0), one);
                            }
                    };

                    int mb = (m0 / U) * U;
                    for (; !failed && mb <= m1 && mb < fs; mb += U) {
                        ensure(mb / kRows);
                        if (!failed) step_masked(mb);
                    }
                    // whole steps, a chunk at a time
                    while (!failed && mb <= fe) {
                        const int ch = mb / kRows;
                        ensure(ch);
                        if (failed) break;
                        const uint32_t cb = ring + ((kbase + (uint32_t)ch) % kStages) * kStageBytes +
                                            (uint32_t)(lane * 16);
                        const int mend = min(fe, (ch + 1) * kRows - U);
                        for (; mb <= mend; mb += U) {
                            T xv[U][V], yv[U][V];
#pragma unroll
                            for (int u = 0; u < U; ++u) {
                                const uint32_t sa = cb + (uint32_t)(((mb + u) % kRows) * kRowBytes);
                                ld_shared(sa, xv[u]);
                                if constexpr (DOT) ld_shared(sa + kChunkBytes, yv[u]);
                            }
#pragma unroll
                            for (int u = 0; u < U; ++u)
#pragma unroll
                                for (int l = 0; l < V; ++l)
                                    feed<VAR, DOT>(cs[u * V + l], ce[u * V + l], xv[u][l],
                                                   DOT ? yv[u][l] : T(0), one);
                        }
                    }
                    for (; !failed && mb <= m1; mb += U) {
                        ensure(mb / kRows);
                        if (!failed) step_masked(mb);
                    }
                    if (failed) break;
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
            if (failed) break;
            // every chunk of tile t is read; move to the next claimed tile
            __syncwarp();
            kbase += (uint32_t)nchunks((int64_t)t);
            freed = kbase;
            if (tn < 0) tn = (int64_t)__shfl_sync(FULL, tn_raw, 0);
            t = (unsigned long long)tn;
            tn = -1;
            if ((int64_t)t < ntiles && lane == 0) tn_raw = atomicAdd(&hdr->tile_next, 1ull);
            if (pt != (int64_t)t) {                          // nothing issued for it yet
                pt = (int64_t)t;
                pc = 0;
                pnc = (int64_t)t < ntiles ? nchunks((int64_t)t) : 0;
            }
        }
        if (failed) {
            if (lane == 0) atomicExch(&hdr->error, kTfErrTimeout);
            // let the copies still in flight land before the block can exit;
            // if one of these bounded waits gives up too, copies may still be
            // landing in this block's shared memory after it exits: that is
            // recorded as its own status (the results of the call are then
            // undefined and the workspace should be dropped)
            bool drained = true;
            for (uint32_t k = freed; k < issued; ++k)
                drained = mbar_wait(bar0 + 8 * (k % kStages), (k / kStages) & 1u, kWaitLimit) && drained;
            if (!drained && lane == 0) atomicExch(&hdr->error, kTfErrUndrained);
        }
    }
}

// shared memory of one block: kStages chunks per warp and operand
size_t csr_tma_smem_bytes(int dot, int block) {
    return (size_t)(block / 32) * kStages * kChunkBytes * (dot ? 2 : 1);
}

bool csr_tma_usable(int dtype, int dot, int block, int64_t tile) {
    const int64_t ce = (int64_t)kRows * 32 * (dtype == 0 ? 4 : 2);
    return block / 32 <= kMaxWarps && tile % ce == 0 && tile >= (int64_t)kStages * ce &&
           csr_tma_smem_bytes(dot, block) <= 200 * 1024;
}

template <typename T, int VAR, bool DOT, int U>
static cudaError_t launch_tma_u(const T* x, const T* y, const int64_t* off, int64_t nseg, void* out,
                                unsigned char* ws, size_t cnt_bytes, const int64_t* tile_seg,
                                int block, int64_t grid, int64_t tile, int out_f64,
                                cudaStream_t st) {
    const size_t smem = csr_tma_smem_bytes(DOT ? 1 : 0, block);
    auto kern = csr_tma_kernel<T, VAR, DOT, U>;
    // raise the kernel's shared-memory limit to the largest ring once per
    // device (outside any graph capture: the first call is a plain launch)
    static std::atomic<unsigned long long> raised{0ull};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(raised.load() & bit)) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)csr_tma_smem_bytes(DOT ? 1 : 0, 32 * kMaxWarps) > 200 * 1024
                                     ? 200 * 1024
                                     : (int)csr_tma_smem_bytes(DOT ? 1 : 0, 32 * kMaxWarps));
        if (e != cudaSuccess) return e;
        raised.fetch_or(bit);
    }
    return launch_dependent(kern, (unsigned)grid, (unsigned)block, smem, st, x, y, off, nseg, out,
                            ws, cnt_bytes, tile_seg, tile, out_f64);
}

template <typename T, int VAR, bool DOT>
static cudaError_t launch_tma_d(int unroll, const void* x, const void* y, const int64_t* off,
                                int64_t nseg, void* out, unsigned char* ws, size_t cnt_bytes,
                                const int64_t* tile_seg, int block, int64_t grid, int64_t tile,
                                int out_f64, cudaStream_t st) {
    const T* xp = static_cast<const T*>(x);
    const T* yp = static_cast<const T*>(y);
    switch (unroll) {
    case 1: return launch_tma_u<T, VAR, DOT, 1>(xp, yp, off, nseg, out, ws, cnt_bytes, tile_seg, block, grid, tile, out_f64, st);
    case 2: return launch_tma_u<T, VAR, DOT, 2>(xp, yp, off, nseg, out, ws, cnt_bytes, tile_seg, block, grid, tile, out_f64, st);
    case 4: return launch_tma_u<T, VAR, DOT, 4>(xp, yp, off, nseg, out, ws, cnt_bytes, tile_seg, block, grid, tile, out_f64, st);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T, int VAR>
static cudaError_t launch_tma_v(int dot, int unroll, const void* x, const void* y,
                                const int64_t* off, int64_t nseg, void* out, unsigned char* ws,
                                size_t cnt_bytes, const int64_t* tile_seg, int block, int64_t grid,
                                int64_t tile, int out_f64, cudaStream_t st) {
    return dot ? launch_tma_d<T, VAR, true>(unroll, x, y, off, nseg, out, ws, cnt_bytes, tile_seg, block, grid, tile, out_f64, st)
               : launch_tma_d<T, VAR, false>(unroll, x, y, off, nseg, out, ws, cnt_bytes, tile_seg, block, grid, tile, out_f64, st);
}

cudaError_t launch_csr_tma(int dtype, int variant, int dot, int unroll, const void* x,
                           const void* y, const int64_t* off, int64_t nseg, void* out,
                           unsigned char* ws, size_t cnt_bytes, const int64_t* tile_seg,
                           int block, int64_t grid, int64_t tile, int out_f64, cudaStream_t st) {
#define TF_TMA(TY, VA) launch_tma_v<TY, VA>(dot, unroll, x, y, off, nseg, out, ws, cnt_bytes, tile_seg, block, grid, tile, out_f64, st)
#define TF_TMA_DOT(TY, VA) (dot ? launch_tma_d<TY, VA, true>(unroll, x, y, off, nseg, out, ws, cnt_bytes, tile_seg, block, grid, tile, out_f64, st) : cudaErrorInvalidValue)
    if (dtype == 0) {
        switch (variant) {
        case PLAIN: return TF_TMA(float, PLAIN);
        case FAST: return TF_TMA(float, FAST);
        case RIGOROUS: return TF_TMA(float, RIGOROUS);
        case WIDE: return TF_TMA(float, WIDE);
        case KAHAN: return TF_TMA(float, KAHAN);
        case FAST_LIT: return TF_TMA_DOT(float, FAST_LIT);
        case RIG_LIT: return TF_TMA_DOT(float, RIG_LIT);
        }
    } else {
        switch (variant) {
        case PLAIN: return TF_TMA(double, PLAIN);
        case FAST: return TF_TMA(double, FAST);
        case RIGOROUS: return TF_TMA(double, RIGOROUS);
        case WIDE: return TF_TMA(double, WIDE);
        case KAHAN: return TF_TMA(double, KAHAN);
        case FAST_LIT: return TF_TMA_DOT(double, FAST_LIT);
        case RIG_LIT: return TF_TMA_DOT(double, RIG_LIT);
        }
    }
#undef TF_TMA
#undef TF_TMA_DOT
    return cudaErrorInvalidValue;
}

}  // namespace tf
