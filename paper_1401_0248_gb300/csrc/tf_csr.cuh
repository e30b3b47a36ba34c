// tf_csr.cuh -- pieces shared by the two batched kernels: the workspace
// layout and the end of a segment's piece (fold, then write or merge).
#pragma once
#include "tf_device.cuh"
#include "tf_internal.h"

namespace tf {

// workspace: header | per-segment tickets | two piece slots per tile | tile map
inline size_t csr_cnt_bytes(int64_t nseg) {
    return ((size_t)(nseg > 0 ? nseg : 1) * 4 + 255) / 256 * 256;
}
inline size_t csr_max_tiles(int64_t n) { return (size_t)((n + kMinTile - 1) / kMinTile) + 1; }

// The piece [max(a, tlo), min(b, thi)) of segment s = [a, b) in tile t has
// been fed into the warp's C chains per lane: fold the chains (tree), the
// lanes (butterfly), then either write the segment (it lies in this tile) or
// store the piece's pair in slot 2t (2t + 1 for the segment's first piece)
// and take the segment's ticket; the warp completing the k-th piece merges
// the k pairs in tile order (lane l takes pieces l, l + 32, ...).
template <typename T, int VAR, int C>
__device__ __forceinline__ void piece_finish(typename Acc<T, VAR>::type (&cs)[C],
                                             typename Acc<T, VAR>::type (&ce)[C], int64_t s,
                                             int64_t a, int64_t b, int64_t t, int64_t tlo,
                                             int64_t thi, int64_t tile, void* out,
                                             unsigned int* cnt,
                                             typename GridAcc<T, VAR>::type* pieces, int lane,
                                             int out_f64) {
    using A = typename Acc<T, VAR>::type;
    using G = typename GridAcc<T, VAR>::type;
    constexpr bool TW = twofold_v<VAR>;
#pragma unroll
    for (int w = C / 2; w >= 1; w >>= 1)
#pragma unroll
        for (int c = 0; c < w; ++c) merge<TW>(cs[c], ce[c], cs[c + w], ce[c + w]);
    A pv = cs[0], pe = ce[0];
    warp_fold<TW>(pv, pe);

    if (a >= tlo && b <= thi) {
        // the whole segment lies in this tile
        if (lane == 0) write_out<T, VAR, G>(out, s, (G)pv, (G)pe, out_f64 != 0);
        return;
    }
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
    if ((int64_t)old != k - 1) return;
    // last piece of the segment: merge the k pieces in tile order
    __threadfence();
    G gv = G(0), ge = G(0);
    if (lane < k) {
        const int64_t s0 = (lane == 0) ? 2 * w0 + 1 : 2 * (w0 + lane);
        ld_pair_cg(pieces + 2 * s0, gv, ge);
        // the merges form one chain per lane; the loads do not depend on
        // them, so fetch 8 pieces at a time
        constexpr int B = 8;
        int64_t i = lane + 32;
        for (; i + 32 * (B - 1) < k; i += 32 * B) {
            G v2[B], e2[B];
#pragma unroll
            for (int j = 0; j < B; ++j) ld_pair_cg(pieces + 2 * (2 * (w0 + i + 32 * j)), v2[j], e2[j]);
#pragma unroll
            for (int j = 0; j < B; ++j) merge<TW>(gv, ge, v2[j], e2[j]);
        }
        for (; i < k; i += 32) {
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

}  // namespace tf
