// tf_csr.cuh -- pieces shared by the two batched kernels and the merge
// kernel after them: the workspace layout, the end of a segment's piece
// (fold, then write, store or merge) and the merge of up to 32 pieces.
#pragma once
#include "tf_device.cuh"
#include "tf_internal.h"

namespace tf {

// workspace: header | one word per piece slot (the arrival counters of the
// trees over more than 32 pieces in even slots; in odd slot 2*t + 1, the
// number of tiles of a segment over 2..32 tiles that starts in tile t) | two
// piece slots per tile | tile map.  Sized for the smallest tile (kMinTile).
inline size_t csr_max_tiles(int64_t n) { return (size_t)((n + kMinTile - 1) / kMinTile) + 1; }
inline size_t csr_cnt_bytes(int64_t n) { return (csr_max_tiles(n) * 2 * 4 + 255) / 256 * 256; }

// The lane that publishes a piece's pair (store, then the arrival atomic):
// not lane 0, which in the staged kernel issues the warp's bulk copies.
constexpr int kPubLane = 31;

// The arrival count of a piece: one atomic add with acquire-release
// semantics at GPU scope, issued by the lane that stored the piece's pair.
// Its release orders that store before the count; when the count shows the
// warp is the last to arrive, its acquire, passed on to the warp's other
// lanes by __syncwarp, orders their loads of the other pieces after every
// count that came before.  One such atomic replaced a fence before the add
// and a fence after it (measured about 1.7 and 1.4 us per piece).
__device__ __forceinline__ unsigned int arrive_acq_rel(unsigned int* ctr) {
    unsigned int old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;"
                 : "=r"(old) : "l"(ctr) : "memory");
    return old;
}

// The three kernels of a batched call follow one another by programmatic
// dependent launch: a kernel's blocks may be scheduled once every block of
// the one before has started (grid_dependents_go), and they wait in hardware
// for that grid to complete, its memory operations visible, before touching
// what it writes (grid_wait).  The gap between the kernels then holds no
// launch latency.  Without the launch attribute both are no-ops.
__device__ __forceinline__ void grid_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dependents_go() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// launch `kern` on `st`, allowed to start before the previous kernel on `st`
// has completed (see grid_wait)
template <typename... P, typename... Args>
inline cudaError_t launch_dependent(void (*kern)(P...), unsigned grid, unsigned block,
                                    size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// piece i of a segment whose first tile is w0: slot 2*w0 + 1 for i = 0 (the
// piece that starts the segment), 2*(w0 + i) after it
__device__ __forceinline__ int64_t piece_slot(int64_t w0, int64_t i) {
    return i == 0 ? 2 * w0 + 1 : 2 * (w0 + i);
}

// The pairwise tree of a segment's k > 32 pieces (see piece_finish), from
// the piece at index st whose pair (gv, ge) the warp holds.  Out of line: the
// streaming loops that call piece_finish keep their registers.
template <typename T, int VAR>
static __device__ __noinline__ void piece_tree(typename GridAcc<T, VAR>::type gv,
                                               typename GridAcc<T, VAR>::type ge, int64_t st,
                                               int64_t w0, int64_t k, int64_t s,
                                               unsigned int* cnt,
                                               typename GridAcc<T, VAR>::type* pieces,
                                               int lane, void* out, int out_f64) {
    using G = typename GridAcc<T, VAR>::type;
    constexpr bool TW = twofold_v<VAR>;
    int64_t w = 1;
    for (;;) {
        if (st == 0 && w >= k) {                // the root: the whole segment
            if (lane == 0) write_out<T, VAR, G>(out, s, gv, ge, out_f64 != 0);
            return;
        }
        const bool left = ((st / w) & 1) == 0;
        if (left && st + w >= k) {              // no right sibling: the parent is this node
            w *= 2;
            continue;
        }
        const int64_t sib = left ? st + w : st - w;
        unsigned int* ctr = &cnt[piece_slot(w0, left ? sib : st)];   // keyed by the right child
        unsigned int old = 0;
        if (lane == kPubLane) {
            G* mine = pieces + 2 * piece_slot(w0, st);
            mine[0] = gv;
            mine[1] = ge;
            old = arrive_acq_rel(ctr);
        }
        old = __shfl_sync(FULL, old, kPubLane);
        if (old == 0u) return;                  // the sibling's warp completes the parent
        __syncwarp();
        G v2, e2;
        ld_pair_cg(pieces + 2 * piece_slot(w0, sib), v2, e2);
        if (left) {
            merge<TW>(gv, ge, v2, e2);
        } else {
            merge<TW>(v2, e2, gv, ge);
            gv = v2;
            ge = e2;
            st = sib;
        }
        if (lane == 0) *ctr = 0u;               // ready for the next call
        w *= 2;
    }
}

// The piece [max(a, tlo), min(b, thi)) of segment s = [a, b) in tile t has
// been fed into the warp's C chains per lane: fold the chains (tree), the
// lanes (butterfly), then write the segment (it lies in this tile), store the
// piece's pair in its slot (a segment over 2..32 tiles: csr_merge, launched
// after this kernel, merges its pieces), or take part in the pairwise tree of
// the k > 32 pieces: the node over pieces [j, j + 2w) being merge(node [j, j
// + w), node [j + w, j + 2w)), or the left node alone when j + w >= k; each
// merge is done by whichever warp completes the second of the two children
// (an arrival counter per node, no waiting), so no warp does more than
// log2(k) merges.  The bits do not depend on which warp does them.
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
    const int64_t w0 = a / tile, k = (b - 1) / tile - w0 + 1;
    G gv = (G)pv, ge = (G)pe;                   // the node [st, st + w) in registers
    if (k <= 32) {
        // plain stores, which csr_merge's wait for this grid to complete
        // orders before its loads; the warp of the first piece records k in
        // the word of slot 2*w0 + 1 (the tree below counts arrivals in even
        // slots only)
        if (lane == kPubLane) {
            G* mine = pieces + 2 * piece_slot(w0, t - w0);
            mine[0] = gv;
            mine[1] = ge;
            if (t == w0) cnt[2 * w0 + 1] = (unsigned int)k;
        }
        return;
    }
    piece_tree<T, VAR>(gv, ge, t - w0, w0, k, s, cnt, pieces, lane, out, out_f64);
}

// The merge of a segment's k <= 32 pieces in the order of the xor butterfly
// over K2 lanes (K2 the power of two >= k, lanes k.. holding +0 pairs),
// lane 0's result: with R(j, K2) = piece j, R(j, o) = merge(R(j, 2o),
// R(j + o, 2o)) for j < o, the result is R(0, 1).  A right operand whose
// pieces all lie at k or after is a +0 pair, which leaves the left pair's
// bits as they are (a piece pair is never -0): that merge is skipped.
template <int O, int K2, bool TW, typename G>
__device__ __forceinline__ void butterfly_node(const G* __restrict__ pieces, int64_t w0, int k,
                                               int j, G& v, G& e) {
    if constexpr (O == K2) {
        const G* p = pieces + 2 * piece_slot(w0, j);
        v = p[0];
        e = p[1];
    } else {
        butterfly_node<2 * O, K2, TW>(pieces, w0, k, j, v, e);
        if (j + O < k) {
            G v2, e2;
            butterfly_node<2 * O, K2, TW>(pieces, w0, k, j + O, v2, e2);
            merge<TW>(v, e, v2, e2);
        }
    }
}

}  // namespace tf
