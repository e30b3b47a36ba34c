/*
 * twofold.h -- C ABI of libtwofold.so: twofold summation and dot products on
 * one NVIDIA GB300 (sm_103a).
 *
 * Method (E. Latkin, "Twofold fast summation", 2013).  A twofold result is a
 * pair (value, error) of floating-point numbers approximating an exact real
 * as value + error (Overview; the twofold<number> type of Example 1).  The
 * value is the floating-point sum in the library's order; the error collects
 * the rounding errors of those additions:
 *   TF_FAST      Dekker's FAST-TWO-SUM step per item (Theorem 1, Example 1)
 *   TF_RIGOROUS  Knuth's TWO-SUM step per item (Theorem 2, Example 3)
 *   TF_PLAIN     direct summation, error = 0 (Example 3, "sum")
 *   TF_WIDE      a wider accumulator, error = 0 or the accumulator's tail:
 *                binary32 data in binary64 (the listing after Example 3,
 *                "sumd"); binary64 data in IEEE binary128 computed with
 *                integer arithmetic (the paper's __float128 comparison),
 *                output (RN64(S), RN64(S - RN64(S)))
 *   TF_KAHAN     Kahan's compensated summation (Example 2): the pair is the
 *                sum and the compensation not yet applied (-c); dots use
 *                the rounded product, as the paper's dotk
 * Dot products feed the product x[i]*y[i] as the item (the paper's remark at
 * the end of the Algorithms section); the twofold variants also add each
 * product's exact rounding
 * error, from TwoProduct p = RN(x*y), ep = fma(x, y, -p), to the error term.
 * TF_WIDE forms the product exactly in its accumulator format.
 *
 * Reduction order.  Work is split into independent chains that follow the
 * per-item steps above, and chain pairs are merged by TWO-SUM on the values
 * plus one addition of the errors: (v, q) = TWO-SUM(v1, v2), e = (e1 + e2) + q.
 * The order is a fixed function of (n, launch plan, SM count), so results are
 * bit-reproducible run to run for a fixed plan:
 *   single vector: with V = 16 / sizeof(element), thread g of P = grid*block
 *   threads takes the 16-byte vectors j = g + P*m (m = 0, 1, ...) and feeds
 *   element l of vector j to its chain (m mod U)*V + l; a trailing partial
 *   vector is vector n/V.  Each thread folds its chains as a binary tree
 *   (c <- c + w for w = UV/2 ... 1).  Binary64 twofold variants fold each
 *   block's thread pairs by the same tree (t <- t + w for w = block/2 ...
 *   1); the others fold each warp by an xor butterfly (offsets 16 ... 1) and
 *   the block's warp pairs by the butterfly over block/32 lanes.  The last
 *   block to finish folds the block pairs (thread t takes pairs t, t+block,
 *   ... in turn, then its thread pairs fold as a block's do).
 *   batched: the concatenated vector is cut into tiles of plan.tile elements;
 *   in a segment's piece of a tile, element at tile offset r goes to lane
 *   (r/V) mod 32, chain ((r/V)/32 mod U)*V + r mod V; each lane folds its
 *   chains as above and the warp's lanes fold by the xor butterfly (offsets
 *   16 ... 1) for every variant;
 *   a segment spanning k <= 32 tiles merges its k piece pairs as 32 lanes
 *   (lane l holds piece l, +0 pairs after k) and the butterfly; beyond 32 by
 *   a pairwise tree in tile order (the pair of piece j, j a multiple of 2w,
 *   takes the pair of piece j + w for w = 1, 2, 4, ... while j + w < k).
 * For binary32 data the cross-block (and cross-tile) merge of the twofold and
 * wide variants runs in binary64 and the output is v = RN32(V),
 * e = RN32((V - v) + E) from the binary64 pair (V, E); the plain variant stays
 * in binary32 throughout.
 *
 * Conventions for every entry point:
 *   - Pointers named x, y, offsets, out, ws are DEVICE pointers owned by the
 *     caller; the library never allocates on these paths, so the calls can be
 *     captured in a CUDA graph.  Host pointers are named *_host.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *     default stream) unless stated otherwise.
 *   - Argument errors are detected on the host and returned before anything
 *     is enqueued.  Launch failures return TF_ERR_CUDA.
 *   - Element arrays need natural alignment only; 16-byte aligned arrays use
 *     128-bit loads, others take scalar loads in the same order (same bits).
 *   - n = 0 (or an empty segment) gives (+0, +0).  NaN/Inf inputs propagate
 *     (value non-finite, error NaN).
 *   - ws: workspace of at least tf_workspace_size() bytes, zero-filled before
 *     its first use (tf_workspace_reset); every completed call leaves it
 *     ready for the next.  Calls that share a workspace must be ordered on one
 *     stream.
 */
#ifndef TWOFOLD_H
#define TWOFOLD_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* tf_stream_t;   /* same type as cudaStream_t */

typedef enum { TF_F32 = 0, TF_F64 = 1 } tf_dtype;
typedef enum { TF_PLAIN = 0, TF_FAST = 1, TF_RIGOROUS = 2, TF_WIDE = 3, TF_KAHAN = 4 } tf_variant;
typedef enum { TF_OP_SUM = 0, TF_OP_DOT = 1 } tf_op;

typedef enum {
    TF_OK = 0,
    TF_ERR_ARG = 1,          /* null pointer, negative size, bad enum, bad plan   */
    TF_ERR_DTYPE = 2,        /* not a supported element type                      */
    TF_ERR_WORKSPACE = 3,    /* ws smaller than tf_workspace_size()               */
    TF_ERR_ALIGN = 4,        /* pointer not aligned to its element size           */
    TF_ERR_CUDA = 5,         /* a CUDA runtime call failed                        */
    TF_ERR_OFFSETS = 6,      /* device-detected: offsets not a valid CSR          */
    TF_ERR_TIMEOUT = 7,      /* a bounded wait gave up                            */
    TF_ERR_UNSUPPORTED = 8,  /* no sm_103a device, or a size beyond the limits    */
    TF_ERR_UNDRAINED = 9     /* device-detected: a bounded wait gave up and so did
                                the wait for the copies still in flight; the
                                call's results are undefined: drop its outputs
                                and its workspace                              */
} tf_status;

/* flags */
#define TF_OUT_F64 0x1u      /* binary32 data: write the binary64 pair (V, E)     */
#define TF_DOT_LITERAL 0x2u  /* fast / rigorous dots: the paper's form, products
                                rounded and their errors not tracked (dottf/dott) */

/* Launch plan: the reduction order is a function of it (see above). */
typedef struct {
    int32_t block;           /* threads per block: 128, 256 or 512                */
    int32_t unroll;          /* 128-bit loads per thread per step U: 1, 2 or 4;
                                a thread runs U * (16 / sizeof(element)) chains    */
    int32_t blocks_per_sm;   /* grid = blocks_per_sm * SM count (1..8); batched:
                                16-byte-aligned inputs stream through a shared-
                                memory ring when that many blocks' rings fit an
                                SM, else through registers (same bits)         */
    int32_t tile;            /* batched only: elements per warp tile, a multiple
                                of 32 * 16 / sizeof(element) (e.g. 4096); 0 flat  */
} tf_plan;

/* ---- single vectors ---------------------------------------------------- */

/* Twofold sum of x[0..n): out receives {value, error} as two elements of the
   data type, or two doubles when flags & TF_OUT_F64 (binary32 data).
   Example 1 (fast), Example 3 (rigorous, direct), "sumd" listing (wide). */
tf_status tf_sum(const void* x, int64_t n, tf_dtype dtype, tf_variant variant,
                 void* out, void* ws, size_t ws_bytes, uint32_t flags,
                 tf_stream_t stream);

/* Twofold dot product sum x[i]*y[i], i < n (x, y of the same dtype): the
   summation loops with the product as the item, plus TwoProduct. */
tf_status tf_dot(const void* x, const void* y, int64_t n, tf_dtype dtype,
                 tf_variant variant, void* out, void* ws, size_t ws_bytes,
                 uint32_t flags, tf_stream_t stream);

/* ---- ragged batches (CSR) ---------------------------------------------- */

/* One twofold sum per segment s < nseg of x: elements [offsets[s],
   offsets[s+1]).  x holds n elements; offsets (device, int64, nseg + 1
   entries) must satisfy offsets[0] = 0, offsets[s] <= offsets[s+1],
   offsets[nseg] <= n.  out receives nseg pairs (2*nseg elements, or doubles
   with TF_OUT_F64).  Enqueues three kernels: an offsets check, one
   persistent reduction over all segments, and the merge of the pieces of the
   segments over 2..32 tiles.  Invalid offsets are detected on
   the device: every output pair is set to NaN and the workspace error word
   to TF_ERR_OFFSETS (read it with tf_get_device_error). */
tf_status tf_sum_batched(const void* x, int64_t n, const int64_t* offsets, int64_t nseg,
                         tf_dtype dtype, tf_variant variant, void* out, void* ws,
                         size_t ws_bytes, uint32_t flags, tf_stream_t stream);

/* Per-segment twofold dot products of x and y (both n elements). */
tf_status tf_dot_batched(const void* x, const void* y, int64_t n, const int64_t* offsets,
                         int64_t nseg, tf_dtype dtype, tf_variant variant, void* out,
                         void* ws, size_t ws_bytes, uint32_t flags, tf_stream_t stream);

/* ---- host buffers (end to end) ----------------------------------------- */

/* Synchronous convenience for host data: copies x_host (n elements; pinned
   memory for full speed) to the caller's device buffer x_dev, reduces it as
   tf_sum does, copies the pair to out_host and waits for the stream. */
tf_status tf_sum_host(const void* x_host, int64_t n, tf_dtype dtype, tf_variant variant,
                      void* out_host, void* x_dev, void* ws, size_t ws_bytes,
                      uint32_t flags, tf_stream_t stream);
tf_status tf_dot_host(const void* x_host, const void* y_host, int64_t n, tf_dtype dtype,
                      tf_variant variant, void* out_host, void* x_dev, void* y_dev,
                      void* ws, size_t ws_bytes, uint32_t flags, tf_stream_t stream);

/* The same without waiting: the copies of x_host (and y_host) go on
   copy_stream (NULL: on stream), the reduction on stream behind them (an
   event orders it), and the pair is copied to out_host on stream; the call
   returns once all of it is enqueued.  Wait on stream (or an event recorded
   on it) before reading out_host or reusing any of the buffers.  Host
   buffers should be pinned (pageable ones make the copies synchronous).  A
   device buffer must not be refilled while an earlier call that reads it is
   still in flight (give consecutive calls distinct x_dev / y_dev, or order
   them).  Calls sharing ws must share stream. */
tf_status tf_sum_host_async(const void* x_host, int64_t n, tf_dtype dtype, tf_variant variant,
                            void* out_host, void* x_dev, void* ws, size_t ws_bytes,
                            uint32_t flags, tf_stream_t stream, tf_stream_t copy_stream);
tf_status tf_dot_host_async(const void* x_host, const void* y_host, int64_t n, tf_dtype dtype,
                            tf_variant variant, void* out_host, void* x_dev, void* y_dev,
                            void* ws, size_t ws_bytes, uint32_t flags, tf_stream_t stream,
                            tf_stream_t copy_stream);

/* ---- no caller workspace ----------------------------------------------- */

/* tf_sum without a caller workspace, for callers that cannot allocate device
   memory (a host framework that owns all device memory through its own pool,
   a fixed device-memory budget that must not grow after start-up, or a
   latency-critical path that must avoid cudaMalloc's implicit device-wide
   synchronization).  The paper has no counterpart: this is a deployment
   convenience.  Same kernel, launch shape and result bits as tf_sum.
   Scratch: a library-owned device array of 33,024 bytes (a 256-byte header
   and 2048 block pairs of 16 bytes) on every GPU that loads the library,
   kept until the process exits; no call allocates or frees memory.  Every
   launch shape fits it except for binary64 data with TF_WIDE, whose
   binary128 pairs take 32 bytes: there a launch shape of more than 1024
   blocks (a plan of more than 6 blocks per SM on 152 SMs) returns
   TF_ERR_UNSUPPORTED.  The first call on a
   device looks up the array's device address (cudaGetSymbolAddress) with
   that device current; make that first call before any stream capture.
   Every call clears the array's header and shares the array, so calls that
   overlap on the GPU (other streams, other host threads) race: order them
   on one stream. */
tf_status tf_sum_noalloc(const void* x, int64_t n, tf_dtype dtype, tf_variant variant,
                         void* out, uint32_t flags, tf_stream_t stream);

/* ---- one vector over several GPUs (or calls) --------------------------- */

/* The last step of one vector cut into G contiguous shards, each reduced on
   its own GPU (or by its own call) and the G pairs gathered in rank order
   into one device array: merges them in rank order into the result.  The
   paper's loops are sequential; this extends the library's merge of chain
   pairs (TWO-SUM, Theorem 2) across shards.
   pairs: device array of G pairs of doubles (V, E), 8-byte aligned: each
   shard's pair as tf_sum / tf_dot write it for binary64 data, or with
   TF_OUT_F64 for binary32 data (the binary64 cross-block pair before its
   final rounding).  G >= 0 (0 gives (+0, +0)).
   variant: the shards' variant (TF_DOT_LITERAL dots merge as fast /
   rigorous).  Twofold variants (fast, rigorous, kahan): from pair 0,
   (V, q) = TWO-SUM(V, V_g), E = (E + E_g) + q for g = 1 .. G-1, in binary64.
   TF_PLAIN: V + V_g in the data type.  TF_WIDE: binary32 data V + V_g in
   binary64; binary64 data S <- (S + V_g) + E_g in binary128 from S = +0.
   out: one pair in tf_sum's output format for dtype and flags.
   One single-thread kernel on `stream`; argument errors return before it. */
tf_status tf_merge_pairs(const void* pairs, int64_t G, tf_dtype dtype, tf_variant variant,
                         void* out, uint32_t flags, tf_stream_t stream);

/* ---- workspace --------------------------------------------------------- */

/* Bytes of workspace for a call (batched != 0: n elements, nseg segments).
   The size covers every plan the tuner may choose for that shape. */
tf_status tf_workspace_size(tf_op op, int batched, tf_dtype dtype, tf_variant variant,
                            int64_t n, int64_t nseg, size_t* bytes);
/* Zero-fill ws (stream-ordered). */
tf_status tf_workspace_reset(void* ws, size_t ws_bytes, tf_stream_t stream);
/* Read and clear the device error word of ws (0 or a tf_status); waits for
   `stream`. */
tf_status tf_get_device_error(void* ws, size_t ws_bytes, int32_t* code, tf_stream_t stream);

/* ---- plans and tuning -------------------------------------------------- */

/* Plans are kept per key (op, class, dtype, variant); the class is
   TF_PLAN_FLAT for single vectors of more than TF_SMALL_N elements,
   TF_PLAN_BATCHED for the batched calls and TF_PLAN_FLAT_SMALL for single
   vectors of at most TF_SMALL_N elements, whose time is set by the latency of
   the folds rather than by memory (they want fewer, wider-spread threads).
   The `batched` argument below takes the class. */
#define TF_PLAN_FLAT 0
#define TF_PLAN_BATCHED 1
#define TF_PLAN_FLAT_SMALL 2
#define TF_SMALL_N (1 << 22)
tf_status tf_plan_get(tf_op op, int batched, tf_dtype dtype, tf_variant variant, tf_plan* plan);
tf_status tf_plan_set(tf_op op, int batched, tf_dtype dtype, tf_variant variant,
                      const tf_plan* plan);
/* The launch shape a call of size n (or total elements n) would use
   (batched: 0 single vector, the class then follows from n; 1 batched). */
tf_status tf_launch_shape(tf_op op, int batched, tf_dtype dtype, tf_variant variant,
                          int64_t n, int32_t* block, int32_t* unroll, int64_t* grid,
                          int64_t* tile);
/* Time every candidate plan on the given problem (device data as for the
   calls above, y/offsets NULL where unused), `reps` timed launches each after
   two warm-up launches, keep the fastest as the plan for its key (single
   vectors: the class of n) and return it.  Synchronous; not capturable. */
tf_status tf_tune(tf_op op, int batched, tf_dtype dtype, tf_variant variant,
                  const void* x, const void* y, int64_t n, const int64_t* offsets,
                  int64_t nseg, void* out, void* ws, size_t ws_bytes, int reps,
                  tf_stream_t stream, tf_plan* best);
/* Plans as text, one line per key: "op class dtype variant block unroll
   blocks_per_sm tile".  Save writes a temporary file and renames it; load
   accepts any subset of the keys. */
tf_status tf_plan_save(const char* path);
tf_status tf_plan_load(const char* path);

/* ---- error signalling -------------------------------------------------- */

/* The paper's intended use of the error term: signal when it grows too large
   for the working precision (the paragraph after Example 2).  Counts the
   pairs (value, error) of `pairs` (npairs pairs of binary32 or binary64, as
   tf_sum / tf_*_batched write them) with |error| > tau * |value|, or with a
   non-finite member, into the device int32 *count (overwritten).  Two
   stream-ordered operations (a 4-byte clear and one kernel); the count stays
   on the device for later device work or an asynchronous copy. */
tf_status tf_count_large_errors(const void* pairs, int64_t npairs, tf_dtype pair_dtype,
                                double tau, int32_t* count, tf_stream_t stream);

/* ---- building blocks and probes ---------------------------------------- */

/* Elementwise error-free transforms on device arrays of n elements:
   prim 0 FAST-TWO-SUM(a, b) (Theorem 1), 1 TWO-SUM(a, b) (Theorem 2),
   2 TwoProduct (p = RN(ab), e = fma(a, b, -p)); the binary64 forms the
   reductions use, with the error (and for 4 the product) computed on the
   integer pipe from the significands: 3 TWO-SUM, 4 TwoProduct, 5 FAST-TWO-SUM.
   3-5 give the bits of 1, 2, 0 (binary32 data use 1, 2, 0).  Outputs to x, y. */
tf_status tf_prim(int prim, tf_dtype dtype, const void* a, const void* b, void* x, void* y,
                  int64_t n, tf_stream_t stream);

/* Memory-read probe (the paper's read1/read2): streams nbytes of x (and of y
   when not NULL; nbytes a multiple of 16, both 16-byte aligned) with the
   reductions' 128-bit streaming loads and no arithmetic, `unroll` loads of
   each array in flight per thread (1, 2, 4 or 8), and writes one word per
   block to sink (blocks words). */
tf_status tf_probe_read(const void* x, const void* y, int64_t nbytes, void* sink,
                        int32_t blocks, int32_t threads, int32_t unroll, tf_stream_t stream);

/* Arithmetic probe (the paper's p-functions): each thread runs `iters`
   iterations of 8 independent chains of one operation, from registers.
   kind: 0 FADD, 1 DADD, 2 FFMA, 3 DFMA, 4 IADD (32-bit), 5 fast step binary32,
   6 rigorous step binary32, 7 fast step binary64, 8 rigorous step binary64,
   9 DMUL, 10 binary64 add issued as fma(a, one, b) with `one` = 1.0 computed
   at run time (how the binary64 sums issue their adds).
   sink receives one word per thread (blocks * threads words). */
tf_status tf_probe_alu(int kind, int64_t iters, void* sink, int32_t blocks, int32_t threads,
                       tf_stream_t stream);

/* The bounded wait of the batched kernel's shared-memory ring (an mbarrier
   phase polled at most `polls` times, 1 <= polls <= 2^22), run by one thread
   on a barrier that nothing completes (arrive = 0) or that the thread
   completes first (arrive = 1).  Writes *flag (device int32) = 1 if the wait
   gave up, else 0.  This is how the kernels' waits end without a result: the
   batched kernel then sets TF_ERR_TIMEOUT in the workspace error word
   (tf_get_device_error) and returns.  Argument errors come back before any
   launch. */
tf_status tf_probe_wait(int32_t arrive, int64_t polls, int32_t* flag, tf_stream_t stream);

/* ---- misc -------------------------------------------------------------- */
const char* tf_status_string(tf_status s);
/* SM count of the current device (0 if none). */
int32_t tf_device_sm_count(void);

#ifdef __cplusplus
}
#endif
#endif
