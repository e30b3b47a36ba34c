// tf_api.cu -- the C ABI of libtwofold.so (declared in include/twofold.h):
// argument checks, launch plans, the plan tuner, workspace helpers and the
// host-buffer calls.  All compute happens in the kernels of tf_flat.cu,
// tf_csr.cu and tf_aux.cu.
#include "twofold.h"
#include "tf_internal.h"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

namespace {

using tf::kHeaderBytes;

constexpr size_t kStageOffset = 16;     // WsHeader::stage

std::mutex g_mu;

struct DevInfo { int sms = 0; int smem_sm = 0; int ok = -1; };
DevInfo g_dev[64];

constexpr int kVariants = 5;          // plain, fast, rigorous, wide, kahan
constexpr int kClasses = 3;           // TF_PLAN_FLAT, TF_PLAN_BATCHED, TF_PLAN_FLAT_SMALL

// plans indexed [op][class][dtype][variant]
tf_plan g_plan[2][kClasses][2][kVariants];
bool g_plan_init = false;

void init_plans_locked() {
    if (g_plan_init) return;
    for (int op = 0; op < 2; ++op)
        for (int c = 0; c < kClasses; ++c)
            for (int dt = 0; dt < 2; ++dt)
                for (int v = 0; v < kVariants; ++v) {
                    tf_plan p;
                    p.block = 512;
                    p.unroll = 2;
                    p.blocks_per_sm = 2;
                    p.tile = 0;
                    if (c == TF_PLAN_BATCHED) {
                        p.block = 256;
                        p.blocks_per_sm = 4;
                        p.tile = dt == 0 ? 4096 : 2048;
                    } else if (c == TF_PLAN_FLAT_SMALL) {
                        p.block = 256;
                        p.unroll = 1;
                    }
                    g_plan[op][c][dt][v] = p;
                }
    g_plan_init = true;
}

// the plan class of a single-vector call of n elements
int flat_class(int64_t n) { return n <= (int64_t)TF_SMALL_N ? TF_PLAN_FLAT_SMALL : TF_PLAN_FLAT; }

tf_status check_device(int* sms, int* smem_sm = nullptr) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return TF_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    DevInfo& d = g_dev[dev];
    if (d.ok < 0) {
        int major = 0, minor = 0, sm = 0, smem = 0;
        if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
                cudaSuccess) {
            cudaGetLastError();
            return TF_ERR_UNSUPPORTED;
        }
        d.sms = sm;
        d.smem_sm = smem;
        d.ok = (major == 10 && minor == 3) ? 1 : 0;
    }
    if (!d.ok) return TF_ERR_UNSUPPORTED;
    *sms = d.sms;
    if (smem_sm) *smem_sm = d.smem_sm;
    return TF_OK;
}

// The batched kernel stages its input through shared memory only when the
// plan's blocks_per_sm blocks, each with its ring (and the 1 KiB the runtime
// keeps per block, plus the kernel's barriers), fit in one SM's shared
// memory; a plan asking for more resident blocks than the rings allow runs
// the register-loading kernel at that residency (same bits).
bool csr_ring_fits(const tf_plan& p, int op, int smem_sm) {
    const size_t per_block = tf::csr_tma_smem_bytes(op, p.block) + 2048;
    return (size_t)p.blocks_per_sm * per_block <= (size_t)smem_sm;
}

bool plan_valid(const tf_plan& p, int cls, int dtype) {
    const bool batched = cls == TF_PLAN_BATCHED;
    if (p.block != 128 && p.block != 256 && p.block != 512) return false;
    if (p.unroll != 1 && p.unroll != 2 && p.unroll != 4) return false;
    if (p.blocks_per_sm < 1 || p.blocks_per_sm > 8) return false;
    if (p.block * p.blocks_per_sm > 2048) return false;
    if (batched) {
        const int V = dtype == 0 ? 4 : 2;
        if (p.tile < tf::kMinTile || p.tile % (32 * V) != 0 || p.tile > (1 << 22)) return false;
    }
    return true;
}

tf_plan get_plan(int op, int batched, int dtype, int variant) {
    std::lock_guard<std::mutex> lk(g_mu);
    init_plans_locked();
    return g_plan[op][batched][dtype][variant];
}

int64_t flat_grid(const tf_plan& p, int64_t n, int dtype, int sms) {
    const int V = dtype == 0 ? 4 : 2;
    const int64_t nv = (n + V - 1) / V;
    const int64_t per_block = (int64_t)p.block * p.unroll;
    int64_t g = std::min<int64_t>((int64_t)p.blocks_per_sm * sms, (nv + per_block - 1) / per_block);
    g = std::max<int64_t>(g, 1);
    return std::min<int64_t>(g, tf::kMaxFlatGrid);
}

int64_t csr_grid(const tf_plan& p, int sms) {
    return std::min<int64_t>((int64_t)p.blocks_per_sm * sms, tf::kMaxFlatGrid);
}

size_t flat_ws_bytes() { return kHeaderBytes + tf::kPairBytes * (size_t)tf::kMaxFlatGrid; }

size_t esize(int dtype) { return dtype == 0 ? 4 : 8; }

// One NVTX range per API call (a no-op unless a profiler is attached), so
// that timelines show the library's calls around its kernels.
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

// the kernels' variant: the literal dot forms are variants 5 and 6 there
int kernel_variant(int op, int variant, uint32_t flags) {
    if (op == 1 && (flags & TF_DOT_LITERAL) && (variant == TF_FAST || variant == TF_RIGOROUS))
        return variant == TF_FAST ? 5 : 6;
    return variant;
}

tf_status common_checks(int op, int dtype, int variant, const void* x, const void* y,
                        int64_t n, void* out, void* ws, size_t ws_bytes) {
    if (op < 0 || op > 1 || variant < 0 || variant >= kVariants) return TF_ERR_ARG;
    if (dtype != TF_F32 && dtype != TF_F64) return TF_ERR_DTYPE;
    if (n < 0 || !out || !ws) return TF_ERR_ARG;
    if (n > 0 && (!x || (op == 1 && !y))) return TF_ERR_ARG;
    const uintptr_t es = esize(dtype);
    if (((uintptr_t)x % es) || (op == 1 && ((uintptr_t)y % es)) || ((uintptr_t)out % es))
        return TF_ERR_ALIGN;
    if ((uintptr_t)ws % 256) return TF_ERR_ALIGN;
    (void)ws_bytes;
    return TF_OK;
}

tf_status run_flat(int op, const void* x, const void* y, int64_t n, int dtype, int variant,
                   void* out, void* ws, size_t ws_bytes, uint32_t flags, cudaStream_t st,
                   const tf_plan* force = nullptr) {
    tf_status s = common_checks(op, dtype, variant, x, y, n, out, ws, ws_bytes);
    if (s != TF_OK) return s;
    if ((flags & TF_OUT_F64) && ((uintptr_t)out % 8)) return TF_ERR_ALIGN;
    if (ws_bytes < flat_ws_bytes()) return TF_ERR_WORKSPACE;
    int sms = 0;
    if ((s = check_device(&sms)) != TF_OK) return s;
    const tf_plan p = force ? *force : get_plan(op, flat_class(n), dtype, variant);
    const int64_t grid = flat_grid(p, n, dtype, sms);
    const int aligned = ((uintptr_t)x % 16 == 0) && (op == 0 || (uintptr_t)y % 16 == 0);
    cudaError_t e = tf::launch_flat(dtype, kernel_variant(op, variant, flags), op, p.unroll, x, y,
                                    n, out, ws, p.block, grid, aligned,
                                    (flags & TF_OUT_F64) ? 1 : 0, st);
    return e == cudaSuccess ? TF_OK : TF_ERR_CUDA;
}

tf_status run_csr(int op, const void* x, const void* y, int64_t n, const int64_t* off,
                  int64_t nseg, int dtype, int variant, void* out, void* ws, size_t ws_bytes,
                  uint32_t flags, cudaStream_t st, const tf_plan* force = nullptr) {
    if (nseg < 0 || !off) return TF_ERR_ARG;
    // no segments: nothing to write (out may be empty), arguments still checked
    static char dummy[16] __attribute__((aligned(16)));
    tf_status s = common_checks(op, dtype, variant, x, y, n, (nseg == 0 && !out) ? dummy : out,
                                ws, ws_bytes);
    if (s != TF_OK) return s;
    if ((uintptr_t)off % 8) return TF_ERR_ALIGN;
    if ((flags & TF_OUT_F64) && ((uintptr_t)out % 8)) return TF_ERR_ALIGN;
    if (ws_bytes < tf::csr_ws_bytes(n, nseg)) return TF_ERR_WORKSPACE;
    if (nseg == 0) return TF_OK;
    if (nseg > (int64_t)1 << 40) return TF_ERR_UNSUPPORTED;
    int sms = 0, smem_sm = 0;
    if ((s = check_device(&sms, &smem_sm)) != TF_OK) return s;
    const tf_plan p = force ? *force : get_plan(op, 1, dtype, variant);
    const int64_t grid = csr_grid(p, sms);
    const int aligned = ((uintptr_t)x % 16 == 0) && (op == 0 || (uintptr_t)y % 16 == 0);
    const int staged = aligned && csr_ring_fits(p, op, smem_sm);
    cudaError_t e = tf::launch_csr(dtype, kernel_variant(op, variant, flags), op, p.unroll, x, y,
                                   n, off, nseg, out, ws, ws_bytes, p.block, grid, p.tile,
                                   aligned, staged, (flags & TF_OUT_F64) ? 1 : 0, st);
    return e == cudaSuccess ? TF_OK : TF_ERR_CUDA;
}

}  // namespace

extern "C" {

const char* tf_status_string(tf_status s) {
    switch (s) {
    case TF_OK: return "ok";
    case TF_ERR_ARG: return "invalid argument";
    case TF_ERR_DTYPE: return "variant not defined for this dtype";
    case TF_ERR_WORKSPACE: return "workspace too small";
    case TF_ERR_ALIGN: return "misaligned pointer";
    case TF_ERR_CUDA: return "CUDA runtime error";
    case TF_ERR_OFFSETS: return "invalid CSR offsets";
    case TF_ERR_TIMEOUT: return "bounded wait timed out";
    case TF_ERR_UNSUPPORTED: return "unsupported device or size";
    case TF_ERR_UNDRAINED: return "bounded wait timed out with copies still in flight";
    }
    return "unknown status";
}

int32_t tf_device_sm_count(void) {
    int sms = 0;
    return check_device(&sms) == TF_OK ? sms : 0;
}

tf_status tf_sum(const void* x, int64_t n, tf_dtype dtype, tf_variant variant, void* out,
                 void* ws, size_t ws_bytes, uint32_t flags, tf_stream_t stream) {
    Range r("tf_sum");
    return run_flat(0, x, nullptr, n, dtype, variant, out, ws, ws_bytes, flags,
                    (cudaStream_t)stream);
}

tf_status tf_dot(const void* x, const void* y, int64_t n, tf_dtype dtype, tf_variant variant,
                 void* out, void* ws, size_t ws_bytes, uint32_t flags, tf_stream_t stream) {
    Range r("tf_dot");
    return run_flat(1, x, y, n, dtype, variant, out, ws, ws_bytes, flags, (cudaStream_t)stream);
}

tf_status tf_sum_batched(const void* x, int64_t n, const int64_t* offsets, int64_t nseg,
                         tf_dtype dtype, tf_variant variant, void* out, void* ws,
                         size_t ws_bytes, uint32_t flags, tf_stream_t stream) {
    Range r("tf_sum_batched");
    return run_csr(0, x, nullptr, n, offsets, nseg, dtype, variant, out, ws, ws_bytes, flags,
                   (cudaStream_t)stream);
}

tf_status tf_dot_batched(const void* x, const void* y, int64_t n, const int64_t* offsets,
                         int64_t nseg, tf_dtype dtype, tf_variant variant, void* out,
                         void* ws, size_t ws_bytes, uint32_t flags, tf_stream_t stream) {
    Range r("tf_dot_batched");
    return run_csr(1, x, y, n, offsets, nseg, dtype, variant, out, ws, ws_bytes, flags,
                   (cudaStream_t)stream);
}

static tf_status host_call(int op, const void* xh, const void* yh, int64_t n, int dtype,
                           int variant, void* out_host, void* xd, void* yd, void* ws,
                           size_t ws_bytes, uint32_t flags, cudaStream_t st) {
    if (!out_host || (n > 0 && (!xh || !xd || (op == 1 && (!yh || !yd))))) return TF_ERR_ARG;
    if (n < 0) return TF_ERR_ARG;
    if (!ws) return TF_ERR_ARG;
    void* stage = (char*)ws + kStageOffset;
    // every argument and the device checked before anything is enqueued
    tf_status s = common_checks(op, dtype, variant, xd, yd, n, stage, ws, ws_bytes);
    if (s != TF_OK) return s;
    if ((flags & TF_OUT_F64) && ((uintptr_t)stage % 8)) return TF_ERR_ALIGN;
    if (ws_bytes < flat_ws_bytes()) return TF_ERR_WORKSPACE;
    int sms = 0;
    if ((s = check_device(&sms)) != TF_OK) return s;
    const size_t bytes = (size_t)n * esize(dtype);
    if (n > 0) {
        if (cudaMemcpyAsync(xd, xh, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return TF_ERR_CUDA;
        if (op == 1 && cudaMemcpyAsync(yd, yh, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return TF_ERR_CUDA;
    }
    s = run_flat(op, xd, yd, n, dtype, variant, stage, ws, ws_bytes, flags, st);
    if (s != TF_OK) return s;
    const size_t ob = (dtype == TF_F64 || (flags & TF_OUT_F64)) ? 16 : 8;
    if (cudaMemcpyAsync(out_host, stage, ob, cudaMemcpyDeviceToHost, st) != cudaSuccess) return TF_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return TF_ERR_CUDA;
    return TF_OK;
}

tf_status tf_sum_host(const void* x_host, int64_t n, tf_dtype dtype, tf_variant variant,
                      void* out_host, void* x_dev, void* ws, size_t ws_bytes, uint32_t flags,
                      tf_stream_t stream) {
    Range r("tf_sum_host");
    return host_call(0, x_host, nullptr, n, dtype, variant, out_host, x_dev, nullptr, ws,
                     ws_bytes, flags, (cudaStream_t)stream);
}

tf_status tf_dot_host(const void* x_host, const void* y_host, int64_t n, tf_dtype dtype,
                      tf_variant variant, void* out_host, void* x_dev, void* y_dev, void* ws,
                      size_t ws_bytes, uint32_t flags, tf_stream_t stream) {
    Range r("tf_dot_host");
    return host_call(1, x_host, y_host, n, dtype, variant, out_host, x_dev, y_dev, ws, ws_bytes,
                     flags, (cudaStream_t)stream);
}

// The asynchronous form: copies on `cs` (or on `st` when cs is NULL or st),
// the reduction on `st` ordered behind them by an event, the pair copied back
// on `st`; nothing waits.
static tf_status host_call_async(int op, const void* xh, const void* yh, int64_t n, int dtype,
                                 int variant, void* out_host, void* xd, void* yd, void* ws,
                                 size_t ws_bytes, uint32_t flags, cudaStream_t st,
                                 cudaStream_t cs) {
    if (!out_host || (n > 0 && (!xh || !xd || (op == 1 && (!yh || !yd))))) return TF_ERR_ARG;
    if (n < 0) return TF_ERR_ARG;
    if (!ws) return TF_ERR_ARG;
    void* stage = (char*)ws + kStageOffset;
    tf_status s = common_checks(op, dtype, variant, xd, yd, n, stage, ws, ws_bytes);
    if (s != TF_OK) return s;
    if (ws_bytes < flat_ws_bytes()) return TF_ERR_WORKSPACE;
    int sms = 0;
    if ((s = check_device(&sms)) != TF_OK) return s;
    const bool two = cs != nullptr && cs != st;
    const size_t bytes = (size_t)n * esize(dtype);
    cudaStream_t c = two ? cs : st;
    if (n > 0) {
        if (cudaMemcpyAsync(xd, xh, bytes, cudaMemcpyHostToDevice, c) != cudaSuccess) return TF_ERR_CUDA;
        if (op == 1 && cudaMemcpyAsync(yd, yh, bytes, cudaMemcpyHostToDevice, c) != cudaSuccess)
            return TF_ERR_CUDA;
    }
    if (two) {
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return TF_ERR_CUDA;
        const bool ok = cudaEventRecord(ev, cs) == cudaSuccess &&
                        cudaStreamWaitEvent(st, ev, 0) == cudaSuccess;
        cudaEventDestroy(ev);              // released once the wait is satisfied
        if (!ok) return TF_ERR_CUDA;
    }
    s = run_flat(op, xd, yd, n, dtype, variant, stage, ws, ws_bytes, flags, st);
    if (s != TF_OK) return s;
    const size_t ob = (dtype == TF_F64 || (flags & TF_OUT_F64)) ? 16 : 8;
    if (cudaMemcpyAsync(out_host, stage, ob, cudaMemcpyDeviceToHost, st) != cudaSuccess) return TF_ERR_CUDA;
    return TF_OK;
}

tf_status tf_sum_host_async(const void* x_host, int64_t n, tf_dtype dtype, tf_variant variant,
                            void* out_host, void* x_dev, void* ws, size_t ws_bytes,
                            uint32_t flags, tf_stream_t stream, tf_stream_t copy_stream) {
    Range r("tf_sum_host_async");
    return host_call_async(0, x_host, nullptr, n, dtype, variant, out_host, x_dev, nullptr, ws,
                           ws_bytes, flags, (cudaStream_t)stream, (cudaStream_t)copy_stream);
}

tf_status tf_dot_host_async(const void* x_host, const void* y_host, int64_t n, tf_dtype dtype,
                            tf_variant variant, void* out_host, void* x_dev, void* y_dev,
                            void* ws, size_t ws_bytes, uint32_t flags, tf_stream_t stream,
                            tf_stream_t copy_stream) {
    Range r("tf_dot_host_async");
    return host_call_async(1, x_host, y_host, n, dtype, variant, out_host, x_dev, y_dev, ws,
                           ws_bytes, flags, (cudaStream_t)stream, (cudaStream_t)copy_stream);
}

tf_status tf_workspace_size(tf_op op, int batched, tf_dtype dtype, tf_variant variant,
                            int64_t n, int64_t nseg, size_t* bytes) {
    if (!bytes || n < 0 || nseg < 0 || op < 0 || op > 1 || variant < 0 || variant >= kVariants)
        return TF_ERR_ARG;
    if (dtype != TF_F32 && dtype != TF_F64) return TF_ERR_DTYPE;
    *bytes = batched ? std::max(tf::csr_ws_bytes(n, nseg), flat_ws_bytes()) : flat_ws_bytes();
    return TF_OK;
}

tf_status tf_workspace_reset(void* ws, size_t ws_bytes, tf_stream_t stream) {
    if (!ws) return TF_ERR_ARG;
    return cudaMemsetAsync(ws, 0, ws_bytes, (cudaStream_t)stream) == cudaSuccess ? TF_OK
                                                                                : TF_ERR_CUDA;
}

tf_status tf_get_device_error(void* ws, size_t ws_bytes, int32_t* code, tf_stream_t stream) {
    if (!ws || !code || ws_bytes < kHeaderBytes) return TF_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int32_t* dev_err = (int32_t*)((char*)ws + 4);
    if (cudaMemcpyAsync(code, dev_err, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) return TF_ERR_CUDA;
    if (cudaMemsetAsync(dev_err, 0, 4, st) != cudaSuccess) return TF_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return TF_ERR_CUDA;
    return TF_OK;
}

tf_status tf_plan_get(tf_op op, int batched, tf_dtype dtype, tf_variant variant, tf_plan* plan) {
    if (!plan || op < 0 || op > 1 || variant < 0 || variant >= kVariants || (dtype != 0 && dtype != 1) ||
        batched < 0 || batched >= kClasses)
        return TF_ERR_ARG;
    *plan = get_plan(op, batched, dtype, variant);
    return TF_OK;
}

tf_status tf_plan_set(tf_op op, int batched, tf_dtype dtype, tf_variant variant,
                      const tf_plan* plan) {
    if (!plan || op < 0 || op > 1 || variant < 0 || variant >= kVariants || (dtype != 0 && dtype != 1) ||
        batched < 0 || batched >= kClasses)
        return TF_ERR_ARG;
    tf_plan p = *plan;
    if (batched != TF_PLAN_BATCHED) p.tile = 0;
    if (!plan_valid(p, batched, dtype)) return TF_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    init_plans_locked();
    g_plan[op][batched][dtype][variant] = p;
    return TF_OK;
}

tf_status tf_launch_shape(tf_op op, int batched, tf_dtype dtype, tf_variant variant, int64_t n,
                          int32_t* block, int32_t* unroll, int64_t* grid, int64_t* tile) {
    if (op < 0 || op > 1 || variant < 0 || variant >= kVariants || (dtype != 0 && dtype != 1) || n < 0)
        return TF_ERR_ARG;
    int sms = 0;
    tf_status s = check_device(&sms);
    if (s != TF_OK) return s;
    const tf_plan p = get_plan(op, batched ? TF_PLAN_BATCHED : flat_class(n), dtype, variant);
    if (block) *block = p.block;
    if (unroll) *unroll = p.unroll;
    if (grid) *grid = batched ? csr_grid(p, sms) : flat_grid(p, n, dtype, sms);
    if (tile) *tile = batched ? p.tile : 0;
    return TF_OK;
}

tf_status tf_tune(tf_op op, int batched, tf_dtype dtype, tf_variant variant, const void* x,
                  const void* y, int64_t n, const int64_t* offsets, int64_t nseg, void* out,
                  void* ws, size_t ws_bytes, int reps, tf_stream_t stream, tf_plan* best) {
    if (reps < 1 || reps > 1000 || op < 0 || op > 1) return TF_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<tf_plan> cands;
    const int V = dtype == 0 ? 4 : 2;
    for (int block : {128, 256, 512})
        for (int unroll : {1, 2, 4})
            for (int bps : {1, 2, 3, 4, 5, 6, 8}) {
                if (block * bps > 2048) continue;
                if (!batched) {
                    cands.push_back({block, unroll, bps, 0});
                } else {
                    for (int tile : {1024, 2048, 4096, 8192, 16384})
                        if (tile % (32 * V) == 0) cands.push_back({block, unroll, bps, tile});
                }
            }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return TF_ERR_CUDA;
    float best_ms = 1e30f;
    const int cls = batched ? TF_PLAN_BATCHED : flat_class(n);
    tf_plan bp = get_plan(op, cls, dtype, variant);
    tf_status rs = TF_OK;
    for (const tf_plan& p : cands) {
        auto run = [&]() {
            return batched ? run_csr(op, x, y, n, offsets, nseg, dtype, variant, out, ws, ws_bytes, 0, st, &p)
                           : run_flat(op, x, y, n, dtype, variant, out, ws, ws_bytes, 0, st, &p);
        };
        tf_status s = run();
        if (s == TF_OK) s = run();
        if (s != TF_OK) { rs = s; break; }
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps && s == TF_OK; ++r) s = run();
        cudaEventRecord(e1, st);
        if (s != TF_OK || cudaEventSynchronize(e1) != cudaSuccess) { rs = s != TF_OK ? s : TF_ERR_CUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) { best_ms = ms; bp = p; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rs != TF_OK) return rs;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        init_plans_locked();
        g_plan[op][cls][dtype][variant] = bp;
    }
    if (best) *best = bp;
    return TF_OK;
}

tf_status tf_plan_save(const char* path) {
    if (!path) return TF_ERR_ARG;
    std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "w");
    if (!f) return TF_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        init_plans_locked();
        fprintf(f, "# op class dtype variant block unroll blocks_per_sm tile "
                   "(class 0 single vector, 1 batched, 2 single vector of at most %d elements)\n",
                TF_SMALL_N);
        for (int op = 0; op < 2; ++op)
            for (int b = 0; b < kClasses; ++b)
                for (int dt = 0; dt < 2; ++dt)
                    for (int v = 0; v < kVariants; ++v) {
                        const tf_plan& p = g_plan[op][b][dt][v];
                        fprintf(f, "%d %d %d %d %d %d %d %d\n", op, b, dt, v, p.block, p.unroll,
                                p.blocks_per_sm, p.tile);
                    }
    }
    if (fclose(f) != 0) return TF_ERR_ARG;
    if (rename(tmp.c_str(), path) != 0) return TF_ERR_ARG;
    return TF_OK;
}

tf_status tf_plan_load(const char* path) {
    if (!path) return TF_ERR_ARG;
    FILE* f = fopen(path, "r");
    if (!f) return TF_ERR_ARG;
    char line[256];
    tf_status rs = TF_OK;
    std::vector<std::pair<int, tf_plan>> rows;
    while (fgets(line, sizeof line, f)) {
        if (line[0] == '#' || line[0] == '\n') continue;
        int op, b, dt, v; tf_plan p;
        if (sscanf(line, "%d %d %d %d %d %d %d %d", &op, &b, &dt, &v, &p.block, &p.unroll,
                   &p.blocks_per_sm, &p.tile) != 8 ||
            op < 0 || op > 1 || b < 0 || b >= kClasses || dt < 0 || dt > 1 || v < 0 ||
            v >= kVariants || !plan_valid(p, b, dt) || (b != TF_PLAN_BATCHED && p.tile != 0)) {
            rs = TF_ERR_ARG;
            break;
        }
        rows.push_back({((op * kClasses + b) * 2 + dt) * kVariants + v, p});
    }
    fclose(f);
    if (rs != TF_OK) return rs;
    std::lock_guard<std::mutex> lk(g_mu);
    init_plans_locked();
    for (auto& r : rows) {
        const int k = r.first;
        g_plan[k / (2 * kClasses * kVariants)][(k / (2 * kVariants)) % kClasses]
              [(k / kVariants) % 2][k % kVariants] = r.second;
    }
    return TF_OK;
}

tf_status tf_merge_pairs(const void* pairs, int64_t G, tf_dtype dtype, tf_variant variant,
                         void* out, uint32_t flags, tf_stream_t stream) {
    Range r("tf_merge_pairs");
    if (G < 0 || G > ((int64_t)1 << 30) || !out || (G > 0 && !pairs) || variant < 0 ||
        variant >= kVariants)
        return TF_ERR_ARG;
    if (dtype != TF_F32 && dtype != TF_F64) return TF_ERR_DTYPE;
    const uintptr_t oes = (dtype == TF_F64 || (flags & TF_OUT_F64)) ? 8 : 4;
    if ((uintptr_t)pairs % 8 || (uintptr_t)out % oes) return TF_ERR_ALIGN;
    int sms = 0;
    tf_status s = check_device(&sms);
    if (s != TF_OK) return s;
    return tf::launch_merge_pairs((const double*)pairs, G, dtype, variant, out,
                                  (flags & TF_OUT_F64) ? 1 : 0, (cudaStream_t)stream) == cudaSuccess
               ? TF_OK : TF_ERR_CUDA;
}

tf_status tf_count_large_errors(const void* pairs, int64_t npairs, tf_dtype pair_dtype,
                                double tau, int32_t* count, tf_stream_t stream) {
    if (npairs < 0 || !count || (npairs > 0 && !pairs) || !(tau >= 0.0)) return TF_ERR_ARG;
    if (pair_dtype != TF_F32 && pair_dtype != TF_F64) return TF_ERR_DTYPE;
    if ((uintptr_t)pairs % esize(pair_dtype) || (uintptr_t)count % 4) return TF_ERR_ALIGN;
    int sms = 0;
    tf_status s = check_device(&sms);
    if (s != TF_OK) return s;
    return tf::launch_large_errors(pairs, npairs, pair_dtype, tau, count, (cudaStream_t)stream) ==
                   cudaSuccess ? TF_OK : TF_ERR_CUDA;
}

tf_status tf_prim(int prim, tf_dtype dtype, const void* a, const void* b, void* x, void* y,
                  int64_t n, tf_stream_t stream) {
    if (prim < 0 || prim > 5 || n < 0 || (n > 0 && (!a || !b || !x || !y))) return TF_ERR_ARG;
    if (dtype != TF_F32 && dtype != TF_F64) return TF_ERR_DTYPE;
    int sms = 0;
    tf_status s = check_device(&sms);
    if (s != TF_OK) return s;
    return tf::launch_prim(prim, dtype, a, b, x, y, n, (cudaStream_t)stream) == cudaSuccess
               ? TF_OK : TF_ERR_CUDA;
}

tf_status tf_probe_read(const void* x, const void* y, int64_t nbytes, void* sink, int32_t blocks,
                        int32_t threads, int32_t unroll, tf_stream_t stream) {
    if (!x || !sink || nbytes < 0 || blocks < 1 || threads < 32 || threads > 1024 || threads % 32 ||
        (unroll != 1 && unroll != 2 && unroll != 4 && unroll != 8))
        return TF_ERR_ARG;
    if ((uintptr_t)x % 16 || (y && (uintptr_t)y % 16) || nbytes % 16) return TF_ERR_ALIGN;
    int sms = 0;
    tf_status s = check_device(&sms);
    if (s != TF_OK) return s;
    return tf::launch_probe_read(x, y, nbytes, sink, blocks, threads, unroll, (cudaStream_t)stream) ==
                   cudaSuccess ? TF_OK : TF_ERR_CUDA;
}

tf_status tf_probe_alu(int kind, int64_t iters, void* sink, int32_t blocks, int32_t threads,
                       tf_stream_t stream) {
    if (kind < 0 || kind > 10 || iters < 0 || !sink || blocks < 1 || threads < 32 ||
        threads > 1024 || threads % 32)
        return TF_ERR_ARG;
    int sms = 0;
    tf_status s = check_device(&sms);
    if (s != TF_OK) return s;
    return tf::launch_probe_alu(kind, iters, sink, blocks, threads, (cudaStream_t)stream) ==
                   cudaSuccess ? TF_OK : TF_ERR_CUDA;
}

tf_status tf_probe_wait(int32_t arrive, int64_t polls, int32_t* flag, tf_stream_t stream) {
    if ((arrive != 0 && arrive != 1) || polls < 1 || polls > (1 << 22) || !flag) return TF_ERR_ARG;
    if ((uintptr_t)flag % 4) return TF_ERR_ALIGN;
    int sms = 0;
    tf_status s = check_device(&sms);
    if (s != TF_OK) return s;
    return tf::launch_probe_wait(arrive, polls, flag, (cudaStream_t)stream) == cudaSuccess
               ? TF_OK : TF_ERR_CUDA;
}

}  // extern "C"
