// tf_noalloc.cu -- tf_sum_noalloc: the single-vector twofold sum with its
// scratch memory in a fixed, library-owned device array.
//
// tf_sum needs a caller workspace (one pair per block plus a ticket).  Some
// callers cannot provide one because they cannot call cudaMalloc: code that
// runs under a host framework which owns all device memory through its own
// pool and forbids raw allocations, code with a fixed device-memory budget
// that must not grow after start-up, and latency-critical paths where the
// device-wide synchronization that cudaMalloc may imply is not acceptable.
// For them this entry point keeps the scratch in a file-scope __device__
// array of a stated size, present on every GPU that loads the library until
// the process exits.  The reduction kernel, launch shape and result bits are
// those of tf_sum.
#include "twofold.h"
#include "tf_internal.h"

#include <mutex>

namespace {

// at most 2048 block pairs (16 bytes each) after a 256-byte header: 33,024 bytes
constexpr int64_t kNoallocMaxBlocks = 2048;
constexpr size_t kNoallocBytes = tf::kHeaderBytes + 16 * (size_t)kNoallocMaxBlocks;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// In host code g_noalloc_scratch names a host-side stand-in, not device
// memory, so the device address is looked up once per device (with that
// device current) and cached.
std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {};

tf_status noalloc_scratch(void** addr) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return TF_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return TF_ERR_CUDA;
        }
        g_noalloc_addr[dev] = p;
    }
    *addr = g_noalloc_addr[dev];
    return TF_OK;
}

}  // namespace

extern "C" tf_status tf_sum_noalloc(const void* x, int64_t n, tf_dtype dtype,
                                    tf_variant variant, void* out, uint32_t flags,
                                    tf_stream_t stream) {
    if (variant < TF_PLAIN || variant > TF_KAHAN) return TF_ERR_ARG;
    if (dtype != TF_F32 && dtype != TF_F64) return TF_ERR_DTYPE;
    if (n < 0 || !out || (n > 0 && !x)) return TF_ERR_ARG;
    const uintptr_t es = dtype == TF_F32 ? 4 : 8;
    if ((uintptr_t)x % es || (uintptr_t)out % ((flags & TF_OUT_F64) ? 8 : es)) return TF_ERR_ALIGN;

    int32_t block = 0, unroll = 0;
    int64_t grid = 0, tile = 0;
    tf_status s = tf_launch_shape(TF_OP_SUM, 0, dtype, variant, n, &block, &unroll, &grid, &tile);
    if (s != TF_OK) return s;
    // every launch shape tf_launch_shape gives has at most kMaxFlatGrid blocks
    // of 16-byte pairs, which the array holds; a binary128 accumulator
    // ('wide' binary64) takes two 16-byte slots per block, so those calls
    // are limited to half as many blocks (a plan of more than 1024 blocks
    // for that key, e.g. 8 blocks per SM on 152 SMs, is rejected)
    static_assert(tf::kMaxFlatGrid <= kNoallocMaxBlocks, "scratch array below the largest grid");
    if (dtype == TF_F64 && variant == TF_WIDE && grid > kNoallocMaxBlocks / 2) return TF_ERR_UNSUPPORTED;

    void* scratch = nullptr;
    if ((s = noalloc_scratch(&scratch)) != TF_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    // the shared array keeps the previous call's contents: clear the tickets
    if (cudaMemsetAsync(scratch, 0, tf::kHeaderBytes, st) != cudaSuccess) return TF_ERR_CUDA;
    const int aligned = (uintptr_t)x % 16 == 0;
    cudaError_t e = tf::launch_flat(dtype, variant, 0, unroll, x, nullptr, n, out, scratch, block,
                                    grid, aligned, (flags & TF_OUT_F64) ? 1 : 0, st);
    return e == cudaSuccess ? TF_OK : TF_ERR_CUDA;
}
