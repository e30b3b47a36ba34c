// tf_internal.h -- host-side declarations shared by the library's translation
// units (not part of the public ABI).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace tf {

// workspace header layout (device side mirrors it in tf_device.cuh)
constexpr size_t kHeaderBytes = 256;
constexpr int64_t kMinTile = 1024;       // smallest batched tile, in elements
constexpr int64_t kMaxFlatGrid = 8 * 256; // blocks_per_sm <= 8, SM count <= 256
constexpr size_t kPairBytes = 32;         // one (value, error) slot: two binary128 at most

// single-vector reduction: dtype 0 f32 / 1 f64, variant 0..3, dot 0/1
cudaError_t launch_flat(int dtype, int variant, int dot, int unroll, const void* x,
                        const void* y, int64_t n, void* out, void* ws, int block,
                        int64_t grid, int aligned, int out_f64, cudaStream_t st);

// batched reduction: the offsets check, the persistent kernel (the
// shared-memory ring one when `staged` and the plan fits its ring, else the
// register-loading one), then the merge of the segments over 2..32 tiles
cudaError_t launch_csr(int dtype, int variant, int dot, int unroll, const void* x,
                       const void* y, int64_t n, const int64_t* off, int64_t nseg,
                       void* out, void* ws, size_t ws_bytes, int block, int64_t grid,
                       int64_t tile, int aligned, int staged, int out_f64, cudaStream_t st);
size_t csr_ws_bytes(int64_t n, int64_t nseg);
// the batched kernel staged through shared memory by bulk copies (16-byte
// aligned inputs; plans whose tile and block fit its ring)
bool csr_tma_usable(int dtype, int dot, int block, int64_t tile);
size_t csr_tma_smem_bytes(int dot, int block);
cudaError_t launch_csr_tma(int dtype, int variant, int dot, int unroll, const void* x,
                           const void* y, const int64_t* off, int64_t nseg, void* out,
                           unsigned char* ws, size_t cnt_bytes, const int64_t* tile_seg,
                           int block, int64_t grid, int64_t tile, int out_f64, cudaStream_t st);

cudaError_t launch_prim(int prim, int dtype, const void* a, const void* b, void* x, void* y,
                        int64_t n, cudaStream_t st);
cudaError_t launch_merge_pairs(const double* pairs, int64_t G, int dtype, int variant, void* out,
                               int out_f64, cudaStream_t st);
cudaError_t launch_large_errors(const void* pairs, int64_t npairs, int dtype, double tau,
                                int* count, cudaStream_t st);
cudaError_t launch_probe_read(const void* x, const void* y, int64_t nbytes, void* sink,
                              int blocks, int threads, int unroll, cudaStream_t st);
cudaError_t launch_probe_alu(int kind, int64_t iters, void* sink, int blocks, int threads,
                             cudaStream_t st);
cudaError_t launch_probe_wait(int arrive, int64_t polls, int* flag, cudaStream_t st);

}  // namespace tf
