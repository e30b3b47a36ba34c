// tf_aux.cu -- elementwise error-free transforms and the two measurement
// probes (sm_103a).
//
//   prim_kernel   FAST-TWO-SUM / TWO-SUM / TwoProduct over arrays, the same
//                 device functions the reductions use.
//   read_probe    the paper's read1/read2: stream one or two arrays with the
//                 reductions' 128-bit loads and no arithmetic.
//   alu_probe     the paper's p-functions: the per-item operations from
//                 registers, 8 independent chains per thread, no loads.
//   merge_pairs_kernel  the rank-order merge of shard pairs (one vector
//                 reduced in contiguous shards, one per GPU or call).
#include "tf_async.cuh"
#include "tf_device.cuh"
#include "tf_internal.h"

namespace tf {

template <typename T>
__global__ void prim_kernel(int prim, const T* __restrict__ a, const T* __restrict__ b,
                            T* __restrict__ x, T* __restrict__ y, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        T u, v;
        if (prim == 0) fast_two_sum(a[i], b[i], u, v);
        else if (prim == 5) {        // binary64 FAST-TWO-SUM with the error on the integer pipe
            if constexpr (sizeof(T) == 8) {
                if (!fast_two_sum_h64(a[i], b[i], u, v)) fast_two_sum(a[i], b[i], u, v);
            } else {
                fast_two_sum(a[i], b[i], u, v);
            }
        }
        else if (prim == 1) two_sum(a[i], b[i], u, v);
        else if (prim == 2) two_product(a[i], b[i], u, v);
        else if (prim == 3) {        // binary64 TWO-SUM with the error on the integer pipe
            if constexpr (sizeof(T) == 8) {
                if (!two_sum_h64(a[i], b[i], u, v)) two_sum(a[i], b[i], u, v);
            } else {
                two_sum(a[i], b[i], u, v);
            }
        } else {                     // 4: binary64 TwoProduct on the integer pipe
            if constexpr (sizeof(T) == 8) {
                if (!two_product_i64(a[i], b[i], u, v)) two_product(a[i], b[i], u, v);
            } else {
                two_product(a[i], b[i], u, v);
            }
        }
        x[i] = u;
        y[i] = v;
    }
}

cudaError_t launch_prim(int prim, int dtype, const void* a, const void* b, void* x, void* y,
                        int64_t n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
    if (dtype == 0)
        prim_kernel<float><<<(unsigned)blocks, 256, 0, st>>>(prim, (const float*)a, (const float*)b,
                                                             (float*)x, (float*)y, n);
    else
        prim_kernel<double><<<(unsigned)blocks, 256, 0, st>>>(prim, (const double*)a, (const double*)b,
                                                              (double*)x, (double*)y, n);
    return cudaGetLastError();
}

// ------------------------------------------------------- error signalling
template <typename T>
__global__ void large_error_kernel(const T* __restrict__ pairs, int64_t npairs, double tau,
                                   int* __restrict__ count) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int local = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npairs; i += stride) {
        const double v = (double)pairs[2 * i], e = (double)pairs[2 * i + 1];
        // NaN compares false, so non-finite pairs count as flagged
        local += (fabs(e) <= tau * fabs(v) && isfinite(v) && isfinite(e)) ? 0 : 1;
    }
    local = __reduce_add_sync(FULL, local);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(count, local);
}

cudaError_t launch_large_errors(const void* pairs, int64_t npairs, int dtype, double tau,
                                int* count, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), st);
    if (e != cudaSuccess || npairs == 0) return e;
    const int64_t blocks = std::min<int64_t>((npairs + 255) / 256, 152 * 8);
    if (dtype == 0)
        large_error_kernel<float><<<(unsigned)blocks, 256, 0, st>>>((const float*)pairs, npairs, tau, count);
    else
        large_error_kernel<double><<<(unsigned)blocks, 256, 0, st>>>((const double*)pairs, npairs, tau, count);
    return cudaGetLastError();
}

// ------------------------------------------------------------- rank merge
// G shard pairs (binary64 (V, E) each: a shard's cross-block pair, as a
// binary32 call writes it with TF_OUT_F64 or a binary64 call writes it)
// merged in rank order by one thread, in the precision of the grid fold:
// the twofold variants by the TWO-SUM merge, plain and wide by one addition;
// the binary128 accumulator ('wide' binary64) as S <- (S + V_g) + E_g.
template <typename T, int VAR>
__global__ void merge_pairs_kernel(const double* __restrict__ pairs, int64_t G,
                                   void* __restrict__ out, int out_f64) {
    using Gt = typename GridAcc<T, VAR>::type;
    constexpr bool TW = twofold_v<VAR>;
    if (threadIdx.x != 0) return;
    if constexpr (sizeof(Gt) == 16) {
        q128 S(0);
        for (int64_t g = 0; g < G; ++g)
            S = q_add(q_add(S, q128(pairs[2 * g])), q128(pairs[2 * g + 1]));
        write_out<T, VAR, q128>(out, 0, S, q128(0), false);
    } else {
        Gt V = Gt(0), E = Gt(0);
        if (G > 0) { V = (Gt)pairs[0]; E = (Gt)pairs[1]; }
        for (int64_t g = 1; g < G; ++g) merge<TW>(V, E, (Gt)pairs[2 * g], (Gt)pairs[2 * g + 1]);
        write_out<T, VAR, Gt>(out, 0, V, E, out_f64 != 0);
    }
}

template <typename T>
static void launch_merge_t(int variant, const double* pairs, int64_t G, void* out, int out_f64,
                           cudaStream_t st) {
    switch (variant) {
    case PLAIN: merge_pairs_kernel<T, PLAIN><<<1, 32, 0, st>>>(pairs, G, out, out_f64); break;
    case FAST: merge_pairs_kernel<T, FAST><<<1, 32, 0, st>>>(pairs, G, out, out_f64); break;
    case RIGOROUS: merge_pairs_kernel<T, RIGOROUS><<<1, 32, 0, st>>>(pairs, G, out, out_f64); break;
    case WIDE: merge_pairs_kernel<T, WIDE><<<1, 32, 0, st>>>(pairs, G, out, out_f64); break;
    default: merge_pairs_kernel<T, KAHAN><<<1, 32, 0, st>>>(pairs, G, out, out_f64); break;
    }
}

cudaError_t launch_merge_pairs(const double* pairs, int64_t G, int dtype, int variant, void* out,
                               int out_f64, cudaStream_t st) {
    if (dtype == 0) launch_merge_t<float>(variant, pairs, G, out, out_f64, st);
    else launch_merge_t<double>(variant, pairs, G, out, out_f64, st);
    return cudaGetLastError();
}

// ------------------------------------------------------------ read probe
// U 16-byte loads of each array in flight per thread and step (U = 1, 2, 4
// or 8); the caller picks U and the launch shape, and a sweep over them gives
// the best streaming read rate of one or two arrays.
template <int U, bool TWO>
__global__ void __launch_bounds__(1024)
read_probe(const float* __restrict__ x, const float* __restrict__ y, int64_t nvec,
           unsigned int* __restrict__ sink) {
    const int64_t P = (int64_t)gridDim.x * blockDim.x;
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned int acc = 0;
    for (; j + (U - 1) * P < nvec; j += U * P) {
        float r[U][4], q[U][4];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            ld_stream(x + 4 * (j + u * P), r[u]);
            if constexpr (TWO) ld_stream(y + 4 * (j + u * P), q[u]);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                acc ^= __float_as_uint(r[u][l]);
                if constexpr (TWO) acc ^= __float_as_uint(q[u][l]);
            }
    }
    for (; j < nvec; j += P) {
        float r[4], q[4];
        ld_stream(x + 4 * j, r);
        if constexpr (TWO) ld_stream(y + 4 * j, q);
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            acc ^= __float_as_uint(r[l]);
            if constexpr (TWO) acc ^= __float_as_uint(q[l]);
        }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) acc ^= __shfl_xor_sync(FULL, acc, o);
    __shared__ unsigned int sm[32];
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t ^= sm[w];
        sink[blockIdx.x] = t;
    }
}

template <int U>
static void launch_read_u(const void* x, const void* y, int64_t nvec, void* sink, int blocks,
                          int threads, cudaStream_t st) {
    if (y)
        read_probe<U, true><<<blocks, threads, 0, st>>>((const float*)x, (const float*)y, nvec,
                                                        (unsigned int*)sink);
    else
        read_probe<U, false><<<blocks, threads, 0, st>>>((const float*)x, nullptr, nvec,
                                                         (unsigned int*)sink);
}

cudaError_t launch_probe_read(const void* x, const void* y, int64_t nbytes, void* sink,
                              int blocks, int threads, int unroll, cudaStream_t st) {
    const int64_t nvec = nbytes / 16;
    switch (unroll) {
    case 1: launch_read_u<1>(x, y, nvec, sink, blocks, threads, st); break;
    case 2: launch_read_u<2>(x, y, nvec, sink, blocks, threads, st); break;
    case 4: launch_read_u<4>(x, y, nvec, sink, blocks, threads, st); break;
    case 8: launch_read_u<8>(x, y, nvec, sink, blocks, threads, st); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------- ALU probe
// kind: 0 FADD, 1 DADD, 2 FFMA, 3 DFMA, 4 IADD (32-bit), 5 / 6 the binary32
// fast / rigorous step, 7 / 8 the binary64 fast / rigorous step, 9 DMUL,
// 10 a binary64 add issued as fma(a, one, b) with `one` = 1.0 computed at run
// time (the form the binary64 sums use, see dadd in tf_device.cuh).
template <int KIND>
__global__ void __launch_bounds__(1024)
alu_probe(int64_t iters, unsigned int* __restrict__ sink, float seed) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned int out = 0;
    if constexpr (KIND == 0 || KIND == 2 || KIND == 5 || KIND == 6) {
        float c[8], e[8];
        const float d = seed * 1e-7f, m = 1.0f - seed * 1e-9f;
#pragma unroll
        for (int k = 0; k < 8; ++k) { c[k] = seed + (float)(tid + k); e[k] = 0.0f; }
        for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if constexpr (KIND == 0) c[k] = __fadd_rn(c[k], d);
                else if constexpr (KIND == 2) c[k] = __fmaf_rn(c[k], m, d);
                else if constexpr (KIND == 5) feed<FAST, false>(c[k], e[k], d, 0.0f);
                else feed<RIGOROUS, false>(c[k], e[k], d, 0.0f);
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) out ^= __float_as_uint(c[k]) ^ __float_as_uint(e[k]);
    } else if constexpr (KIND == 1 || KIND == 3 || KIND == 7 || KIND == 8 || KIND == 9 ||
                         KIND == 10) {
        double c[8], e[8];
        const double d = (double)seed * 1e-15, m = 1.0 - (double)seed * 1e-17;
        // a 1.0 the compiler cannot see (it would fold a known 1.0 into a DADD)
        const double one = (double)(seed > 0.0f) + (double)(iters < 0);
#pragma unroll
        for (int k = 0; k < 8; ++k) { c[k] = (double)seed + (double)(tid + k); e[k] = 0.0; }
        for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if constexpr (KIND == 1) c[k] = __dadd_rn(c[k], d);
                else if constexpr (KIND == 3) c[k] = __fma_rn(c[k], m, d);
                else if constexpr (KIND == 7) feed<FAST, false>(c[k], e[k], d, 0.0);
                else if constexpr (KIND == 8) feed<RIGOROUS, false>(c[k], e[k], d, 0.0);
                else if constexpr (KIND == 9) c[k] = __dmul_rn(c[k], m);
                else c[k] = __fma_rn(c[k], one, d);
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            unsigned long long b = __double_as_longlong(c[k]) ^ __double_as_longlong(e[k]);
            out ^= (unsigned int)b ^ (unsigned int)(b >> 32);
        }
    } else {  // KIND 4: 32-bit integer adds
        unsigned int c[8];
        const unsigned int d = __float_as_uint(seed) | 1u;
#pragma unroll
        for (int k = 0; k < 8; ++k) c[k] = (unsigned int)(tid + k);
        for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < 8; ++k) asm volatile("add.u32 %0, %0, %1;" : "+r"(c[k]) : "r"(d));
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) out ^= c[k];
    }
    sink[tid] = out;
}

cudaError_t launch_probe_alu(int kind, int64_t iters, void* sink, int blocks, int threads,
                             cudaStream_t st) {
    unsigned int* s = (unsigned int*)sink;
    const float seed = 1.25f;
    switch (kind) {
    case 0: alu_probe<0><<<blocks, threads, 0, st>>>(iters, s, seed); break;
    case 1: alu_probe<1><<<blocks, threads, 0, st>>>(iters, s, seed); break;
    case 2: alu_probe<2><<<blocks, threads, 0, st>>>(iters, s, seed); break;
    case 3: alu_probe<3><<<blocks, threads, 0, st>>>(iters, s, seed); break;
    case 4: alu_probe<4><<<blocks, threads, 0, st>>>(iters, s, seed); break;
    case 5: alu_probe<5><<<blocks, threads, 0, st>>>(iters, s, seed); break;
    case 6: alu_probe<6><<<blocks, threads, 0, st>>>(iters, s, seed); break;
    case 7: alu_probe<7><<<blocks, threads, 0, st>>>(iters, s, seed); break;
    case 8: alu_probe<8><<<blocks, threads, 0, st>>>(iters, s, seed); break;
    case 9: alu_probe<9><<<blocks, threads, 0, st>>>(iters, s, seed); break;
    case 10: alu_probe<10><<<blocks, threads, 0, st>>>(iters, s, seed); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// The batched kernel's bounded mbarrier wait, on one barrier of one thread:
// with arrive = 0 nothing completes the phase and the wait gives up after
// `polls` polls; with arrive = 1 the thread completes it first.  flag[0] = 1
// if the wait gave up, else 0; the barrier is then released, nothing is left
// in flight and the context stays usable.
__global__ void wait_probe_kernel(int arrive, unsigned polls, int* flag) {
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t b = smem_u32(&bar);
    mbar_init(b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (arrive) mbar_arrive_expect_tx(b, 0);
    flag[0] = mbar_wait(b, 0, polls) ? 0 : 1;
}

cudaError_t launch_probe_wait(int arrive, int64_t polls, int* flag, cudaStream_t st) {
    wait_probe_kernel<<<1, 1, 0, st>>>(arrive, (unsigned)polls, flag);
    return cudaGetLastError();
}

}  // namespace tf
