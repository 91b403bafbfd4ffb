// Microbenchmarks of the per-SM rates the listing kernels are bound by
// (kcl_measure_int_peaks in include/kcl.h).  They give the roofline
// denominators of the integer-pipe kernels measured on the device at hand
// instead of table values: the BitJoin word of Algorithm 6 (a 32-bit AND, a
// population count and an accumulate over a shared-memory bit-row), the
// single instructions it is made of, 128-bit shared-memory loads, and the
// SplitMix64 round of the listing checksum.
//
// Every probe launches exactly one CTA per SM (the CTA asks for more than
// half of an SM's shared memory, so no two can share one), 1024 threads, and
// times its loop with the SM's own cycle counter (clock64) between two
// barriers, so each rate is per SM per SM clock and independent of the clock
// speed.  The SM clock itself is the probe's cycles over its CUDA-event time.
// Each thread runs 8 independent dependency chains, enough to cover the
// pipelines' latencies with 32 warps, and the chains' results are written
// out so no instruction is dead.
#include <algorithm>
#include <vector>

#include "kcl_internal.cuh"

namespace kcl {

namespace {

constexpr int kThreads = 1024;
constexpr int kChains = 8;
constexpr size_t kProbeSmem = 160 * 1024;  // > half an SM: one CTA per SM
constexpr uint32_t kRowU4 = 4096;           // uint4 rows region read by the shared-memory probes

enum Probe { P_POPC = 0, P_LOP3, P_IADD, P_BITJOIN, P_LDS128, P_MIX64, P_COUNT };

__device__ __forceinline__ uint32_t popc_asm(uint32_t x) {
    uint32_t r;
    asm volatile("popc.b32 %0, %1;" : "=r"(r) : "r"(x));
    return r;
}

__device__ __forceinline__ uint32_t xor3_asm(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t r;
    asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}

__device__ __forceinline__ uint32_t add_asm(uint32_t a, uint32_t b) {
    uint32_t r;
    asm volatile("add.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

// out[blockIdx.x] = cycles of the timed loop; sink[...] keeps the results live.
template <int P>
__global__ void __launch_bounds__(kThreads, 1) k_probe(uint32_t iters, uint32_t seed,
                                                       unsigned long long *cycles,
                                                       uint32_t *sink) {
    extern __shared__ uint4 rows[];
    const uint32_t tid = threadIdx.x;
    if (P == P_BITJOIN || P == P_LDS128)
        for (uint32_t i = tid; i < kRowU4; i += blockDim.x)
            rows[i] = make_uint4(seed * (i + 1), seed ^ i, ~i * 2654435761u, i + seed);
    uint32_t x[kChains];
    uint64_t h[kChains];
#pragma unroll
    for (int j = 0; j < kChains; j++) {
        x[j] = seed * (tid + 1) + 0x9E3779B9u * j;
        h[j] = ((uint64_t)x[j] << 32) | (x[j] ^ 0x85EBCA6Bu);
    }
    const uint32_t y = seed ^ 0x27D4EB2Fu, z = seed * 3u + 1u;
    __syncthreads();
    long long t0 = 0;
    if (tid == 0) t0 = clock64();
    __syncthreads();
    for (uint32_t it = 0; it < iters; it++) {
        if (P == P_POPC) {
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int j = 0; j < kChains; j++) x[j] = popc_asm(x[j]);
        } else if (P == P_LOP3) {
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int j = 0; j < kChains; j++) x[j] = xor3_asm(x[j], y, z);
        } else if (P == P_IADD) {
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int j = 0; j < kChains; j++) x[j] = add_asm(x[j], y);
        } else if (P == P_BITJOIN || P == P_LDS128) {
            // lane i reads row chunk (i + it * blockDim) (consecutive lanes,
            // consecutive 16-byte chunks: conflict-free) and the candidate
            // chunk it % 16, the same for every lane (a broadcast)
#pragma unroll
            for (int j = 0; j < kChains; j++) {
                const uint4 a = rows[(tid + (it * kChains + j) * 64u) & (kRowU4 - 1)];
                if (P == P_BITJOIN) {
                    const uint4 c = rows[(it * kChains + j) & 15u];
                    x[j] += __popc(a.x & c.x) + __popc(a.y & c.y) + __popc(a.z & c.z) +
                            __popc(a.w & c.w);
                } else {
                    x[j] = xor3_asm(x[j], a.x ^ a.y, a.z ^ a.w);
                }
            }
        } else if (P == P_MIX64) {
#pragma unroll
            for (int j = 0; j < kChains; j++) h[j] = mix64(h[j] ^ (uint64_t)it);
        }
    }
    __syncthreads();
    if (tid == 0) cycles[blockIdx.x] = (unsigned long long)(clock64() - t0);
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < kChains; j++) acc ^= x[j] ^ (uint32_t)h[j] ^ (uint32_t)(h[j] >> 32);
    sink[blockIdx.x * blockDim.x + tid] = acc;
}

// Operations (or bytes) one thread performs per loop iteration.
double ops_per_iter(int p) {
    switch (p) {
        case P_POPC: case P_LOP3: case P_IADD: return 4.0 * kChains;
        case P_BITJOIN: return 4.0 * kChains;   // BitJoin words
        case P_LDS128: return 16.0 * kChains;   // bytes
        case P_MIX64: return 1.0 * kChains;     // SplitMix64 rounds
    }
    return 0.0;
}

template <int P>
cudaError_t run_probe(int sms, uint32_t iters, unsigned long long *cyc, uint32_t *sink,
                      cudaStream_t s) {
    auto kern = k_probe<P>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kProbeSmem);
    if (e != cudaSuccess) return e;
    kern<<<sms, kThreads, kProbeSmem, s>>>(iters, 0x1234567u, cyc, sink);
    return cudaGetLastError();
}

cudaError_t launch_probe(int p, int sms, uint32_t iters, unsigned long long *cyc, uint32_t *sink,
                         cudaStream_t s) {
    switch (p) {
        case P_POPC: return run_probe<P_POPC>(sms, iters, cyc, sink, s);
        case P_LOP3: return run_probe<P_LOP3>(sms, iters, cyc, sink, s);
        case P_IADD: return run_probe<P_IADD>(sms, iters, cyc, sink, s);
        case P_BITJOIN: return run_probe<P_BITJOIN>(sms, iters, cyc, sink, s);
        case P_LDS128: return run_probe<P_LDS128>(sms, iters, cyc, sink, s);
        case P_MIX64: return run_probe<P_MIX64>(sms, iters, cyc, sink, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

}  // namespace kcl

extern "C" kcl_status kcl_measure_int_peaks(void *stream, kcl_int_peaks *out) {
    using namespace kcl;
    if (!out) return KCL_EINVAL;
    *out = kcl_int_peaks{};
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
        (void)cudaGetLastError();
        return KCL_ECUDA;
    }
    unsigned long long *cyc = nullptr;
    uint32_t *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::vector<unsigned long long> h((size_t)sms);
    kcl_status st = KCL_OK;
    if (cudaMalloc((void **)&cyc, (size_t)sms * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc((void **)&sink, (size_t)sms * kThreads * sizeof(uint32_t)) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        st = KCL_ENOMEM;
    double rate[P_COUNT] = {};
    double clk_sum = 0.0;
    int clk_n = 0;
    // iterations: about 2^24 cycles per probe at the expected rates
    const uint32_t iters[P_COUNT] = {1u << 14, 1u << 15, 1u << 15, 1u << 14, 1u << 15, 1u << 13};
    for (int p = 0; st == KCL_OK && p < P_COUNT; p++) {
        for (int rep = 0; rep < 2 && st == KCL_OK; rep++) {  // the first run warms up
            if (cudaEventRecord(e0, s) != cudaSuccess ||
                launch_probe(p, sms, iters[p], cyc, sink, s) != cudaSuccess ||
                cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaMemcpy(h.data(), cyc, (size_t)sms * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost) != cudaSuccess) {
                st = KCL_ECUDA;
                break;
            }
            if (rep == 0) continue;
            // the median SM: cycles differ slightly between SMs
            std::vector<unsigned long long> sorted(h);
            std::sort(sorted.begin(), sorted.end());
            const double cycles = (double)sorted[sorted.size() / 2];
            rate[p] = ops_per_iter(p) * kThreads * (double)iters[p] / cycles;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f) {
                clk_sum += (double)sorted.back() / (ms * 1e3);  // cycles per microsecond = MHz
                clk_n++;
            }
        }
    }
    (void)cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(cyc);
    cudaFree(sink);
    if (st != KCL_OK) return st;
    out->num_sms = (uint32_t)sms;
    out->sm_clock_mhz = clk_n ? clk_sum / clk_n : 0.0;
    out->popc_per_sm_clk = rate[P_POPC];
    out->lop3_per_sm_clk = rate[P_LOP3];
    out->iadd_per_sm_clk = rate[P_IADD];
    out->bitjoin_words_per_sm_clk = rate[P_BITJOIN];
    out->lds128_bytes_per_sm_clk = rate[P_LDS128];
    out->mix64_per_sm_clk = rate[P_MIX64];
    return KCL_OK;
}
