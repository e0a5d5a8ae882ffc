// genrate.cu -- the entry-generation ceiling of the reduced-precision level kernels, and the
// arithmetic throughput probes (FP32, FP64, INT32, special-function unit) behind the ALU rooflines.
//
// Every sampled entry the BF16/E4M3 level kernels consume is a fresh normal (Philox4x32-10 block
// per four entries, special-function-unit Box-Muller per pair), scaled and shifted (M + S z) and
// rounded to bfloat16.  This kernel does only that, with eight independent Philox chains per
// thread (as the level kernel's generator does), in one wave of as many resident blocks as fit,
// so its rate is the number of entries per second the GPU's integer, FP32 and special-function
// pipes can produce: the third bound of the level kernel beside HBM bandwidth and tensor
// throughput.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "rng.cuh"

namespace mlmc {
namespace {

constexpr int kRateThreads = 256;
constexpr uint32_t kRateBlocks = 2048;   // Philox blocks per thread (8192 entries)

__device__ __forceinline__ uint32_t bf16x2_bits(float a, float b)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__global__ void __launch_bounds__(kRateThreads) generation_rate_kernel(const PhiloxRoundKeys rk, float m0, float s0,
                                                                       uint32_t* sink)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
#pragma unroll 1
    for (uint32_t b = 0; b < kRateBlocks; b += 8) {
        uint4 w[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) w[u] = philox4x32_10_rk(make_uint4(t, b + u, 0x5A5Au, 0u), rk);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            float z[4];
            normals4_mufu(w[u], z);
            const float m = m0 + static_cast<float>(u);
            acc ^= bf16x2_bits(fmaf(s0, z[0], m), fmaf(s0, z[1], m));
            acc ^= bf16x2_bits(fmaf(s0, z[2], m), fmaf(s0, z[3], m));
        }
    }
    if (acc == 0x9E3779B9u) sink[t & 255] = acc;   // keeps the work observable; practically never taken
}

// Throughput probes: every thread runs kChains independent dependency chains of kChainLen
// operations of one kind, in one wave of as many resident blocks as fit; the rate is the count of
// operations over the best time of three launches after a warm-up.  KIND 0: FP32 FMA, 1: FP64 FMA,
// 2: INT32 multiply-add, 3: special-function sine (sin.approx, one MUFU operation each).
constexpr int kChains = 8;
constexpr int kChainLen = 4096;

template <int KIND>
__global__ void __launch_bounds__(kRateThreads) peak_chain_kernel(float f0, double d0, uint32_t u0, uint32_t* sink)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t out = 0;
    if constexpr (KIND == 0) {
        float a[kChains];
        const float b = f0 * 0.999f, c = f0 * 1e-3f;
#pragma unroll
        for (int u = 0; u < kChains; ++u) a[u] = f0 + static_cast<float>(t + u);
#pragma unroll 1
        for (int i = 0; i < kChainLen; i += 8)
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int u = 0; u < kChains; ++u) a[u] = fmaf(a[u], b, c);
#pragma unroll
        for (int u = 0; u < kChains; ++u) out ^= __float_as_uint(a[u]);
    } else if constexpr (KIND == 1) {
        double a[kChains];
        const double b = d0 * 0.999, c = d0 * 1e-3;
#pragma unroll
        for (int u = 0; u < kChains; ++u) a[u] = d0 + static_cast<double>(t + u);
#pragma unroll 1
        for (int i = 0; i < kChainLen; i += 8)
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int u = 0; u < kChains; ++u) a[u] = fma(a[u], b, c);
#pragma unroll
        for (int u = 0; u < kChains; ++u) out ^= static_cast<uint32_t>(__double_as_longlong(a[u]));
    } else if constexpr (KIND == 2) {
        uint32_t a[kChains];
        const uint32_t b = u0 | 1u, c = u0 >> 3;
#pragma unroll
        for (int u = 0; u < kChains; ++u) a[u] = u0 + t + static_cast<uint32_t>(u);
#pragma unroll 1
        for (int i = 0; i < kChainLen; i += 8)
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int u = 0; u < kChains; ++u) a[u] = a[u] * b + c;
#pragma unroll
        for (int u = 0; u < kChains; ++u) out ^= a[u];
    } else {
        float a[kChains];
#pragma unroll
        for (int u = 0; u < kChains; ++u) a[u] = f0 + 1e-3f * static_cast<float>(t + u);
#pragma unroll 1
        for (int i = 0; i < kChainLen; i += 8)
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int u = 0; u < kChains; ++u) a[u] = __sinf(a[u]);
#pragma unroll
        for (int u = 0; u < kChains; ++u) out ^= __float_as_uint(a[u]);
    }
    if (out == 0x9E3779B9u) sink[t & 255] = out;   // keeps the work observable; practically never taken
}

template <int KIND>
cudaError_t time_chain(cudaStream_t st, int num_sms, uint32_t* sink, cudaEvent_t e0, cudaEvent_t e1, double* ops_per_s)
{
    int per_sm = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, peak_chain_kernel<KIND>, kRateThreads, 0);
    const unsigned grid = static_cast<unsigned>(num_sms * (per_sm > 0 ? per_sm : 1));
    float best = 0.0f;
    for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {   // the first run warms up
        err = cudaEventRecord(e0, st);
        if (err == cudaSuccess) {
            peak_chain_kernel<KIND><<<grid, kRateThreads, 0, st>>>(0.5f, 0.5, 0x9E37u, sink);
            err = cudaGetLastError();
        }
        if (err == cudaSuccess) err = cudaEventRecord(e1, st);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err == cudaSuccess && rep > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    if (err == cudaSuccess) {
        const double ops = double(grid) * kRateThreads * kChains * kChainLen;
        *ops_per_s = best > 0.0f ? ops / (double(best) * 1e-3) : 0.0;
    }
    return err;
}

}  // namespace

cudaError_t measure_peaks(cudaStream_t st, int num_sms, double out[4])
{
    uint32_t* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaMalloc(&sink, 256 * sizeof(uint32_t));
    if (err == cudaSuccess) err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    if (err == cudaSuccess) err = time_chain<0>(st, num_sms, sink, e0, e1, &out[0]);
    if (err == cudaSuccess) err = time_chain<1>(st, num_sms, sink, e0, e1, &out[1]);
    if (err == cudaSuccess) err = time_chain<2>(st, num_sms, sink, e0, e1, &out[2]);
    if (err == cudaSuccess) err = time_chain<3>(st, num_sms, sink, e0, e1, &out[3]);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    return err;
}

cudaError_t measure_generation_rate(cudaStream_t st, int num_sms, double* entries_per_s)
{
    uint32_t* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaMalloc(&sink, 256 * sizeof(uint32_t));
    if (err == cudaSuccess) err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    const PhiloxRoundKeys rk = philox_round_keys(make_uint2(0x1234u, 0x5678u));
    int per_sm = 0;   // resident blocks per SM: one full wave
    if (err == cudaSuccess)
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, generation_rate_kernel, kRateThreads, 0);
    const unsigned grid = static_cast<unsigned>(num_sms * (per_sm > 0 ? per_sm : 1));
    float best = 0.0f;
    for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {   // the first run warms up
        err = cudaEventRecord(e0, st);
        if (err == cudaSuccess) {
            generation_rate_kernel<<<grid, kRateThreads, 0, st>>>(rk, 0.25f, 0.5f, sink);
            err = cudaGetLastError();
        }
        if (err == cudaSuccess) err = cudaEventRecord(e1, st);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err == cudaSuccess && rep > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (err == cudaSuccess) {
        const double entries = double(grid) * kRateThreads * kRateBlocks * 4.0;
        *entries_per_s = best > 0.0f ? entries / (double(best) * 1e-3) : 0.0;
    }
    return err;
}

}  // namespace mlmc
