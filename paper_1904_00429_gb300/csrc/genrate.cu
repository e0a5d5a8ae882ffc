// genrate.cu -- the entry-generation ceiling of the reduced-precision level kernels.
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

}  // namespace

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
