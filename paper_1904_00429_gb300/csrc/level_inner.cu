// level_inner.cu -- the inner-product case m = p = 1 (Sec. 2: the estimator of a^T b of a random
// row a and column b) on the CUDA cores, FP64 and FP32, uniform index law.
//
// A sample's D is one number, so the 64 x 64 output tile of the general CUDA-core kernel would
// idle all but one of its threads.  Here one warp evaluates one sample: its lanes take the slot
// pairs of the sample (one Philox block per pair of indices), gather the sampled (M, S) and
// (M', S') pairs (one 64-byte row of the plan's layout per index), generate a = M + S z_A and
// b = M' + S' z_B (the first normal of the entry's Philox block, row 0 / column 0), and sum
// w_t a_t b_t -- or, with a targeted function, the fine and coarse sums apart -- then reduce over
// the warp in a fixed shuffle tree.  A block of 8 warps covers one chunk of samples; thread 0
// folds the chunk's samples in sample order into its sum and its M2 (Welford's update, as in the
// other level kernels), so the partials and the merge are those of the general kernels with
// m p = 1 and one tile.
#include <cuda_runtime.h>

#include "internal.h"
#include "rng.cuh"

namespace mlmc {
namespace {

constexpr int kInnerWarps = 8;

template <typename T>
__device__ __forceinline__ T first_normal(uint4 w);

template <>
__device__ __forceinline__ double first_normal<double>(uint4 w)
{
    double zc, zs;
    box_muller_f64(w.x, w.y, zc, zs);
    return zc;
}

template <>
__device__ __forceinline__ float first_normal<float>(uint4 w)
{
    float zc, zs;
    box_muller_f32(w.x, w.y, zc, zs);
    return zc;
}

// |x| H(2 - x), H(0) = 1 (mlmc_function 1); F = 0: the identity
template <int F, typename T>
__device__ __forceinline__ T inner_f(T x)
{
    if constexpr (F == 1) return (T(2) - x >= T(0)) ? fabs(x) : T(0);
    return x;
}

template <typename T, int F>
__global__ void __launch_bounds__(kInnerWarps * 32) level_inner_kernel(const LevelParams prm)
{
    __shared__ T d_s[kMaxChunkSamples];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t chunk = prm.chunk0 + blockIdx.x;
    const uint64_t sa = max(prm.s_begin, chunk * static_cast<uint64_t>(prm.chunk));
    const uint64_t sb = min(prm.s_end, (chunk + 1) * static_cast<uint64_t>(prm.chunk));
    const int ns = static_cast<int>(sb - sa);
    const T* PA = static_cast<const T*>(prm.PA);
    const T* PB = static_cast<const T*>(prm.PB);
    const T wf = static_cast<T>(prm.w_fine);
    const T wc = static_cast<T>(prm.w_coarse);
    const T wcn = static_cast<T>(prm.w_fine - prm.w_coarse);   // n / c_{l-1}
    for (int si = warp; si < ns; si += kInnerWarps) {
        const uint64_t s = sa + static_cast<uint64_t>(si);
        const uint32_t lsw = level_sample_word(prm.l, s);
        const uint32_t s_lo = static_cast<uint32_t>(s);
        T fine = T(0), coarse = T(0);
        for (int tp = lane; 2 * tp < prm.c; tp += 32) {
            int64_t r0, r1;
            index_pair(prm.keyI, lsw, s_lo, tp, static_cast<uint64_t>(prm.n), r0, r1);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int t = 2 * tp + e;
                if (t >= prm.c) break;
                const int64_t k = e ? r1 : r0;
                const T* pa = PA + k * prm.ldPA;
                const T* pb = PB + k * prm.ldPB;
                const T za = first_normal<T>(philox4x32_10(make_uint4(0u, static_cast<uint32_t>(k), s_lo, lsw), prm.keyA));
                const T zb = first_normal<T>(philox4x32_10(make_uint4(0u, static_cast<uint32_t>(k), s_lo, lsw), prm.keyB));
                const T a = fma(pa[1], za, pa[0]);
                const T b = fma(pb[1], zb, pb[0]);
                const bool is_coarse = prm.l > 0 && (t % prm.R) == prm.R - 1;
                if constexpr (F == 0) {
                    fine = fma((is_coarse ? wc : wf) * a, b, fine);
                } else {
                    fine = fma(a, b, fine);
                    if (is_coarse) coarse = fma(a, b, coarse);
                }
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            fine += __shfl_xor_sync(0xffffffffu, fine, off);
            if constexpr (F != 0) coarse += __shfl_xor_sync(0xffffffffu, coarse, off);
        }
        if (lane == 0) {
            T D = fine;
            if constexpr (F != 0)
                D = prm.l > 0 ? inner_f<F>(wf * fine) - inner_f<F>(wcn * coarse) : inner_f<F>(wf * fine);
            d_s[si] = D;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // the chunk's sum and its M2 by Welford's update in sample order:
        // with k samples before, M2 += (k D - sum_k)^2 / (k (k + 1))
        T sum = T(0), q = T(0);   // in T: FP32 plans stay in FP32
        for (int si = 0; si < ns; ++si) {
            const T D = d_s[si];
            if (si > 0) {
                const T dk = fma(static_cast<T>(si), D, -sum);
                q = fma(dk * dk, T(1) / static_cast<T>(si * (si + 1)), q);
            }
            sum += D;
        }
        static_cast<T*>(prm.partial_sum)[blockIdx.x] = sum;
        prm.partial_q[blockIdx.x] = static_cast<double>(q);
    }
}

template <typename T>
cudaError_t launch(const LevelParams& prm, int f, cudaStream_t st)
{
    const dim3 grid(static_cast<unsigned>(prm.nchunks));
    if (f == 0)
        level_inner_kernel<T, 0><<<grid, kInnerWarps * 32, 0, st>>>(prm);
    else if (f == 1)
        level_inner_kernel<T, 1><<<grid, kInnerWarps * 32, 0, st>>>(prm);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_level_inner(const LevelParams& prm, bool f64, int f, cudaStream_t st)
{
    if (prm.m != 1 || prm.p != 1 || prm.tiles_m != 1 || prm.tiles_p != 1) return cudaErrorInvalidValue;
    return f64 ? launch<double>(prm, f, st) : launch<float>(prm, f, st);
}

}  // namespace mlmc
