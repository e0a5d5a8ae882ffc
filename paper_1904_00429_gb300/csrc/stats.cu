// stats.cu -- per-level statistics (Eq. hatYl, Remark 3.6), the telescoping
// sum (Eq. hatY), the parameter layout copy and the verification kernels.
//
// A level's state is (N, per-entry FP64 sum of D, FP64 sum of ||D||_F^2).
// Chunk partials are added to it strictly in chunk order, one thread per
// entry, so the state is a deterministic function of the samples folded in.
// Y_l = sum / N and V_l = (sumsq - ||sum||^2 / N) / (N - 1).
#include <algorithm>

#include <cuda_runtime.h>

#include "internal.h"
#include "rng.cuh"

namespace mlmc {
namespace {

constexpr int kMergeThreads = 256;
constexpr int kMaxMergeChunks = 4096;

template <typename T>
__global__ void merge_sum_kernel(const T* __restrict__ partial, int nchunks, int64_t mp, double* level_sum)
{
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= mp) return;
    double acc = level_sum[e];
    int c = 0;
    // eight independent loads in flight, then the adds in chunk order
    for (; c + 8 <= nchunks; c += 8) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = static_cast<double>(partial[static_cast<int64_t>(c + u) * mp + e]);
#pragma unroll
        for (int u = 0; u < 8; ++u) acc += v[u];
    }
    for (; c < nchunks; ++c) acc += static_cast<double>(partial[static_cast<int64_t>(c) * mp + e]);
    level_sum[e] = acc;
}

// One block: chunk totals in parallel (tiles in fixed order), then one thread
// adds them to the level's sum of squares in chunk order.
__global__ void merge_sumsq_kernel(const double* __restrict__ partial_q, int nchunks, int tiles,
                                   double* level_sumsq)
{
    __shared__ double chunk_q[kMaxMergeChunks];
    for (int c = threadIdx.x; c < nchunks; c += blockDim.x) {
        double t = 0.0;
        for (int x = 0; x < tiles; ++x) t += partial_q[static_cast<int64_t>(c) * tiles + x];
        chunk_q[c] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double acc = *level_sumsq;
        for (int c = 0; c < nchunks; ++c) acc += chunk_q[c];
        *level_sumsq = acc;
    }
}

// Batched merge: the jobs of one wave (count read from the device), each folded into its
// level's FP64 state in chunk order exactly as merge_sum_kernel / merge_sumsq_kernel do.  The
// grid is fixed (grid-stride over jobs in y and elements in x) so that a captured graph stays
// valid when the wave's contents change; a wave holds at most one job per (problem, level).
__global__ void merge_batch_kernel(const MergeJob* __restrict__ jobs, const int* __restrict__ njobs_dev)
{
    __shared__ double chunk_q[kMaxMergeChunks];
    const int njobs = *njobs_dev;
    for (int j = blockIdx.y; j < njobs; j += gridDim.y) {
        const MergeJob jb = jobs[j];
        for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < jb.mp;
             e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
            double acc = jb.sum[e];
            int c = 0;
            for (; c + 8 <= jb.nchunks; c += 8) {
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = jb.partial[static_cast<int64_t>(c + u) * jb.mp + e];
#pragma unroll
                for (int u = 0; u < 8; ++u) acc += static_cast<double>(v[u]);
            }
            for (; c < jb.nchunks; ++c) acc += static_cast<double>(jb.partial[static_cast<int64_t>(c) * jb.mp + e]);
            jb.sum[e] = acc;
        }
        if (blockIdx.x == 0) {
            for (int c = threadIdx.x; c < jb.nchunks; c += blockDim.x) {
                double t = 0.0;
                for (int x = 0; x < jb.tiles; ++x) t += jb.partial_q[static_cast<int64_t>(c) * jb.tiles + x];
                chunk_q[c] = t;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                double acc = *jb.sumsq;
                for (int c = 0; c < jb.nchunks; ++c) acc += chunk_q[c];
                *jb.sumsq = acc;
            }
            __syncthreads();
        }
    }
}

// One block per level: ||sum||^2 by a fixed-shape reduction, then M2.
__global__ void finalize_kernel(const double* __restrict__ sum, const double* __restrict__ sumsq,
                                const LevelCounts counts, int first, int64_t mp, double* mean, double* M2)
{
    __shared__ double red[kMergeThreads / 32];
    const int lvl = blockIdx.x;
    const double* s = sum + static_cast<int64_t>(lvl) * mp;
    const uint64_t n = counts.v[first + lvl];
    const double inv = n > 0 ? 1.0 / static_cast<double>(n) : 0.0;
    double local = 0.0;
    for (int64_t e = threadIdx.x; e < mp; e += blockDim.x) {
        const double v = s[e];
        local = fma(v, v, local);
        if (mean) mean[static_cast<int64_t>(lvl) * mp + e] = v * inv;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) local += __shfl_xor_sync(0xffffffffu, local, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kMergeThreads / 32; ++w) t += red[w];
        M2[lvl] = n > 0 ? sumsq[lvl] - t * inv : 0.0;
    }
}

__global__ void telescoping_kernel(const double* __restrict__ sum, const LevelCounts counts, int levels,
                                   int64_t mp, double* yhat)
{
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= mp) return;
    double y = 0.0;
    for (int l = 0; l < levels; ++l) {
        const uint64_t n = counts.v[l];
        if (n > 0) y += sum[static_cast<int64_t>(l) * mp + e] / static_cast<double>(n);
    }
    yhat[e] = y;
}

template <typename S>
__device__ __forceinline__ double load_param(const void* p, int64_t off)
{
    return static_cast<double>(static_cast<const S*>(p)[off]);
}

// [M|S] (m x n, row-major, ldA) -> PA[k][i][2] through a 32 x 32 shared tile.
template <typename S, typename D>
__global__ void layout_A_kernel(const void* M, const void* Sg, int64_t ldA, int64_t m, int64_t n,
                                int64_t m_pad, D* PA, int64_t ld_dst)
{
    __shared__ double tm[32][33];
    __shared__ double ts[32][33];
    const int64_t k0 = static_cast<int64_t>(blockIdx.x) * 32;
    const int64_t i0 = static_cast<int64_t>(blockIdx.y) * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int64_t i = i0 + y, k = k0 + threadIdx.x;
        const bool ok = i < m && k < n;
        tm[y][threadIdx.x] = ok ? load_param<S>(M, i * ldA + k) : 0.0;
        ts[y][threadIdx.x] = ok ? load_param<S>(Sg, i * ldA + k) : 0.0;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int64_t k = k0 + y, i = i0 + threadIdx.x;
        if (k < n && i < m_pad) {
            PA[k * ld_dst + 2 * i] = static_cast<D>(tm[threadIdx.x][y]);
            PA[k * ld_dst + 2 * i + 1] = static_cast<D>(ts[threadIdx.x][y]);
        }
    }
}

// [M'|S'] (n x p, row-major, ldB) -> PB[k][j][2] (already row-contiguous: interleave only).
template <typename S, typename D>
__global__ void layout_B_kernel(const void* Mp, const void* Sp, int64_t ldB, int64_t n, int64_t p,
                                int64_t p_pad, D* PB, int64_t ld_dst)
{
    const int64_t total = n * p_pad;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t k = e / p_pad, j = e % p_pad;
        const bool ok = j < p;
        PB[k * ld_dst + 2 * j] = static_cast<D>(ok ? load_param<S>(Mp, k * ldB + j) : 0.0);
        PB[k * ld_dst + 2 * j + 1] = static_cast<D>(ok ? load_param<S>(Sp, k * ldB + j) : 0.0);
    }
}

__global__ void debug_philox_kernel(const uint32_t* ctr, const uint32_t* key, int64_t count, uint32_t* out)
{
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= count) return;
    const uint4 c = make_uint4(ctr[4 * e], ctr[4 * e + 1], ctr[4 * e + 2], ctr[4 * e + 3]);
    const uint4 w = philox4x32_10(c, make_uint2(key[2 * e], key[2 * e + 1]));
    out[4 * e] = w.x;
    out[4 * e + 1] = w.y;
    out[4 * e + 2] = w.z;
    out[4 * e + 3] = w.w;
}

__global__ void debug_indices_kernel(uint2 keyI, int l, uint64_t s, int64_t n, int64_t t0, int64_t count,
                                     int64_t* out)
{
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= count) return;
    const int64_t t = t0 + e;
    int64_t r0, r1;
    index_pair(keyI, level_sample_word(l, s), static_cast<uint32_t>(s), t >> 1, static_cast<uint64_t>(n), r0, r1);
    out[e] = (t & 1) ? r1 : r0;
}

__global__ void debug_indices_xi_kernel(uint2 keyI, int l, uint64_t s, int64_t n, int64_t t0, int64_t count,
                                        const double* Q, const double* q, const int* G, int64_t* out)
{
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= count) return;
    const int64_t t = t0 + e;
    uint64_t w0, w1;
    index_words(keyI, level_sample_word(l, s), static_cast<uint32_t>(s), t >> 1, w0, w1);
    out[e] = index_from_cdf((t & 1) ? w1 : w0, Q, q, G, n);
}

// q[k] of xi**: one thread per k, sums in index order with separate roundings (no contraction).
template <typename T>
__global__ void xi_weights_kernel(const T* __restrict__ PAB, int64_t ld, int64_t m, int64_t m_pad, int64_t n,
                                  int64_t p, double* q)
{
    const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const T* row = PAB + k * ld;
    double ea = 0.0, eb = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        const double mv = static_cast<double>(row[2 * i]), sv = static_cast<double>(row[2 * i + 1]);
        ea = __dadd_rn(ea, __dadd_rn(__dmul_rn(mv, mv), __dmul_rn(sv, sv)));
    }
    const T* rb = row + 2 * m_pad;
    for (int64_t j = 0; j < p; ++j) {
        const double mv = static_cast<double>(rb[2 * j]), sv = static_cast<double>(rb[2 * j + 1]);
        eb = __dadd_rn(eb, __dadd_rn(__dmul_rn(mv, mv), __dmul_rn(sv, sv)));
    }
    q[k] = __dsqrt_rn(__dmul_rn(ea, eb));
}

// Guide table of the cumulative law: G[b] = the smallest j with Q[j] > b Q[n-1] / n (a lower
// bound for every x in bucket b; exactness of the draw does not depend on it).
__global__ void xi_guide_kernel(const double* __restrict__ Q, int64_t n, int* G)
{
    const int64_t b = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const double thr = static_cast<double>(b) / static_cast<double>(n) * Q[n - 1];
    int64_t lo = 0, hi = n - 1;   // Q[n-1] > thr for b < n (up to rounding: clamped below)
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (Q[mid] > thr)
            hi = mid;
        else
            lo = mid + 1;
    }
    G[b] = static_cast<int>(lo);
}

// Q[k] = q[0] + ... + q[k]: one sequential pass (the order fixes every rounding).
__global__ void xi_scan_kernel(const double* __restrict__ q, int64_t n, double* Q)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double run = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        run = __dadd_rn(run, q[k]);
        Q[k] = run;
    }
}

template <typename T>
__global__ void debug_normals_kernel(uint2 key, int l, uint64_t s, int64_t k, int64_t row0, int64_t count,
                                     double* out)
{
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= count) return;
    const int64_t row = row0 + e;
    const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(row >> 2), static_cast<uint32_t>(k),
                                             static_cast<uint32_t>(s), level_sample_word(l, s)),
                                  key);
    T z[4];
    Normals<T>::four(w, z);
    out[e] = static_cast<double>(z[row & 3]);
}

inline unsigned blocks_for(int64_t n, int threads) { return static_cast<unsigned>((n + threads - 1) / threads); }

}  // namespace

cudaError_t launch_merge_partials(const void* partial_sum, bool partial_f64, const double* partial_q,
                                  int nchunks, int tiles, int64_t mp, double* level_sum, double* level_sumsq,
                                  cudaStream_t st)
{
    if (nchunks > kMaxMergeChunks) return cudaErrorInvalidValue;
    const unsigned g = blocks_for(mp, kMergeThreads);
    if (partial_f64)
        merge_sum_kernel<double><<<g, kMergeThreads, 0, st>>>(static_cast<const double*>(partial_sum), nchunks,
                                                              mp, level_sum);
    else
        merge_sum_kernel<float><<<g, kMergeThreads, 0, st>>>(static_cast<const float*>(partial_sum), nchunks,
                                                             mp, level_sum);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    merge_sumsq_kernel<<<1, kMergeThreads, 0, st>>>(partial_q, nchunks, tiles, level_sumsq);
    return cudaGetLastError();
}

cudaError_t launch_merge_batch(const MergeJob* jobs, const int* njobs_dev, cudaStream_t st)
{
    merge_batch_kernel<<<dim3(64, 256), kMergeThreads, 0, st>>>(jobs, njobs_dev);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const double* sum, const double* sumsq, LevelCounts counts, int first, int count,
                            int64_t mp, double* mean, double* M2, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    finalize_kernel<<<count, kMergeThreads, 0, st>>>(sum, sumsq, counts, first, mp, mean, M2);
    return cudaGetLastError();
}

cudaError_t launch_telescoping(const double* sum, LevelCounts counts, int levels, int64_t mp, double* yhat,
                               cudaStream_t st)
{
    telescoping_kernel<<<blocks_for(mp, kMergeThreads), kMergeThreads, 0, st>>>(sum, counts, levels, mp, yhat);
    return cudaGetLastError();
}

cudaError_t launch_layout_A(const void* M, const void* S, int src_dtype, int64_t ldA, int64_t m, int64_t n,
                            int64_t m_pad, void* PA, int64_t ld_dst, bool dst_f64, cudaStream_t st)
{
    dim3 block(32, 8);
    dim3 grid(static_cast<unsigned>((n + 31) / 32), static_cast<unsigned>((m_pad + 31) / 32));
    const bool src_f64 = src_dtype == MLMC_DTYPE_F64;
    if (src_f64 && dst_f64)
        layout_A_kernel<double, double><<<grid, block, 0, st>>>(M, S, ldA, m, n, m_pad, static_cast<double*>(PA), ld_dst);
    else if (src_f64)
        layout_A_kernel<double, float><<<grid, block, 0, st>>>(M, S, ldA, m, n, m_pad, static_cast<float*>(PA), ld_dst);
    else if (dst_f64)
        layout_A_kernel<float, double><<<grid, block, 0, st>>>(M, S, ldA, m, n, m_pad, static_cast<double*>(PA), ld_dst);
    else
        layout_A_kernel<float, float><<<grid, block, 0, st>>>(M, S, ldA, m, n, m_pad, static_cast<float*>(PA), ld_dst);
    return cudaGetLastError();
}

cudaError_t launch_layout_B(const void* Mp, const void* Sp, int src_dtype, int64_t ldB, int64_t n, int64_t p,
                            int64_t p_pad, void* PB, int64_t ld_dst, bool dst_f64, cudaStream_t st)
{
    const unsigned g = static_cast<unsigned>(std::min<int64_t>(blocks_for(n * p_pad, 256), 152 * 32));
    const bool src_f64 = src_dtype == MLMC_DTYPE_F64;
    if (src_f64 && dst_f64)
        layout_B_kernel<double, double><<<g, 256, 0, st>>>(Mp, Sp, ldB, n, p, p_pad, static_cast<double*>(PB), ld_dst);
    else if (src_f64)
        layout_B_kernel<double, float><<<g, 256, 0, st>>>(Mp, Sp, ldB, n, p, p_pad, static_cast<float*>(PB), ld_dst);
    else if (dst_f64)
        layout_B_kernel<float, double><<<g, 256, 0, st>>>(Mp, Sp, ldB, n, p, p_pad, static_cast<double*>(PB), ld_dst);
    else
        layout_B_kernel<float, float><<<g, 256, 0, st>>>(Mp, Sp, ldB, n, p, p_pad, static_cast<float*>(PB), ld_dst);
    return cudaGetLastError();
}

cudaError_t launch_debug_philox(const uint32_t* ctr, const uint32_t* key, int64_t count, uint32_t* out,
                                cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    debug_philox_kernel<<<blocks_for(count, 256), 256, 0, st>>>(ctr, key, count, out);
    return cudaGetLastError();
}

cudaError_t launch_debug_indices(uint2 keyI, int l, uint64_t s, int64_t n, int64_t t0, int64_t count, int64_t* out,
                                 cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    debug_indices_kernel<<<blocks_for(count, 256), 256, 0, st>>>(keyI, l, s, n, t0, count, out);
    return cudaGetLastError();
}

cudaError_t launch_debug_indices_xi(uint2 keyI, int l, uint64_t s, int64_t n, int64_t t0, int64_t count,
                                    const double* Q, const double* q, const int* G, int64_t* out, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    debug_indices_xi_kernel<<<static_cast<unsigned>((count + 255) / 256), 256, 0, st>>>(keyI, l, s, n, t0, count, Q, q,
                                                                                         G, out);
    return cudaGetLastError();
}

cudaError_t launch_xi_optimal(const void* PAB, bool f64, int64_t ld, int64_t m, int64_t m_pad, int64_t n,
                              int64_t p, double* q, double* Q, int* G, cudaStream_t st)
{
    const unsigned blocks = static_cast<unsigned>((n + 255) / 256);
    if (f64)
        xi_weights_kernel<double><<<blocks, 256, 0, st>>>(static_cast<const double*>(PAB), ld, m, m_pad, n, p, q);
    else
        xi_weights_kernel<float><<<blocks, 256, 0, st>>>(static_cast<const float*>(PAB), ld, m, m_pad, n, p, q);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    xi_scan_kernel<<<1, 1, 0, st>>>(q, n, Q);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    xi_guide_kernel<<<blocks, 256, 0, st>>>(Q, n, G);
    return cudaGetLastError();
}

cudaError_t launch_debug_normals(uint2 key, bool f64, int l, uint64_t s, int64_t k, int64_t row0, int64_t count,
                                 double* out, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    if (f64)
        debug_normals_kernel<double><<<blocks_for(count, 256), 256, 0, st>>>(key, l, s, k, row0, count, out);
    else
        debug_normals_kernel<float><<<blocks_for(count, 256), 256, 0, st>>>(key, l, s, k, row0, count, out);
    return cudaGetLastError();
}

}  // namespace mlmc
