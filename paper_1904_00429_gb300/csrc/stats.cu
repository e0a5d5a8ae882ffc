// stats.cu -- per-level statistics (Eq. hatYl, Remark 3.6), the telescoping
// sum (Eq. hatY), the parameter layout copy and the verification kernels.
//
// A level's state is (N, per-entry FP64 sum of D, FP64 M2), M2 = sum_s ||D_s - mean||_F^2.
// The level kernels hand over, per chunk of samples, the chunk's sum of D and its own M2
// (accumulated sample by sample with Welford's update).  The merge folds the chunks into the
// level strictly in chunk order with Chan's pairwise update
//     M2 <- M2 + M2_c + N n_c / (N + n_c) ||mean_c - mean||_F^2,   sum <- sum + sum_c,
// one thread per entry for the sums (blocks of kMergeGroup entries, so that the few thousand
// entries of a small problem still spread over most SMs), so the state is a deterministic
// function of the samples folded in.  Y_l = sum / N and V_l = M2 / (N - 1).
#include <algorithm>

#include <cuda_runtime.h>

#include "internal.h"
#include "rng.cuh"

namespace mlmc {
namespace {

constexpr int kMergeThreads = 256;
// kMergeGroup (internal.h) entries per block of the chunk folds and per share of the
// between-chunk term: the fold is a chain over the chunks in order, so its parallelism is the
// number of entries.
constexpr int kMaxMergeChunks = 4096;

// Per-chunk coefficients of Chan's update, the same for every entry: computed once per block
// and tile of chunks into shared memory.  N_c, the samples before chunk c, has a closed form
// (n_before plus the ids of the run before the chunk), so the chunks of a tile are independent.
constexpr int kCoefTile = 128;

template <typename T>
struct ChanCoef {
    T nc;        // n_c
    T inv_nc;    // 1 / n_c
    T inv_next;  // 1 / (N_c + n_c)
    T w;         // N_c n_c / (N_c + n_c)
};

template <typename T>
__device__ __forceinline__ void chan_coefs(const ChunkRun& run, int c0, int cnt, ChanCoef<T>* coef)
{
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const int c = c0 + i;
        const uint64_t lo = (run.chunk0 + static_cast<uint64_t>(c)) * run.chunk;
        const uint64_t before = run.n_before + ((run.s_begin > lo ? run.s_begin : lo) - run.s_begin);
        const uint64_t nc = chunk_count(run, c);
        // in T: FP32 partials take FP32 coefficients (FP64 runs at 1/64 of the FP32 rate here)
        const T nb = static_cast<T>(before), n = static_cast<T>(nc);
        const T inv_next = T(1) / (nb + n);
        coef[i] = ChanCoef<T>{n, T(1) / n, inv_next, nb * n * inv_next};
    }
}

// Fold the chunk partials of entry e into its FP64 level sum, in chunk order, and return the
// entry's share of Chan's between-chunk term, sum_c N_c n_c / (N_c + n_c) (mu_c - mu_{<c})^2
// (N_c the samples folded before chunk c, mu_c the chunk's mean and mu_{<c} the running mean).
// The means are carried in the partials' precision T as offsets from a shift K (the level's
// mean when the run starts, else the first chunk's mean): t = sum_c - n_c K is one fused
// rounding of a small number and r = sum_{<c} - N_c K stays small, so a mean far above the
// spread cancels inside the shift instead of inside the squares.  Every thread of the block
// calls this (the coefficient tiles are built together); `active` selects the entry's work.
template <typename T>
__device__ __forceinline__ double chan_fold(const T* __restrict__ partial, int64_t mp, int64_t e, bool active,
                                            const ChunkRun& run, double* __restrict__ sum_e, ChanCoef<T>* coef)
{
    double acc = active ? *sum_e : 0.0;
    double chan = 0.0;
    T K = T(0), r = T(0);
    int c = 0;
    if (run.n_before > 0) {
        const double N = static_cast<double>(run.n_before);
        K = static_cast<T>(acc / N);
        r = static_cast<T>(acc - N * static_cast<double>(K));
    } else if (active) {
        const T v = partial[e];
        const T nc = static_cast<T>(chunk_count(run, 0));
        K = v / nc;
        r = fma(-nc, K, v);
        acc += static_cast<double>(v);
    }
    if (run.n_before == 0) c = 1;
    T inv_N = T(0);
    for (int t0 = c; t0 < run.nchunks; t0 += kCoefTile) {
        const int cnt = min(kCoefTile, run.nchunks - t0);
        __syncthreads();   // the previous tile's coefficients are no longer read
        chan_coefs<T>(run, t0, cnt, coef);
        __syncthreads();
        if (t0 == c) {
            const uint64_t lo = (run.chunk0 + static_cast<uint64_t>(c)) * run.chunk;
            const uint64_t before = run.n_before + ((run.s_begin > lo ? run.s_begin : lo) - run.s_begin);
            inv_N = T(1) / static_cast<T>(before);
        }
        if (!active) continue;
        // kLoads independent loads in flight, then the folds in chunk order
        constexpr int kLoads = 16;
        for (int i = 0; i < cnt; i += kLoads) {
            const int k = min(kLoads, cnt - i);
            T v[kLoads];
#pragma unroll
            for (int u = 0; u < kLoads; ++u)
                v[u] = u < k ? partial[static_cast<int64_t>(t0 + i + u) * mp + e] : T(0);
            T grp = T(0);
#pragma unroll
            for (int u = 0; u < kLoads; ++u) {
                if (u < k) {
                    const ChanCoef<T> cf = coef[i + u];
                    const T t = fma(-cf.nc, K, v[u]);            // sum_c - n_c K
                    const T d = t * cf.inv_nc - r * inv_N;       // mu_c - mu_{<c}
                    grp = fma(cf.w * d, d, grp);
                    r += t;
                    acc += static_cast<double>(v[u]);
                    inv_N = cf.inv_next;
                }
            }
            chan += static_cast<double>(grp);
        }
    }
    if (active) *sum_e = acc;
    return chan;
}

// Sum of `v` over a block of kThreads threads in a fixed shape; the result is valid in
// thread 0.  `red` holds kThreads / 32 doubles.
template <int kThreads>
__device__ __forceinline__ double block_sum(double v, double* red)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();   // red may still be read by an earlier call
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    return t;
}

// One thread per entry, one block per group of kMergeGroup entries: the sums, and each
// group's share of the between-chunk term in chan_out[group].
template <typename T>
__global__ void __launch_bounds__(kMergeGroup)
merge_chan_kernel(const T* __restrict__ partial, const ChunkRun run, int64_t mp, double* level_sum,
                  double* chan_out)
{
    __shared__ double red[kMergeGroup / 32];
    __shared__ ChanCoef<T> coef[kCoefTile];
    const int64_t e = static_cast<int64_t>(blockIdx.x) * kMergeGroup + threadIdx.x;
    const double chan = chan_fold<T>(partial, mp, e, e < mp, run, level_sum + e, coef);
    const double t = block_sum<kMergeGroup>(chan, red);
    if (threadIdx.x == 0) chan_out[blockIdx.x] = t;
}

// M2 <- M2 + sum_c M2_c (chunk order; M2_c the sum over the chunk's tiles) + the sum of the
// groups' between-chunk terms (a fixed shape over the groups).  One block of kMergeThreads.
// The chunk order keeps a run split into two calls, the first of one chunk, bit-identical to
// one call (the first call's between-chunk terms are zero); other splits move the launches'
// between-chunk sums by rounding.
__device__ __forceinline__ void fold_m2(const double* __restrict__ partial_q, int nchunks, int tiles,
                                        const double* __restrict__ chan, int groups, double* level_M2,
                                        double* chunk_q, double* red)
{
    for (int c = threadIdx.x; c < nchunks; c += blockDim.x) {
        double t = 0.0;
        for (int x = 0; x < tiles; ++x) t += partial_q[static_cast<int64_t>(c) * tiles + x];
        chunk_q[c] = t;
    }
    double cg = 0.0;
    for (int g = threadIdx.x; g < groups; g += blockDim.x) cg += chan[g];
    const double chan_sum = block_sum<kMergeThreads>(cg, red);   // ends with a block barrier
    if (threadIdx.x == 0) {
        double acc = *level_M2;
        for (int c = 0; c < nchunks; ++c) acc += chunk_q[c];
        *level_M2 = acc + chan_sum;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kMergeThreads)
merge_m2_kernel(const double* __restrict__ partial_q, int nchunks, int tiles, const double* __restrict__ chan,
                int groups, double* level_M2)
{
    __shared__ double chunk_q[kMaxMergeChunks];
    __shared__ double red[kMergeThreads / 32];
    fold_m2(partial_q, nchunks, tiles, chan, groups, level_M2, chunk_q, red);
}

// Batched merge: the jobs of one wave (count read from the device), each folded into its
// level's FP64 state exactly as merge_chan_kernel / merge_m2_kernel do (the same per-entry fold,
// the same groups of kMergeGroup entries, the same orders), so a batched call and the same
// ranges run one by one give the same bits.  The grid is fixed (grid-stride over jobs in y and
// entry groups in x) so that a captured graph stays valid when the wave's contents change; a
// wave holds at most one job per (problem, level).
__global__ void __launch_bounds__(kMergeGroup) merge_batch_kernel(const MergeJob* __restrict__ jobs,
                                                                  const int* __restrict__ njobs_dev)
{
    __shared__ double red[kMergeGroup / 32];
    __shared__ ChanCoef<float> coef[kCoefTile];
    const int njobs = *njobs_dev;
    for (int j = blockIdx.y; j < njobs; j += gridDim.y) {
        const MergeJob jb = jobs[j];
        const int64_t groups = (jb.mp + kMergeGroup - 1) / kMergeGroup;
        for (int64_t g = blockIdx.x; g < groups; g += gridDim.x) {
            const int64_t e = g * kMergeGroup + threadIdx.x;
            const double chan = chan_fold<float>(jb.partial, jb.mp, e, e < jb.mp, jb.run, jb.sum + e, coef);
            const double t = block_sum<kMergeGroup>(chan, red);
            if (threadIdx.x == 0) jb.chan[g] = t;
        }
    }
}

__global__ void __launch_bounds__(kMergeThreads)
merge_batch_m2_kernel(const MergeJob* __restrict__ jobs, const int* __restrict__ njobs_dev)
{
    __shared__ double chunk_q[kMaxMergeChunks];
    __shared__ double red[kMergeThreads / 32];
    const int njobs = *njobs_dev;
    for (int j = blockIdx.x; j < njobs; j += gridDim.x) {
        const MergeJob jb = jobs[j];
        const int groups = static_cast<int>((jb.mp + kMergeGroup - 1) / kMergeGroup);
        fold_m2(jb.partial_q, jb.run.nchunks, jb.tiles, jb.chan, groups, jb.M2, chunk_q, red);
    }
}

// mean = sum / N for `count` levels laid out back to back.
__global__ void finalize_kernel(const double* __restrict__ sum, const LevelCounts counts, int first, int64_t mp,
                                double* mean)
{
    const int lvl = blockIdx.y;
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= mp) return;
    const uint64_t n = counts.v[first + lvl];
    const double inv = n > 0 ? 1.0 / static_cast<double>(n) : 0.0;
    mean[static_cast<int64_t>(lvl) * mp + e] = sum[static_cast<int64_t>(lvl) * mp + e] * inv;
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

int merge_groups(int64_t mp) { return static_cast<int>((mp + kMergeGroup - 1) / kMergeGroup); }

cudaError_t launch_merge_partials(const void* partial_sum, bool partial_f64, const double* partial_q, int tiles,
                                  int64_t mp, const ChunkRun& run, double* level_sum, double* level_M2,
                                  double* chan_scratch, cudaStream_t st)
{
    if (run.nchunks < 1 || run.nchunks > kMaxMergeChunks) return cudaErrorInvalidValue;
    const unsigned g = static_cast<unsigned>(merge_groups(mp));
    if (partial_f64)
        merge_chan_kernel<double><<<g, kMergeGroup, 0, st>>>(static_cast<const double*>(partial_sum), run, mp,
                                                               level_sum, chan_scratch);
    else
        merge_chan_kernel<float><<<g, kMergeGroup, 0, st>>>(static_cast<const float*>(partial_sum), run, mp,
                                                              level_sum, chan_scratch);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    merge_m2_kernel<<<1, kMergeThreads, 0, st>>>(partial_q, run.nchunks, tiles, chan_scratch, static_cast<int>(g),
                                                level_M2);
    return cudaGetLastError();
}

cudaError_t launch_merge_batch(const MergeJob* jobs, const int* njobs_dev, cudaStream_t st)
{
    merge_batch_kernel<<<dim3(128, 256), kMergeGroup, 0, st>>>(jobs, njobs_dev);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    merge_batch_m2_kernel<<<256, kMergeThreads, 0, st>>>(jobs, njobs_dev);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const double* sum, LevelCounts counts, int first, int count, int64_t mp, double* mean,
                            cudaStream_t st)
{
    if (count <= 0 || mp <= 0) return cudaSuccess;
    finalize_kernel<<<dim3(blocks_for(mp, kMergeThreads), static_cast<unsigned>(count)), kMergeThreads, 0, st>>>(
        sum, counts, first, mp, mean);
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
