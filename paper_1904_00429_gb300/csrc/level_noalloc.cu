// level_noalloc.cu -- level statistics without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while a stream is being
// captured into a CUDA graph, plugins of inference runtimes whose enqueue step
// must not allocate, and applications that hand all device memory to their own
// pool at start-up.  mlmc_level_stats_noalloc serves them: it reads the
// caller's parameter matrices in place (row-major, no sample-major copy),
// writes the caller's output buffers, and keeps its chunk partials in a
// fixed, file-scope device array instead of memory it would have to allocate.
//
// The array below is part of the library image: every GPU that loads the
// library holds it (kNoallocScratchBytes) until the process exits, whether or
// not this entry point is called.  All calls share it, so calls whose work
// overlaps on the GPU (other streams, other threads) race on it; the caller
// must order them (one stream, or events).  Host code cannot use the array's
// name as a device address: the address is fetched once per device with
// cudaGetSymbolAddress (with that device current) on the first call made on
// that device, so make that first call before any stream capture begins.  The
// address is kept for the life of the process: after cudaDeviceReset (or any
// other teardown of the device's primary context) it is stale, and the entry
// point must not be called again in that process.
//
// The arithmetic is the one of the plan's CUDA-core level kernel: the same
// draws, the same fused weighted rank-c_l update and the same chunk-ordered
// fold, so the results equal those of mlmc_level_stats up to the order in
// which parameters are loaded.
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include <cuda_runtime.h>

#include "internal.h"
#include "mlmc.h"
#include "rng.cuh"

namespace mlmc {
namespace {

constexpr size_t kNoallocScratchBytes = size_t(4) << 20;  // 4 MiB per device
constexpr int kNoallocMaxDevices = 64;
constexpr int kNoallocMaxChunks = 4096;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_noalloc_mutex;
void* g_noalloc_scratch_ptr[kNoallocMaxDevices] = {};

struct RowMajorParams {
    const void* M;
    const void* S;
    int64_t ldA;
    const void* Mp;
    const void* Sp;
    int64_t ldB;
};

// Same structure as the plan's level kernel (64 x 64 output tile, 32 slots per
// step, 4 x 4 register tile per thread, chunk partials per CTA); parameters are
// loaded from the caller's row-major matrices.
template <typename T>
__global__ void __launch_bounds__(256) level_rowmajor_kernel(const LevelParams prm, const RowMajorParams src)
{
    constexpr int TM = 64, TP = 64, TK = 32, RM = 4, RP = 4;
    constexpr int NT = (TM / RM) * (TP / RP);
    constexpr int TXN = TP / RP;

    __shared__ __align__(16) T As[TK][TM];
    __shared__ __align__(16) T Bs[TK][TP];
    __shared__ int idx_s[TK];
    __shared__ T w_s[TK];
    __shared__ double red_s[NT / 32];

    const int tid = threadIdx.x;
    const int tile = blockIdx.x;
    const int tm0 = (tile / prm.tiles_p) * TM;
    const int tp0 = (tile % prm.tiles_p) * TP;
    const int tx = tid % TXN;
    const int ty = tid / TXN;
    const uint64_t chunk = prm.chunk0 + blockIdx.y;
    const uint64_t sa = max(prm.s_begin, chunk * kChunk);
    const uint64_t sb = min(prm.s_end, (chunk + 1) * kChunk);
    const T* M = static_cast<const T*>(src.M);
    const T* S = static_cast<const T*>(src.S);
    const T* Mp = static_cast<const T*>(src.Mp);
    const T* Sp = static_cast<const T*>(src.Sp);
    const T wf = static_cast<T>(prm.w_fine);
    const T wc = static_cast<T>(prm.w_coarse);

    T sum[RM][RP];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RP; ++j) sum[i][j] = T(0);
    T qw = T(0);   // the chunk's M2 (Welford terms)

    for (uint64_t s = sa; s < sb; ++s) {
        const uint32_t lsw = level_sample_word(prm.l, s);
        const uint32_t s_lo = static_cast<uint32_t>(s);
        T acc[RM][RP];
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
            for (int j = 0; j < RP; ++j) acc[i][j] = T(0);
        for (int k0 = 0; k0 < prm.c; k0 += TK) {
            for (int h = tid; h < TK / 2; h += NT) {
                const int t = k0 + 2 * h;
                if (t < prm.c) {
                    int64_t r0, r1;
                    index_pair(prm.keyI, lsw, s_lo, t >> 1, static_cast<uint64_t>(prm.n), r0, r1);
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int te = t + e;
                        const bool valid = te < prm.c;
                        const bool coarse = prm.l > 0 && (te % prm.R) == prm.R - 1;
                        idx_s[2 * h + e] = valid ? static_cast<int>(e ? r1 : r0) : -1;
                        w_s[2 * h + e] = valid ? (coarse ? wc : wf) : T(0);
                    }
                } else {
                    idx_s[2 * h] = idx_s[2 * h + 1] = -1;
                    w_s[2 * h] = w_s[2 * h + 1] = T(0);
                }
            }
            __syncthreads();
            for (int it = tid; it < TK * (TM / 4); it += NT) {
                const int tt = it / (TM / 4);
                const int q4 = it % (TM / 4);
                const int i = tm0 + 4 * q4;
                const int k = idx_s[tt];
                T a[4] = {T(0), T(0), T(0), T(0)};
                if (k >= 0 && i < prm.m) {
                    const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(i >> 2), static_cast<uint32_t>(k),
                                                             s_lo, lsw),
                                                  prm.keyA);
                    T z[4];
                    Normals<T>::four(w, z);
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        if (i + r < prm.m) {
                            const int64_t off = static_cast<int64_t>(i + r) * src.ldA + k;
                            a[r] = fma(S[off], z[r], M[off]);
                        }
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) As[tt][4 * q4 + r] = a[r];
            }
            for (int it = tid; it < TK * (TP / 4); it += NT) {
                const int tt = it / (TP / 4);
                const int q4 = it % (TP / 4);
                const int j = tp0 + 4 * q4;
                const int k = idx_s[tt];
                T b[4] = {T(0), T(0), T(0), T(0)};
                if (k >= 0 && j < prm.p) {
                    const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(j >> 2), static_cast<uint32_t>(k),
                                                             s_lo, lsw),
                                                  prm.keyB);
                    T z[4];
                    Normals<T>::four(w, z);
                    const T wt = w_s[tt];
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        if (j + r < prm.p) {
                            const int64_t off = static_cast<int64_t>(k) * src.ldB + j + r;
                            b[r] = wt * fma(Sp[off], z[r], Mp[off]);
                        }
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) Bs[tt][4 * q4 + r] = b[r];
            }
            __syncthreads();
            const int kt = min(TK, prm.c - k0);
            for (int tt = 0; tt < kt; ++tt) {
                T av[RM], bv[RP];
#pragma unroll
                for (int i = 0; i < RM; ++i) av[i] = As[tt][ty * RM + i];
#pragma unroll
                for (int j = 0; j < RP; ++j) bv[j] = Bs[tt][tx * RP + j];
#pragma unroll
                for (int i = 0; i < RM; ++i)
#pragma unroll
                    for (int j = 0; j < RP; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
            }
            __syncthreads();
        }
        // Welford's update of the chunk's M2, as in the plan's level kernel
        const int kprev = static_cast<int>(s - sa);
        if (kprev > 0) {
            // in T (FP64 runs at 1/64 of the FP32 rate on this GPU: FP32 plans stay in FP32)
            const T kf = static_cast<T>(kprev);
            T qs = T(0);
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < RP; ++j) {
                    const T dk = fma(kf, acc[i][j], -sum[i][j]);
                    qs = fma(dk, dk, qs);
                }
            qw = fma(qs, T(1) / static_cast<T>(kprev * (kprev + 1)), qw);
        }
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
            for (int j = 0; j < RP; ++j) sum[i][j] += acc[i][j];
    }
    T* out = static_cast<T*>(prm.partial_sum) + static_cast<int64_t>(blockIdx.y) * prm.m * prm.p;
#pragma unroll
    for (int i = 0; i < RM; ++i) {
        const int gi = tm0 + ty * RM + i;
        if (gi >= prm.m) continue;
#pragma unroll
        for (int j = 0; j < RP; ++j) {
            const int gj = tp0 + tx * RP + j;
            if (gj < prm.p) out[static_cast<int64_t>(gi) * prm.p + gj] = sum[i][j];
        }
    }
    double q = static_cast<double>(qw);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) q += __shfl_xor_sync(0xffffffffu, q, off);
    if ((tid & 31) == 0) red_s[tid >> 5] = q;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < NT / 32; ++w) t += red_s[w];
        prm.partial_q[static_cast<int64_t>(blockIdx.y) * prm.tiles_m * prm.tiles_p + tile] = t;
    }
}

// Device address of the scratch array on the current device (set up once per device).
cudaError_t scratch_address(void** out)
{
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev < 0 || dev >= kNoallocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_scratch_ptr[dev]) {
        void* p = nullptr;
        err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (err != cudaSuccess) return err;
        g_noalloc_scratch_ptr[dev] = p;
    }
    *out = g_noalloc_scratch_ptr[dev];
    return cudaSuccess;
}

mlmc_status noalloc_fail(mlmc_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return report_error(st, buf);
}

}  // namespace
}  // namespace mlmc

using namespace mlmc;

extern "C" mlmc_status mlmc_level_stats_noalloc(const mlmc_problem* problem, const mlmc_options* options,
                                                 int32_t level, uint64_t sample_begin, uint64_t count,
                                                 double* sum_dev, double* M2_dev, void* stream)
{
    if (!problem || !options || !sum_dev || !M2_dev) return noalloc_fail(MLMC_ERR_INVALID_ARG, "null argument");
    const mlmc_problem& pr = *problem;
    const mlmc_options& o = *options;
    const bool f64 = o.precision == MLMC_FP64;
    if (o.precision != MLMC_FP64 && o.precision != MLMC_FP32)
        return noalloc_fail(MLMC_ERR_UNSUPPORTED, "no-alloc level statistics support FP64 and FP32 only");
    if ((f64 && pr.dtype != MLMC_DTYPE_F64) || (!f64 && pr.dtype != MLMC_DTYPE_F32))
        return noalloc_fail(MLMC_ERR_UNSUPPORTED, "parameter dtype must match the precision (F64/FP64, F32/FP32)");
    if (o.c0 < 1 || o.ratio < 2) return noalloc_fail(MLMC_ERR_INVALID_ARG, "c0 must be >= 1 and ratio >= 2");
    if (o.f != MLMC_F_IDENTITY) return noalloc_fail(MLMC_ERR_UNSUPPORTED, "the no-alloc entry point evaluates f = x only");
    if (o.sampling != MLMC_XI_UNIFORM)
        return noalloc_fail(MLMC_ERR_UNSUPPORTED, "the no-alloc entry point draws indices uniformly only");
    if (pr.m < 1 || pr.p < 1 || pr.m > 65536 || pr.p > 65536 || pr.n < 1 || pr.n >= (int64_t(1) << 31))
        return noalloc_fail(MLMC_ERR_INVALID_ARG, "m, p must be in [1, 65536] and n in [1, 2^31)");
    if (pr.ldA < pr.n || pr.ldB < pr.p) return noalloc_fail(MLMC_ERR_INVALID_ARG, "leading dimension too small");
    if (!pr.M_dev || !pr.S_dev || !pr.Mp_dev || !pr.Sp_dev)
        return noalloc_fail(MLMC_ERR_INVALID_ARG, "null parameter pointer");
    if (level < 0 || level >= MLMC_MAX_LEVELS) return noalloc_fail(MLMC_ERR_INVALID_ARG, "level out of range");
    int64_t c = o.c0;
    for (int l = 0; l < level; ++l) {
        c *= o.ratio;
        if (c > (int64_t(1) << 30)) return noalloc_fail(MLMC_ERR_INVALID_ARG, "c_l exceeds 2^30");
    }
    if (sample_begin + count < sample_begin || sample_begin + count > (uint64_t(1) << 56))
        return noalloc_fail(MLMC_ERR_INVALID_ARG, "sample ids must stay below 2^56");
    const int tiles_m = int((pr.m + 63) / 64), tiles_p = int((pr.p + 63) / 64);
    const size_t elem = f64 ? 8 : 4;
    const int64_t mp = pr.m * pr.p;
    const size_t tiles = size_t(tiles_m) * size_t(tiles_p);
    // scratch of `ch` chunks: the merge's between-chunk terms (one double per kMergeGroup entries), the
    // chunks' M2 per tile, then their partial sums, each part starting on a 256-byte boundary
    const size_t chan_bytes = (size_t(merge_groups(mp)) * 8 + 255) / 256 * 256;
    auto need = [&](size_t ch) { return chan_bytes + (ch * tiles * 8 + 255) / 256 * 256 + ch * size_t(mp) * elem; };
    size_t chunks = kNoallocScratchBytes / (size_t(mp) * elem + tiles * 8);
    if (chunks > size_t(kNoallocMaxChunks)) chunks = size_t(kNoallocMaxChunks);
    while (chunks > 0 && need(chunks) > kNoallocScratchBytes) --chunks;
    if (chunks == 0)
        return noalloc_fail(MLMC_ERR_INVALID_ARG,
                            "m*p = %lld too large for the %zu-byte no-alloc scratch (needs m*p*%zu + 8*tiles + "
                            "8*ceil(m*p/64), each rounded up to 256, <= %zu bytes)",
                            (long long)mp, kNoallocScratchBytes, elem, kNoallocScratchBytes);
    const size_t q_bytes = (chunks * tiles * 8 + 255) / 256 * 256;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* scratch = nullptr;
    cudaError_t err = scratch_address(&scratch);
    if (err != cudaSuccess) return noalloc_fail(MLMC_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(err));
    // outputs are written, not accumulated: the in-order fold starts from zero
    err = cudaMemsetAsync(sum_dev, 0, sizeof(double) * size_t(mp), st);
    if (err == cudaSuccess) err = cudaMemsetAsync(M2_dev, 0, sizeof(double), st);
    if (err != cudaSuccess) return noalloc_fail(MLMC_ERR_CUDA, "clearing outputs: %s", cudaGetErrorString(err));
    if (count == 0) return MLMC_OK;

    // scratch layout: the merge's between-chunk terms, the chunks' M2, then their partial sums
    double* chan = static_cast<double*>(scratch);
    double* partial_q = reinterpret_cast<double*>(static_cast<unsigned char*>(scratch) + chan_bytes);
    void* partial_sum = static_cast<unsigned char*>(scratch) + chan_bytes + q_bytes;

    LevelParams prm{};
    prm.n = pr.n;
    prm.m = int(pr.m);
    prm.p = int(pr.p);
    prm.l = level;
    prm.c = int(c);
    prm.R = o.ratio;
    prm.w_fine = double(pr.n) / double(c);
    prm.w_coarse = level > 0 ? double(pr.n) / double(c) - double(pr.n) / double(c / o.ratio) : 0.0;
    prm.keyA = make_uint2(pr.seed_A, pr.problem_id);
    prm.keyB = make_uint2(pr.seed_B, pr.problem_id);
    prm.keyI = make_uint2(pr.seed_idx, pr.problem_id);
    prm.tiles_m = tiles_m;
    prm.tiles_p = tiles_p;
    prm.chunk = kChunk;
    prm.ldPA = pr.ldA;
    prm.ldPB = pr.ldB;
    prm.partial_sum = partial_sum;
    prm.partial_q = partial_q;
    const RowMajorParams src{pr.M_dev, pr.S_dev, pr.ldA, pr.Mp_dev, pr.Sp_dev, pr.ldB};
    const uint64_t s_end = sample_begin + count;
    const uint64_t chunk_first = sample_begin / kChunk;
    const uint64_t chunk_last = (s_end - 1) / kChunk;
    for (uint64_t cb = chunk_first; cb <= chunk_last; cb += uint64_t(chunks)) {
        const int nb = int((chunk_last - cb + 1) < uint64_t(chunks) ? (chunk_last - cb + 1) : uint64_t(chunks));
        prm.chunk0 = cb;
        prm.nchunks = nb;
        prm.s_begin = sample_begin > cb * kChunk ? sample_begin : cb * kChunk;
        prm.s_end = s_end < (cb + nb) * kChunk ? s_end : (cb + nb) * kChunk;
        dim3 grid(unsigned(tiles_m * tiles_p), unsigned(nb));
        if (f64)
            level_rowmajor_kernel<double><<<grid, 256, 0, st>>>(prm, src);
        else
            level_rowmajor_kernel<float><<<grid, 256, 0, st>>>(prm, src);
        err = cudaGetLastError();
        const ChunkRun run{prm.s_begin, prm.s_end, cb, uint64_t(kChunk), prm.s_begin - sample_begin, nb};
        if (err == cudaSuccess)
            err = launch_merge_partials(partial_sum, f64, partial_q, tiles_m * tiles_p, mp, run, sum_dev, M2_dev,
                                        chan, st);
        if (err != cudaSuccess) return noalloc_fail(MLMC_ERR_CUDA, "no-alloc level launch: %s", cudaGetErrorString(err));
    }
    return MLMC_OK;
}
