// adjoint.cu -- reparameterised gradient of <G, Yhat> with respect to M, S, M', S'.
//
// Yhat = sum_l (1/N_l) sum_{s < N_l} D_{l,s} with D = sum_t w_t a_t b_t^T, a_t = A[:, r_t],
// b_t = B[r_t, :] (Alg. 1, Eq. hatYl, Eq. hatY).  With the draws held fixed (A = M + S o Z,
// B = M' + S' o Z'), every sampled product contributes, for omega = w_t / N_l and k = r_t,
//     dM[:, k]  += omega G b_t            dS[:, k]  += omega z_t o (G b_t)
//     dM'[k, :] += omega G^T a_t          dS'[k, :] += omega z'_t o (G^T a_t)
// where z_t = Z[:, k] and z'_t = Z'[k, :] of sample (l, s).  The contributions to one k are
// gathered by a counting sort of all (l, s, t) records on k, and each segment is reduced by one
// CTA that regenerates a_t, b_t and their normals from Philox (nothing of the forward is
// stored), contracts them with G on the CUDA cores and writes the four gradient slices of k
// once per batch of records: no atomics on the gradients.  Records within a segment are summed
// in FP64 in the order the sort left them (the counting sort's placement is not ordered within
// a segment), so repeated runs agree to FP64 rounding of the FP32 (or FP64) contractions.
//
// Record layout (64 bits): bits 0-4 level, bit 5 "slot is also coarse", bits 6-63 sample id.
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "rng.cuh"

namespace mlmc {
namespace {

constexpr int kScanBlock = 1024;   // entries per block of the prefix sum
constexpr int kAdjThreads = 256;
constexpr int kAdjChunk = 16;      // contributions per smem chunk in the segment kernel

__device__ __forceinline__ uint64_t pack_record(int l, bool coarse, uint64_t s)
{
    return static_cast<uint64_t>(l & 31) | (static_cast<uint64_t>(coarse ? 1 : 0) << 5) | (s << 6);
}

// --- 1. enumerate records: histogram pass (count) or placement pass (scatter) ----------------
// Work unit: one Philox block = two consecutive slots of one sample of one level.
__global__ void enumerate_kernel(AdjLevels lv, uint2 keyI, int64_t n, int R, int* __restrict__ counts,
                                 int64_t* __restrict__ cursor, uint64_t* __restrict__ records)
{
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < lv.total_pairs;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        int q = 0;
        while (q + 1 < lv.count && e >= lv.pair_begin[q + 1]) ++q;
        const int l = lv.lev[q];
        const int64_t c = lv.c[q];
        const int64_t within = e - lv.pair_begin[q];
        const int64_t pairs_per_sample = (c + 1) / 2;
        const uint64_t s = lv.s0[q] + static_cast<uint64_t>(within / pairs_per_sample);
        const int64_t tp = within % pairs_per_sample;
        int64_t r0, r1;
        index_pair(keyI, level_sample_word(l, s), static_cast<uint32_t>(s), tp, static_cast<uint64_t>(n), r0, r1);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t t = 2 * tp + h;
            if (t >= c) break;
            const int64_t k = h ? r1 : r0;
            if (counts) {
                atomicAdd(counts + k, 1);
            } else {
                const bool coarse = l > 0 && (t % R) == R - 1;
                const int64_t pos = static_cast<int64_t>(
                    atomicAdd(reinterpret_cast<unsigned long long*>(cursor + k), 1ull));
                records[pos] = pack_record(l, coarse, s);
            }
        }
    }
}

// --- 2. exclusive prefix sum of int counts into int64 offsets (three levels of blocks) --------
__global__ void scan_block_kernel(const int* __restrict__ in, int64_t count, int64_t* __restrict__ out,
                                  int64_t* __restrict__ block_sums)
{
    __shared__ int64_t buf[kScanBlock];
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanBlock;
    for (int i = threadIdx.x; i < kScanBlock; i += blockDim.x)
        buf[i] = base + i < count ? static_cast<int64_t>(in[base + i]) : 0;
    __syncthreads();
    // Hillis-Steele on the block (kScanBlock is small; clarity over work efficiency)
    for (int off = 1; off < kScanBlock; off <<= 1) {
        int64_t tmp[kScanBlock / 256];
        for (int q = 0; q < kScanBlock / 256; ++q) {
            const int i = threadIdx.x + q * 256;
            tmp[q] = i >= off ? buf[i - off] : 0;
        }
        __syncthreads();
        for (int q = 0; q < kScanBlock / 256; ++q) buf[threadIdx.x + q * 256] += tmp[q];
        __syncthreads();
    }
    for (int i = threadIdx.x; i < kScanBlock; i += blockDim.x)
        if (base + i < count) out[base + i] = buf[i] - (base + i < count ? static_cast<int64_t>(in[base + i]) : 0);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = buf[kScanBlock - 1];
}

__global__ void scan_i64_block_kernel(const int64_t* __restrict__ in, int64_t count, int64_t* __restrict__ out,
                                      int64_t* __restrict__ block_sums)
{
    __shared__ int64_t buf[kScanBlock];
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanBlock;
    for (int i = threadIdx.x; i < kScanBlock; i += blockDim.x) buf[i] = base + i < count ? in[base + i] : 0;
    __syncthreads();
    for (int off = 1; off < kScanBlock; off <<= 1) {
        int64_t tmp[kScanBlock / 256];
        for (int q = 0; q < kScanBlock / 256; ++q) {
            const int i = threadIdx.x + q * 256;
            tmp[q] = i >= off ? buf[i - off] : 0;
        }
        __syncthreads();
        for (int q = 0; q < kScanBlock / 256; ++q) buf[threadIdx.x + q * 256] += tmp[q];
        __syncthreads();
    }
    for (int i = threadIdx.x; i < kScanBlock; i += blockDim.x)
        if (base + i < count) out[base + i] = buf[i] - (base + i < count ? in[base + i] : 0);
    if (threadIdx.x == 0 && block_sums) block_sums[blockIdx.x] = buf[kScanBlock - 1];
}

__global__ void scan_add_kernel(int64_t* __restrict__ data, int64_t count, const int64_t* __restrict__ block_offsets)
{
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < count) data[i] += block_offsets[i / kScanBlock];
}

// --- 3. segment reduction ---------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T round_operand(T x, bool bf16)
{
    return bf16 ? static_cast<T>(__bfloat162float(__float2bfloat16_rn(static_cast<float>(x)))) : x;
}

// Segment reduction for one side.  A side (side == 0): outputs o index rows of A (o < m), the
// contracted vector is b_j = B[k, :] (x < p) and u_j[o] = sum_x G[o, x] b_j[x].  B side
// (side == 1): outputs o index columns of B (o < p), the vector is a_j = A[:, k] (x < m) and
// u_j[o] = sum_x G[x, o] a_j[x].  A CTA owns an OB-wide block of outputs (blockIdx.y) and keeps
// that block of G resident in shared memory, transposed as Gs[x][o]; it walks a batch of
// segments k (blockIdx.x, grid-stride), regenerating each contribution's vector (all x) and
// the normals of its own outputs, and accumulates in FP64
//     gM[k, o] = sum_j omega_j u_j[o],   gS[k, o] = sum_j omega_j z_j[o] u_j[o].
template <typename T>
__global__ void __launch_bounds__(kAdjThreads) segment_kernel(AdjSegmentParams prm, int side)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int kin = side == 0 ? prm.p : prm.m;
    const int kout = side == 0 ? prm.m : prm.p;
    const int OB = prm.ob;
    const int o0 = blockIdx.y * OB;
    const int ob = min(OB, kout - o0);
    T* Gs = reinterpret_cast<T*>(smem_raw);                               // [kin][OB]
    T* vin = Gs + static_cast<int64_t>(kin) * OB;                           // [kAdjChunk][kin]
    T* zo = vin + static_cast<int64_t>(kAdjChunk) * kin;                    // [kAdjChunk][OB]
    double* omega = reinterpret_cast<double*>(zo + static_cast<int64_t>(kAdjChunk) * OB);  // [kAdjChunk]
    __shared__ uint64_t rec_s[kAdjChunk];

    // resident block of G, transposed
    for (int64_t e = threadIdx.x; e < static_cast<int64_t>(kin) * OB; e += blockDim.x) {
        const int x = static_cast<int>(e / OB), oo = static_cast<int>(e % OB);
        const int o = o0 + oo;
        double g = 0.0;
        if (oo < ob) g = side == 0 ? prm.G[static_cast<int64_t>(o) * prm.p + x] : prm.G[static_cast<int64_t>(x) * prm.p + o];
        Gs[e] = static_cast<T>(g);
    }
    const T* P = static_cast<const T*>(prm.PAB);
    const int64_t in_off = side == 0 ? 2 * static_cast<int64_t>(prm.m_pad) : 0;   // pairs of the contracted vector
    const PhiloxRoundKeys& rk_in = side == 0 ? prm.rkB : prm.rkA;
    const PhiloxRoundKeys& rk_out = side == 0 ? prm.rkA : prm.rkB;
    const int groups = blockDim.x / OB;   // contributions handled in parallel per output
    const int oo = threadIdx.x % OB;
    const int grp = threadIdx.x / OB;
    __syncthreads();

    for (int64_t k = blockIdx.x; k < prm.n; k += gridDim.x) {
        const int64_t seg0 = prm.offsets[k];
        const int64_t seg1 = k + 1 < prm.n ? prm.offsets[k + 1] : prm.total;
        double accM = 0.0, accS = 0.0;
        const T* row = P + k * prm.ld;
        for (int64_t c0 = seg0; c0 < seg1; c0 += kAdjChunk) {
            const int nc = static_cast<int>(seg1 - c0 < kAdjChunk ? seg1 - c0 : kAdjChunk);
            if (threadIdx.x < nc) rec_s[threadIdx.x] = prm.records[c0 + threadIdx.x];
            __syncthreads();
            // regenerate the contracted vectors (all x) and the normals of this output block
            const int nin4 = (kin + 3) / 4, nout4 = (ob + 3) / 4;
            for (int e = threadIdx.x; e < nc * (nin4 + nout4); e += blockDim.x) {
                const int j = e / (nin4 + nout4);
                const int r = e % (nin4 + nout4);
                const uint64_t rec = rec_s[j];
                const int l = static_cast<int>(rec & 31);
                const uint64_t s = rec >> 6;
                const bool is_in = r < nin4;
                const int g4 = is_in ? r : (o0 >> 2) + (r - nin4);   // block of four rows/columns
                const uint4 w = philox4x32_10_rk(make_uint4(static_cast<uint32_t>(g4), static_cast<uint32_t>(k),
                                                            static_cast<uint32_t>(s), level_sample_word(l, s)),
                                                 is_in ? rk_in : rk_out);
                T z[4];
                Normals<T>::four(w, z);
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int x = 4 * g4 + h;
                    if (is_in) {
                        if (x < kin) {
                            const T val = fma(row[in_off + 2 * x + 1], z[h], row[in_off + 2 * x]);
                            vin[static_cast<int64_t>(j) * kin + x] = round_operand(val, prm.bf16);
                        }
                    } else if (x - o0 < ob) {
                        zo[static_cast<int64_t>(j) * OB + (x - o0)] = z[h];
                    }
                }
            }
            if (threadIdx.x < nc) {
                const uint64_t rec = rec_s[threadIdx.x];
                const int l = static_cast<int>(rec & 31);
                const bool coarse = (rec >> 5) & 1;
                omega[threadIdx.x] = (prm.w_fine[l] + (coarse ? prm.w_coarse_extra[l] : 0.0)) * prm.inv_N[l];
            }
            __syncthreads();
            if (oo < ob) {
                for (int j = grp; j < nc; j += groups) {
                    const T* v = vin + static_cast<int64_t>(j) * kin;
                    T u = T(0);
                    for (int x = 0; x < kin; ++x) u = fma(Gs[static_cast<int64_t>(x) * OB + oo], v[x], u);
                    const double wu = omega[j] * static_cast<double>(u);
                    accM += wu;
                    accS += wu * static_cast<double>(zo[static_cast<int64_t>(j) * OB + oo]);
                }
            }
            __syncthreads();
        }
        // combine the contribution groups of each output in a fixed order, then write
        double* red = reinterpret_cast<double*>(vin);   // reuse: [groups][OB] x 2
        red[grp * OB + oo] = accM;
        red[(groups + grp) * OB + oo] = accS;
        __syncthreads();
        if (grp == 0 && oo < ob) {
            double tm = 0.0, ts = 0.0;
            for (int g = 0; g < groups; ++g) {
                tm += red[g * OB + oo];
                ts += red[(groups + g) * OB + oo];
            }
            const int o = o0 + oo;
            if (side == 0) {
                prm.gM_t[k * prm.m + o] += tm;
                prm.gS_t[k * prm.m + o] += ts;
            } else {
                prm.gMp[k * prm.p + o] += tm;
                prm.gSp[k * prm.p + o] += ts;
            }
        }
        __syncthreads();
    }
}

// n-major FP64 staging (n x m) -> caller's row-major m x n (leading dimension ld) in dtype D.
template <typename D>
__global__ void transpose_out_kernel(const double* __restrict__ src, int64_t n, int64_t m, D* dst, int64_t ld)
{
    __shared__ double tile[32][33];
    const int64_t k0 = static_cast<int64_t>(blockIdx.x) * 32, i0 = static_cast<int64_t>(blockIdx.y) * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int64_t k = k0 + y, i = i0 + threadIdx.x;
        tile[y][threadIdx.x] = (k < n && i < m) ? src[k * m + i] : 0.0;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int64_t i = i0 + y, k = k0 + threadIdx.x;
        if (i < m && k < n) dst[i * ld + k] = static_cast<D>(tile[threadIdx.x][y]);
    }
}

// n x p FP64 -> caller's n x p (leading dimension ld) in dtype D.
template <typename D>
__global__ void copy_out_kernel(const double* __restrict__ src, int64_t n, int64_t p, D* dst, int64_t ld)
{
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < n * p;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x)
        dst[(e / p) * ld + (e % p)] = static_cast<D>(src[e]);
}

inline unsigned blocks_for(int64_t n, int threads) { return static_cast<unsigned>((n + threads - 1) / threads); }

}  // namespace

cudaError_t adjoint_count(const AdjLevels& lv, uint2 keyI, int64_t n, int R, int* counts, cudaStream_t st)
{
    if (lv.total_pairs == 0) return cudaSuccess;
    const unsigned g = static_cast<unsigned>(std::min<int64_t>(blocks_for(lv.total_pairs, 256), 152 * 16));
    enumerate_kernel<<<g, 256, 0, st>>>(lv, keyI, n, R, counts, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t adjoint_scatter(const AdjLevels& lv, uint2 keyI, int64_t n, int R, int64_t* cursor, uint64_t* records,
                            cudaStream_t st)
{
    if (lv.total_pairs == 0) return cudaSuccess;
    const unsigned g = static_cast<unsigned>(std::min<int64_t>(blocks_for(lv.total_pairs, 256), 152 * 16));
    enumerate_kernel<<<g, 256, 0, st>>>(lv, keyI, n, R, nullptr, cursor, records);
    return cudaGetLastError();
}

int64_t adjoint_scan_scratch(int64_t n)
{
    const int64_t b1 = (n + kScanBlock - 1) / kScanBlock;
    const int64_t b2 = (b1 + kScanBlock - 1) / kScanBlock;
    return b1 + b1 + b2 + b2 + 1;
}

cudaError_t adjoint_scan(const int* counts, int64_t n, int64_t* offsets, int64_t* scratch, cudaStream_t st)
{
    const int64_t b1 = (n + kScanBlock - 1) / kScanBlock;
    const int64_t b2 = (b1 + kScanBlock - 1) / kScanBlock;
    if (b2 > kScanBlock) return cudaErrorInvalidValue;  // n above kScanBlock^3
    int64_t* sums1 = scratch;         // b1
    int64_t* offs1 = sums1 + b1;      // b1
    int64_t* sums2 = offs1 + b1;      // b2
    int64_t* offs2 = sums2 + b2;      // b2
    int64_t* tail = offs2 + b2;       // 1
    scan_block_kernel<<<static_cast<unsigned>(b1), 256, 0, st>>>(counts, n, offsets, sums1);
    scan_i64_block_kernel<<<static_cast<unsigned>(b2), 256, 0, st>>>(sums1, b1, offs1, sums2);
    scan_i64_block_kernel<<<1, 256, 0, st>>>(sums2, b2, offs2, tail);
    scan_add_kernel<<<blocks_for(b1, 256), 256, 0, st>>>(offs1, b1, offs2);
    scan_add_kernel<<<blocks_for(n, 256), 256, 0, st>>>(offsets, n, offs1);
    return cudaGetLastError();
}

size_t adjoint_segment_smem(int kin, int ob, bool f64)
{
    const size_t e = f64 ? 8 : 4;
    const size_t body = size_t(kin) * ob * e + size_t(kAdjChunk) * kin * e + size_t(kAdjChunk) * ob * e +
                        size_t(kAdjChunk) * 8;
    // the FP64 group reduction reuses the vector area: 2 * (threads / ob) * ob doubles
    const size_t red = size_t(2) * kAdjThreads * 8;
    const size_t vin_area = size_t(kAdjChunk) * kin * e;
    return body + (red > vin_area ? red - vin_area : 0);
}

int adjoint_output_block(int kin, bool f64)
{
    // largest power of two <= 64 whose G block (kin x ob) stays within 96 KB
    const size_t e = f64 ? 8 : 4;
    int ob = 64;
    while (ob > 8 && size_t(kin) * ob * e > 96 * 1024) ob /= 2;
    return ob;
}

cudaError_t adjoint_segments(const AdjSegmentParams& prm, bool f64, int side, int num_sms, cudaStream_t st)
{
    const int kin = side == 0 ? prm.p : prm.m;
    const int kout = side == 0 ? prm.m : prm.p;
    const size_t smem = adjoint_segment_smem(kin, prm.ob, f64);
    const int oblocks = (kout + prm.ob - 1) / prm.ob;
    const int batches = std::max(1, std::min<int>(static_cast<int>(std::min<int64_t>(prm.n, 1 << 20)),
                                                  (2 * num_sms + oblocks - 1) / oblocks));
    dim3 grid(static_cast<unsigned>(batches), static_cast<unsigned>(oblocks));
    cudaError_t e;
    if (f64) {
        e = cudaFuncSetAttribute(segment_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        segment_kernel<double><<<grid, kAdjThreads, smem, st>>>(prm, side);
    } else {
        e = cudaFuncSetAttribute(segment_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        segment_kernel<float><<<grid, kAdjThreads, smem, st>>>(prm, side);
    }
    return cudaGetLastError();
}

cudaError_t adjoint_write_A(const double* src, int64_t n, int64_t m, void* dst, int64_t ld, int dtype, cudaStream_t st)
{
    dim3 block(32, 8), grid(static_cast<unsigned>((n + 31) / 32), static_cast<unsigned>((m + 31) / 32));
    if (dtype == MLMC_DTYPE_F64)
        transpose_out_kernel<double><<<grid, block, 0, st>>>(src, n, m, static_cast<double*>(dst), ld);
    else
        transpose_out_kernel<float><<<grid, block, 0, st>>>(src, n, m, static_cast<float*>(dst), ld);
    return cudaGetLastError();
}

cudaError_t adjoint_write_B(const double* src, int64_t n, int64_t p, void* dst, int64_t ld, int dtype, cudaStream_t st)
{
    const unsigned g = static_cast<unsigned>(std::min<int64_t>(blocks_for(n * p, 256), 152 * 32));
    if (dtype == MLMC_DTYPE_F64)
        copy_out_kernel<double><<<g, 256, 0, st>>>(src, n, p, static_cast<double*>(dst), ld);
    else
        copy_out_kernel<float><<<g, 256, 0, st>>>(src, n, p, static_cast<float*>(dst), ld);
    return cudaGetLastError();
}

}  // namespace mlmc
