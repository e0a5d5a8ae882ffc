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
constexpr size_t kAdjSmemMax = 227 * 1024;

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

// Normals of the replayed entries: the form the forward kernel of the plan's precision used.
// BF16 plans draw them with the special-function-unit Box-Muller of the tensor-core kernel, so
// the straight-through gradient sees the very entries the forward rounded.
template <typename T>
__device__ __forceinline__ void adj_normals(uint4 w, T z[4], bool sfu)
{
    if constexpr (sizeof(T) == 4) {
        if (sfu)
            normals4_mufu(w, z);
        else
            Normals<T>::four(w, z);
    } else {
        Normals<T>::four(w, z);
    }
}
template <typename T>
__device__ __forceinline__ T round_operand(T x, bool bf16)
{
    return bf16 ? static_cast<T>(__bfloat162float(__float2bfloat16_rn(static_cast<float>(x)))) : x;
}

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
    static __device__ __forceinline__ void load(const float* p, float v[4])
    {
        const float4 a = *reinterpret_cast<const float4*>(p);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    }
};
template <>
struct Vec4<double> {
    static __device__ __forceinline__ void load(const double* p, double v[4])
    {
        const double2 a = reinterpret_cast<const double2*>(p)[0];
        const double2 b = reinterpret_cast<const double2*>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
};

constexpr int kAdjNJ = 8;                    // records per warp per chunk
constexpr int kAdjRec = kAdjNJ * (kAdjThreads / 32);   // records per chunk (64)
constexpr int kAdjSlab = 64;                 // contracted entries regenerated per slab

// Shared-memory layout of the segment kernel (bytes from the base), for kin contracted
// entries, OB = 32 * opt outputs and element size e.
struct SegSmem {
    size_t g, vin, zo, omega, red, rec, total;
    __host__ __device__ SegSmem(int kin, int opt, int e)
    {
        const size_t OB = size_t(32) * opt;
        const size_t kin4 = (size_t(kin) + 3) / 4 * 4;
        g = 0;
        vin = g + kin4 * OB * e;
        zo = vin + size_t(kAdjRec) * kAdjSlab * e;
        omega = zo + size_t(kAdjRec) * OB * e;
        red = (omega + size_t(kAdjRec) * e + 15) / 16 * 16;
        rec = red + size_t(2) * (kAdjThreads / 32) * OB * 8;
        total = rec + size_t(kAdjRec) * 8;
    }
};

// Segment reduction for one side.  A side (side == 0): outputs o index rows of A (o < m), the
// contracted vector is b_j = B[k, :] (x < p) and u_j[o] = sum_x G[o, x] b_j[x].  B side
// (side == 1): outputs o index columns of B (o < p), the vector is a_j = A[:, k] (x < m) and
// u_j[o] = sum_x G[x, o] a_j[x].  A CTA owns OB = 32 * OPT outputs (blockIdx.y) and keeps that
// block of G resident in shared memory, transposed as Gs[x][o]; it walks a batch of segments k
// (blockIdx.x, grid-stride).  The records of a segment are taken 64 at a time: warp w owns
// records 8w .. 8w + 7 of the chunk and lane t the outputs t, t + 32, ..., so every thread
// carries an OPT x 8 register tile of u.  The contracted vectors are regenerated from Philox in
// slabs of 64 entries (all records of the chunk), the normals of the CTA's outputs once per
// chunk.  Per chunk each thread folds its 8 records in the working precision, then adds the
// result to FP64 accumulators
//     gM[k, o] += sum_j omega_j u_j[o],   gS[k, o] += sum_j omega_j z_j[o] u_j[o];
// at the end of the segment the 8 warps' accumulators are summed in warp order.
template <typename T, int OPT, int side>
__global__ void __launch_bounds__(kAdjThreads, 1) segment_kernel(const AdjSegmentParams prm)
{
    constexpr int OB = 32 * OPT;
    constexpr int NW = kAdjThreads / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int kin = side == 0 ? prm.p : prm.m;
    const int kin4 = (kin + 3) & ~3;
    const int kout = side == 0 ? prm.m : prm.p;
    const int o0 = blockIdx.y * OB;
    const int ob = min(OB, kout - o0);
    const SegSmem L(kin, OPT, int(sizeof(T)));
    T* Gs = reinterpret_cast<T*>(smem_raw + L.g);          // [kin4][OB]
    T* vin = reinterpret_cast<T*>(smem_raw + L.vin);       // [kAdjRec][kAdjSlab]
    T* zo = reinterpret_cast<T*>(smem_raw + L.zo);         // [kAdjRec][OB]
    T* omega = reinterpret_cast<T*>(smem_raw + L.omega);   // [kAdjRec]
    double* red = reinterpret_cast<double*>(smem_raw + L.red);   // [2][NW][OB]
    uint64_t* rec_s = reinterpret_cast<uint64_t*>(smem_raw + L.rec);

    for (int e = threadIdx.x; e < kin4 * OB; e += kAdjThreads) {
        const int x = e / OB, oo = e % OB;
        const int o = o0 + oo;
        double g = 0.0;
        if (oo < ob && x < kin)
            g = side == 0 ? prm.G[static_cast<int64_t>(o) * prm.p + x] : prm.G[static_cast<int64_t>(x) * prm.p + o];
        Gs[e] = static_cast<T>(g);
    }
    const T* P = static_cast<const T*>(prm.PAB);
    const int64_t in_off = side == 0 ? 2 * static_cast<int64_t>(prm.m_pad) : 0;
    const PhiloxRoundKeys& rk_in = side == 0 ? prm.rkB : prm.rkA;
    const PhiloxRoundKeys& rk_out = side == 0 ? prm.rkA : prm.rkB;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    __syncthreads();

    for (int64_t k = blockIdx.x; k < prm.n; k += gridDim.x) {
        const int64_t seg0 = prm.offsets[k];
        const int64_t seg1 = k + 1 < prm.n ? prm.offsets[k + 1] : prm.total;
        if (seg0 == seg1) continue;   // uniform across the CTA
        double accM[OPT], accS[OPT];
#pragma unroll
        for (int q = 0; q < OPT; ++q) accM[q] = accS[q] = 0.0;
        const T* row = P + k * prm.ld + in_off;
        for (int64_t c0 = seg0; c0 < seg1; c0 += kAdjRec) {
            const int nc = static_cast<int>(seg1 - c0 < kAdjRec ? seg1 - c0 : kAdjRec);
            // records, weights and the normals of this CTA's outputs
            if (threadIdx.x < kAdjRec) {
                uint64_t rec = 0;
                T om = T(0);
                if (threadIdx.x < nc) {
                    rec = prm.records[c0 + threadIdx.x];
                    const int l = static_cast<int>(rec & 31);
                    const bool coarse = (rec >> 5) & 1;
                    om = static_cast<T>((prm.w_fine[l] + (coarse ? prm.w_coarse_extra[l] : 0.0)) * prm.inv_N[l]);
                }
                rec_s[threadIdx.x] = rec;
                omega[threadIdx.x] = om;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < kAdjRec * (OB / 4); e += kAdjThreads) {
                const int j = e / (OB / 4), g4 = e % (OB / 4);
                T z[4] = {T(0), T(0), T(0), T(0)};
                if (j < nc && 4 * g4 < ob) {
                    const uint64_t rec = rec_s[j];
                    const uint64_t s = rec >> 6;
                    const uint4 w = philox4x32_10_rk(
                        make_uint4(static_cast<uint32_t>((o0 >> 2) + g4), static_cast<uint32_t>(k),
                                   static_cast<uint32_t>(s), level_sample_word(static_cast<int>(rec & 31), s)),
                        rk_out);
                    adj_normals<T>(w, z, prm.bf16 != 0);
                }
#pragma unroll
                for (int h = 0; h < 4; ++h) zo[j * OB + 4 * g4 + h] = z[h];
            }
            T u[OPT][kAdjNJ];
#pragma unroll
            for (int q = 0; q < OPT; ++q)
#pragma unroll
                for (int j = 0; j < kAdjNJ; ++j) u[q][j] = T(0);

            for (int x0 = 0; x0 < kin4; x0 += kAdjSlab) {
                const int len = min(kAdjSlab, kin4 - x0);
                __syncthreads();   // previous slab consumed
                for (int e = threadIdx.x; e < kAdjRec * (kAdjSlab / 4); e += kAdjThreads) {
                    const int j = e / (kAdjSlab / 4), g4 = e % (kAdjSlab / 4);
                    const int x = x0 + 4 * g4;
                    T v[4] = {T(0), T(0), T(0), T(0)};
                    if (j < nc && x < kin) {
                        const uint64_t rec = rec_s[j];
                        const uint64_t s = rec >> 6;
                        const uint4 w = philox4x32_10_rk(
                            make_uint4(static_cast<uint32_t>(x >> 2), static_cast<uint32_t>(k), static_cast<uint32_t>(s),
                                       level_sample_word(static_cast<int>(rec & 31), s)),
                            rk_in);
                        T z[4];
                        adj_normals<T>(w, z, prm.bf16 != 0);
#pragma unroll
                        for (int h = 0; h < 4; ++h)
                            if (x + h < kin) v[h] = round_operand(fma(row[2 * (x + h) + 1], z[h], row[2 * (x + h)]), prm.bf16);
                    }
#pragma unroll
                    for (int h = 0; h < 4; ++h) vin[j * kAdjSlab + 4 * g4 + h] = v[h];
                }
                __syncthreads();
                const T* vw = vin + warp * kAdjNJ * kAdjSlab;
                const T* gx = Gs + static_cast<int64_t>(x0) * OB + lane;
                for (int xx = 0; xx < len; xx += 4) {
                    T g[4][OPT];
#pragma unroll
                    for (int h = 0; h < 4; ++h)
#pragma unroll
                        for (int q = 0; q < OPT; ++q) g[h][q] = gx[(xx + h) * OB + 32 * q];
#pragma unroll
                    for (int j = 0; j < kAdjNJ; ++j) {
                        T v[4];
                        Vec4<T>::load(vw + j * kAdjSlab + xx, v);
#pragma unroll
                        for (int q = 0; q < OPT; ++q) {
                            T a = u[q][j];
                            a = fma(g[0][q], v[0], a);
                            a = fma(g[1][q], v[1], a);
                            a = fma(g[2][q], v[2], a);
                            a = fma(g[3][q], v[3], a);
                            u[q][j] = a;
                        }
                    }
                }
            }
            // fold this chunk's records (working precision), then into the FP64 accumulators
#pragma unroll
            for (int q = 0; q < OPT; ++q) {
                const int oo = lane + 32 * q;
                T sm = T(0), ss = T(0);
#pragma unroll
                for (int j = 0; j < kAdjNJ; ++j) {
                    const int jj = warp * kAdjNJ + j;
                    const T wu = omega[jj] * u[q][j];
                    sm += wu;
                    ss = fma(wu, zo[jj * OB + oo], ss);
                }
                accM[q] += static_cast<double>(sm);
                accS[q] += static_cast<double>(ss);
            }
            __syncthreads();   // records, weights and normals of the chunk consumed
        }
#pragma unroll
        for (int q = 0; q < OPT; ++q) {
            red[warp * OB + lane + 32 * q] = accM[q];
            red[(NW + warp) * OB + lane + 32 * q] = accS[q];
        }
        __syncthreads();
        for (int oo = threadIdx.x; oo < ob; oo += kAdjThreads) {
            double tm = 0.0, ts = 0.0;
            for (int w = 0; w < NW; ++w) {
                tm += red[w * OB + oo];
                ts += red[(NW + w) * OB + oo];
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

size_t adjoint_segment_smem(int kin, int opt, bool f64) { return SegSmem(kin, opt, f64 ? 8 : 4).total; }

int adjoint_output_block(int kin, bool f64)
{
    // widest register tile whose resident block of G fits next to the slab buffers
    for (int opt = 4; opt >= 1; opt /= 2)
        if (adjoint_segment_smem(kin, opt, f64) <= kAdjSmemMax) return opt;
    return 0;
}

template <typename T, int OPT, int side>
cudaError_t launch_segments(const AdjSegmentParams& prm, int num_sms, cudaStream_t st)
{
    const int kin = side == 0 ? prm.p : prm.m;
    const int kout = side == 0 ? prm.m : prm.p;
    const size_t smem = adjoint_segment_smem(kin, OPT, sizeof(T) == 8);
    const int oblocks = (kout + 32 * OPT - 1) / (32 * OPT);
    const int64_t want = (int64_t(2) * num_sms + oblocks - 1) / oblocks;
    const unsigned batches = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(prm.n, want)));
    cudaError_t e = cudaFuncSetAttribute(segment_kernel<T, OPT, side>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    segment_kernel<T, OPT, side><<<dim3(batches, static_cast<unsigned>(oblocks)), kAdjThreads, smem, st>>>(prm);
    return cudaGetLastError();
}

cudaError_t adjoint_segments(const AdjSegmentParams& prm, bool f64, int side, int num_sms, cudaStream_t st)
{
    switch ((f64 ? 16 : 0) + (side ? 8 : 0) + prm.ob) {
    case 1: return launch_segments<float, 1, 0>(prm, num_sms, st);
    case 2: return launch_segments<float, 2, 0>(prm, num_sms, st);
    case 4: return launch_segments<float, 4, 0>(prm, num_sms, st);
    case 9: return launch_segments<float, 1, 1>(prm, num_sms, st);
    case 10: return launch_segments<float, 2, 1>(prm, num_sms, st);
    case 12: return launch_segments<float, 4, 1>(prm, num_sms, st);
    case 17: return launch_segments<double, 1, 0>(prm, num_sms, st);
    case 18: return launch_segments<double, 2, 0>(prm, num_sms, st);
    case 20: return launch_segments<double, 4, 0>(prm, num_sms, st);
    case 25: return launch_segments<double, 1, 1>(prm, num_sms, st);
    case 26: return launch_segments<double, 2, 1>(prm, num_sms, st);
    case 28: return launch_segments<double, 4, 1>(prm, num_sms, st);
    default: return cudaErrorInvalidValue;
    }
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
