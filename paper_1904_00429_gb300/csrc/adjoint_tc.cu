// adjoint_tc.cu -- segment reduction of the adjoint on the tensor cores (BF16 plans).
//
// For a BF16 plan the replayed entries are bfloat16 values (the forward rounded them, and the
// straight-through gradient differentiates the rounded entries), so the contraction of one output
// block with the records of a chunk is a dense product: for the A side
//     U[o, j] = sum_x G[o, x] b_j[x],   o in the CTA's 128 outputs, j in the chunk's 64 records,
// (B side: G^T and the vectors a_j).  G is split into bfloat16 parts G = G_hi + G_lo + O(2^-17 |G|)
// once per CTA; each chunk runs M = 128, N = 64, K = 16 tcgen05 MMAs over both parts into one FP32
// accumulator in tensor memory.  The epilogue reads U (one output row per lane) and folds
//     gM[k, o] += sum_j omega_j U[o, j],   gS[k, o] += sum_j omega_j z_j[o] U[o, j]
// in FP32 per chunk and FP64 across chunks, exactly as the CUDA-core segment kernel does.
// Records, segments, weights and the regeneration of the vectors (Philox, the special-function-unit
// Box-Muller of the forward kernel, bfloat16 rounding) follow adjoint.cu.  Waits are bounded.
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "rng.cuh"
#include "tc_ptx.cuh"

namespace mlmc {
namespace {

constexpr int kTcThreads = 512;
constexpr int kTcGroups = kTcThreads / 128;   // record groups of the epilogue (4 warps each)
constexpr int kTcRec = 64;      // records per chunk = MMA N
constexpr int kTcOut = 128;     // outputs per CTA = MMA M
constexpr int kTcMaxKin = 256;  // contracted entries the resident G block allows

struct TcAdjSmem {
    // bytes from the 1024-aligned base
    size_t g_hi, g_lo, v, zo, omega, rec, red, bar, total;
    __host__ __device__ explicit TcAdjSmem(int kin)
    {
        const size_t atoms = (static_cast<size_t>(kin) + 63) / 64;   // 64 bf16 of K per swizzle atom
        g_hi = 0;
        g_lo = g_hi + atoms * kTcOut * 128;
        v = g_lo + atoms * kTcOut * 128;
        zo = v + atoms * kTcRec * 128;
        omega = zo + static_cast<size_t>(kTcRec) * kTcOut * 4;
        rec = omega + kTcRec * 4;
        red = rec + kTcRec * 8;
        bar = red + static_cast<size_t>(2 * kTcGroups) * kTcOut * 8;   // [record group][M, S][outputs]
        total = bar + 16 + 16;                              // mbarrier, tmem address, abort flag
    }
};

__device__ __forceinline__ uint16_t bf16_bits(float x)
{
    const __nv_bfloat16 b = __float2bfloat16_rn(x);
    return *reinterpret_cast<const uint16_t*>(&b);
}

template <int side>
__global__ void __launch_bounds__(kTcThreads, 1) segment_tc_kernel(const AdjSegmentParams prm, const TcLaunch tl)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~static_cast<uintptr_t>(1023));
    const int kin = side == 0 ? prm.p : prm.m;
    const int kout = side == 0 ? prm.m : prm.p;
    const int atoms = (kin + 63) / 64;
    const int o0 = blockIdx.y * kTcOut;
    const int ob = min(kTcOut, kout - o0);
    const TcAdjSmem L(kin);
    unsigned char* g_hi = smem + L.g_hi;
    unsigned char* g_lo = smem + L.g_lo;
    unsigned char* vt = smem + L.v;
    float* zo = reinterpret_cast<float*>(smem + L.zo);           // [kTcRec][kTcOut]
    float* omega = reinterpret_cast<float*>(smem + L.omega);     // [kTcRec]
    uint64_t* rec_s = reinterpret_cast<uint64_t*>(smem + L.rec);
    double* red = reinterpret_cast<double*>(smem + L.red);       // [kTcGroups][2][kTcOut]
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);
    uint32_t* tmem_s = reinterpret_cast<uint32_t*>(smem + L.bar + 8);
    volatile int* abort_s = reinterpret_cast<volatile int*>(smem + L.bar + 16);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t bar_a = tc::smem_addr(bar);
    if (warp == 0) tc::tmem_alloc(tc::smem_addr(tmem_s), kTcRec);
    if (tid == 0) {
        tc::mbar_init(bar_a, 1);
        tc::mbar_init_fence();
        *abort_s = 0;
    }
    // the CTA's block of G as bfloat16 hi and lo parts, K-major (K = contracted index), 128-byte swizzle
    for (int e = tid; e < kTcOut * atoms * 64; e += kTcThreads) {
        const int r = e / (atoms * 64), x = e % (atoms * 64);
        double g = 0.0;
        if (r < ob && x < kin)
            g = side == 0 ? prm.G[static_cast<int64_t>(o0 + r) * prm.p + x] : prm.G[static_cast<int64_t>(x) * prm.p + o0 + r];
        const float gf = static_cast<float>(g);
        const uint16_t hi = bf16_bits(gf);
        const float hif = __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(&hi));
        const uint16_t lo = bf16_bits(gf - hif);
        const uint32_t off = static_cast<uint32_t>((x >> 6) * kTcOut * 128) + tc::sw128_offset(r, (x & 63) >> 3) +
                             2u * static_cast<uint32_t>(x & 7);
        *reinterpret_cast<uint16_t*>(g_hi + off) = hi;
        *reinterpret_cast<uint16_t*>(g_lo + off) = lo;
    }
    tc::fence_proxy_async_smem();
    tc::tc_fence_before_sync();
    __syncthreads();
    tc::tc_fence_after_sync();
    const uint32_t tmem = *tmem_s;

    const float* P = static_cast<const float*>(prm.PAB);
    const int64_t in_off = side == 0 ? 2 * static_cast<int64_t>(prm.m_pad) : 0;
    const PhiloxRoundKeys& rk_in = side == 0 ? prm.rkB : prm.rkA;
    const PhiloxRoundKeys& rk_out = side == 0 ? prm.rkA : prm.rkB;
    constexpr uint32_t idesc = tc::idesc_bf16_f32(kTcOut, kTcRec);
    const int quarter = warp & 3;        // TMEM lanes (outputs) 32 * quarter ..
    constexpr int kGroupRec = kTcRec / kTcGroups;
    const int group = warp >> 2;         // records kGroupRec * group ..
    const int o_loc = quarter * 32 + lane;
    uint32_t chunks_done = 0;
    bool aborted = false;

    for (int64_t k = blockIdx.x; k < prm.n && !aborted; k += gridDim.x) {
        const int64_t seg0 = prm.offsets[k];
        const int64_t seg1 = k + 1 < prm.n ? prm.offsets[k + 1] : prm.total;
        if (seg0 == seg1) continue;   // uniform across the CTA
        double accM = 0.0, accS = 0.0;
        const float* row = P + k * prm.ld + in_off;
        for (int64_t c0 = seg0; c0 < seg1; c0 += kTcRec) {
            const int nc = static_cast<int>(seg1 - c0 < kTcRec ? seg1 - c0 : kTcRec);
            if (tid < kTcRec) {
                uint64_t rec = 0;
                float om = 0.0f;
                if (tid < nc) {
                    rec = prm.records[c0 + tid];
                    const int l = static_cast<int>(rec & 31);
                    const bool coarse = (rec >> 5) & 1;
                    om = static_cast<float>((prm.w_fine[l] + (coarse ? prm.w_coarse_extra[l] : 0.0)) * prm.inv_N[l]);
                }
                rec_s[tid] = rec;
                omega[tid] = om;
            }
            __syncthreads();
            // the chunk's contracted vectors, bfloat16, as the K-major B operand (one row per record)
            for (int e = tid; e < kTcRec * atoms * 16; e += kTcThreads) {
                const int j = e / (atoms * 16), g4 = e % (atoms * 16);
                const int x = 4 * g4;
                float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                if (j < nc && x < kin) {
                    const uint64_t rec = rec_s[j];
                    const uint64_t s = rec >> 6;
                    const uint4 w = philox4x32_10_rk(
                        make_uint4(static_cast<uint32_t>(g4), static_cast<uint32_t>(k), static_cast<uint32_t>(s),
                                   level_sample_word(static_cast<int>(rec & 31), s)),
                        rk_in);
                    float z[4];
                    normals4_mufu(w, z);
#pragma unroll
                    for (int h = 0; h < 4; ++h)
                        if (x + h < kin) v[h] = fmaf(row[2 * (x + h) + 1], z[h], row[2 * (x + h)]);
                }
                const uint32_t lo2 = static_cast<uint32_t>(bf16_bits(v[0])) | (static_cast<uint32_t>(bf16_bits(v[1])) << 16);
                const uint32_t hi2 = static_cast<uint32_t>(bf16_bits(v[2])) | (static_cast<uint32_t>(bf16_bits(v[3])) << 16);
                const uint32_t off = static_cast<uint32_t>((x >> 6) * kTcRec * 128) + tc::sw128_offset(j, (x & 63) >> 3) +
                                     2u * static_cast<uint32_t>(x & 7);
                *reinterpret_cast<uint2*>(vt + off) = make_uint2(lo2, hi2);
            }
            // normals of this CTA's outputs for every record of the chunk
            for (int e = tid; e < kTcRec * (kTcOut / 4); e += kTcThreads) {
                const int j = e / (kTcOut / 4), g4 = e % (kTcOut / 4);
                float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                if (j < nc && 4 * g4 < ob) {
                    const uint64_t rec = rec_s[j];
                    const uint64_t s = rec >> 6;
                    const uint4 w = philox4x32_10_rk(
                        make_uint4(static_cast<uint32_t>((o0 >> 2) + g4), static_cast<uint32_t>(k), static_cast<uint32_t>(s),
                                   level_sample_word(static_cast<int>(rec & 31), s)),
                        rk_out);
                    normals4_mufu(w, z);
                }
                *reinterpret_cast<float4*>(zo + j * kTcOut + 4 * g4) = make_float4(z[0], z[1], z[2], z[3]);
            }
            tc::fence_proxy_async_smem();
            tc::tc_fence_before_sync();
            __syncthreads();
            if (tid == 0) {
                tc::tc_fence_after_sync();
                for (int part = 0; part < 2; ++part) {
                    const uint32_t ga = tc::smem_addr(part ? g_lo : g_hi);
                    for (int ks = 0; ks < atoms * 4; ++ks) {
                        const uint64_t adesc = tc::sw128_kmajor_desc(ga + (ks >> 2) * kTcOut * 128 + 32 * (ks & 3));
                        const uint64_t bdesc =
                            tc::sw128_kmajor_desc(tc::smem_addr(vt) + (ks >> 2) * kTcRec * 128 + 32 * (ks & 3));
                        tc::mma_bf16(tmem, adesc, bdesc, idesc, (part > 0 || ks > 0) ? 1u : 0u);
                    }
                }
                tc::mma_commit(bar_a);
            }
            if (!tc::mbar_wait_bounded(bar_a, chunks_done & 1, tc::globaltimer() + tl.timeout_ns)) {
                *abort_s = 1;
                atomicExch(tl.err_flag, MLMC_ERR_TIMEOUT);
            }
            ++chunks_done;
            tc::tc_fence_after_sync();
            float u[kGroupRec];
            static_assert(kGroupRec == 16, "one 16-column TMEM load per warp");
            tc::tmem_ld_32x32b_x16_nowait(
                tmem + (static_cast<uint32_t>(quarter * 32) << 16) + static_cast<uint32_t>(group * kGroupRec), u);
            tc::tmem_ld_wait();
            float sm = 0.0f, ss = 0.0f;
#pragma unroll
            for (int jj = 0; jj < kGroupRec; ++jj) {
                const int j = group * kGroupRec + jj;
                const float wu = omega[j] * u[jj];
                sm += wu;
                ss = fmaf(wu, zo[j * kTcOut + o_loc], ss);
            }
            accM += static_cast<double>(sm);
            accS += static_cast<double>(ss);
            tc::tc_fence_before_sync();
            __syncthreads();   // vectors, normals and the accumulator may be overwritten
            if (*abort_s) {
                aborted = true;
                break;
            }
        }
        if (aborted) break;
        // the record groups of every output, summed in a fixed order
        red[(group * 2 + 0) * kTcOut + o_loc] = accM;
        red[(group * 2 + 1) * kTcOut + o_loc] = accS;
        __syncthreads();
        if (tid < ob) {
            double tm = 0.0, ts = 0.0;
#pragma unroll
            for (int g = 0; g < kTcGroups; ++g) {
                tm += red[(2 * g) * kTcOut + tid];
                ts += red[(2 * g + 1) * kTcOut + tid];
            }
            const int o = o0 + tid;
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
    if (aborted && tid == 0) {
        // no MMA may still write tensor memory when it is freed: wait (bounded) once more for the
        // commit of the chunk whose wait gave up
        tc::mbar_wait_bounded(bar_a, (chunks_done - 1) & 1, tc::globaltimer() + 100000000ull);
    }
    tc::tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTcRec);
}

template <int side>
cudaError_t launch_side(const AdjSegmentParams& prm, const TcLaunch& tl, cudaStream_t st)
{
    const int kin = side == 0 ? prm.p : prm.m;
    const int kout = side == 0 ? prm.m : prm.p;
    const size_t smem = TcAdjSmem(kin).total + 1024;
    cudaError_t e = cudaFuncSetAttribute(segment_tc_kernel<side>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int oblocks = (kout + kTcOut - 1) / kTcOut;
    const int64_t want = (static_cast<int64_t>(tl.num_sms) + oblocks - 1) / oblocks;
    const unsigned batches = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(prm.n, want)));
    segment_tc_kernel<side><<<dim3(batches, static_cast<unsigned>(oblocks)), kTcThreads, smem, st>>>(prm, tl);
    return cudaGetLastError();
}

}  // namespace

bool adjoint_tc_supported(int kin) { return kin >= 1 && kin <= kTcMaxKin && TcAdjSmem(kin).total + 1024 <= 227 * 1024; }

cudaError_t adjoint_segments_tc(const AdjSegmentParams& prm, int side, const TcLaunch& tl, cudaStream_t st)
{
    if (!adjoint_tc_supported(side == 0 ? prm.p : prm.m)) return cudaErrorInvalidValue;
    return side == 0 ? launch_side<0>(prm, tl, st) : launch_side<1>(prm, tl, st);
}

}  // namespace mlmc
