// level_tc_bf16.cu -- fused level kernel on the 5th-generation tensor cores (BF16 operands,
// FP32 accumulation in tensor memory).
//
// Per sample s of level l the kernel forms D = (n/c_l) sum_t sigma_t a_t b_t^T, the coupled
// difference P_l - P_{l-1} of Alg. 1 for ratio R = 2: every slot carries weight n/c_l and the
// odd (coarse, r_{2j}) slots additionally -2 n/c_l, i.e. sigma_t = +1 for even and -1 for odd
// slots at l >= 1 (sigma = +1 at l = 0).  sigma is folded into the B operand before rounding
// (exact); the magnitude n/c_l is applied to the FP32 accumulator.
//
// Persistent CTAs of 8 warps walk (chunk of samples, output tile) work items.  For each
// 64-slot K-block of a sample, all warps draw the slot indices, gather the sampled (M, S) /
// (M', S') pairs, generate A = M + S Z and sigma (M' + S' Z') from Philox, round them to bf16
// and store them into a 128-byte-swizzled K-major tile of a 2- or 3-stage shared-memory ring;
// one thread then issues tcgen05.mma (M = 128 per half, N = tile width, K = 16 steps) into
// TMEM and commits to the stage's mbarrier, so the next stage is generated while the tensor
// core works.  After the last K-block of a sample, the 8 warps drain the accumulator with
// tcgen05.ld, add the sample's D to the chunk partial in global memory (the TMEM is fully
// used by D for 256 x 256 tiles) and accumulate ||D||_F^2.  Every mbarrier wait is bounded by
// a %globaltimer deadline; on timeout the kernel records MLMC_ERR_TIMEOUT and leaves after
// freeing its tensor memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "rng.cuh"
#include "tc_ptx.cuh"

namespace mlmc {
namespace {

constexpr int kThreads = 256;
constexpr int kKB = 64;  // slots per K-block: one 128-byte swizzle atom of bf16

template <int MH, int BN>
struct TcCfg {
    static constexpr int kRows = 128 * MH;                  // output rows of a tile
    static constexpr int kABytes = kRows * 128;             // kRows x 64 bf16
    static constexpr int kBBytes = BN * 128;                // BN x 64 bf16 (B transposed, K-major)
    static constexpr int kStageBytes = kABytes + kBBytes;
    static constexpr int kStages = kStageBytes * 3 <= 200 * 1024 ? 3 : 2;
    static constexpr int kTileCols = MH * BN;
    static constexpr int kTmemCols = kTileCols <= 32 ? 32 : kTileCols <= 64 ? 64 : kTileCols <= 128 ? 128
                                     : kTileCols <= 256 ? 256 : 512;
    // dynamic shared memory: stage tiles (1024-aligned), then bookkeeping
    static constexpr int kBookBytes = kStages * kKB * 4 /*idx*/ + kStages * kKB * 4 /*sign*/ +
                                      (kStages + 1) * 8 /*mbarriers*/ + 16 /*tmem addr, abort*/ + 8 * 8 /*red*/;
    static constexpr int kSmemBytes = 1024 /*align slack*/ + kStages * kStageBytes + kBookBytes;
    static_assert(kTileCols <= 512, "tile exceeds tensor memory");
    static_assert(BN % 16 == 0 && BN >= 32 && BN <= 256, "N of the MMA");
};

struct TcExtra {
    int* err_flag;
    uint64_t timeout_ns;
    int total_items;  // nchunks * tiles
    float scale;      // n / c_l
};

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

template <int MH, int BN>
__global__ void __launch_bounds__(kThreads, 1) level_tc_bf16_kernel(const LevelParams prm, const TcExtra ex)
{
    using C = TcCfg<MH, BN>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~static_cast<uintptr_t>(1023));
    unsigned char* tiles = smem;
    int* idx_s = reinterpret_cast<int*>(smem + C::kStages * C::kStageBytes);
    float* sgn_s = reinterpret_cast<float*>(idx_s + C::kStages * kKB);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sgn_s + C::kStages * kKB);  // [kStages] free + [1] done
    uint32_t* tmem_s = reinterpret_cast<uint32_t*>(bars + C::kStages + 1);
    int* abort_s = reinterpret_cast<int*>(tmem_s + 1);
    double* red_s = reinterpret_cast<double*>(tmem_s + 4);

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const uint32_t bar_done = tc::smem_addr(&bars[C::kStages]);

    if (warp == 0) tc::tmem_alloc(tc::smem_addr(tmem_s), C::kTmemCols);
    if (tid == 0) {
        for (int st = 0; st <= C::kStages; ++st) tc::mbar_init(tc::smem_addr(&bars[st]), 1);
        tc::mbar_init_fence();
        *abort_s = 0;
    }
    tc::tc_fence_before_sync();
    __syncthreads();
    tc::tc_fence_after_sync();
    const uint32_t tmem = *tmem_s;

    const int tiles_n = prm.tiles_m * prm.tiles_p;
    const float* PA = static_cast<const float*>(prm.PA);
    const float* PB = static_cast<const float*>(prm.PB);
    const int nkb = (prm.c + kKB - 1) / kKB;
    constexpr uint32_t idesc = tc::idesc_bf16_f32(128, BN);

    uint32_t kb_count = 0;    // K-blocks issued by this CTA (ring position and phase)
    uint32_t done_count = 0;  // samples completed by this CTA (phase of the done barrier)
    bool aborted = false;

    for (int item = blockIdx.x; item < ex.total_items && !aborted; item += gridDim.x) {
        const int cy = item / tiles_n;
        const int tile = item % tiles_n;
        const int tm0 = (tile / prm.tiles_p) * C::kRows;
        const int tp0 = (tile % prm.tiles_p) * BN;
        const uint64_t chunk = prm.chunk0 + static_cast<uint64_t>(cy);
        const uint64_t sa = max(prm.s_begin, chunk * kChunk);
        const uint64_t sb = min(prm.s_end, (chunk + 1) * kChunk);
        float* part = static_cast<float*>(prm.partial_sum) + static_cast<int64_t>(cy) * prm.m * prm.p;
        double q = 0.0;

        for (uint64_t s = sa; s < sb && !aborted; ++s) {
            const uint32_t lsw = level_sample_word(prm.l, s);
            const uint32_t s_lo = static_cast<uint32_t>(s);
            for (int kb = 0; kb < nkb; ++kb, ++kb_count) {
                const int stage = static_cast<int>(kb_count % C::kStages);
                unsigned char* a_tile = tiles + stage * C::kStageBytes;
                unsigned char* b_tile = a_tile + C::kABytes;
                int* idx = idx_s + stage * kKB;
                float* sgn = sgn_s + stage * kKB;
                // the ring slot is free once the MMAs of K-block kb_count - kStages completed
                if (kb_count >= static_cast<uint32_t>(C::kStages)) {
                    const uint32_t use = kb_count / C::kStages - 1;
                    if (!tc::mbar_wait_bounded(tc::smem_addr(&bars[stage]), use & 1,
                                               tc::globaltimer() + ex.timeout_ns)) {
                        *abort_s = 1;
                        atomicExch(ex.err_flag, MLMC_ERR_TIMEOUT);
                    }
                }
                // slot indices and signs of this K-block
                if (tid < kKB / 2) {
                    const int t = kb * kKB + 2 * tid;
                    int64_t r0 = -1, r1 = -1;
                    if (t < prm.c) index_pair(prm.keyI, lsw, s_lo, t >> 1, static_cast<uint64_t>(prm.n), r0, r1);
                    idx[2 * tid] = t < prm.c ? static_cast<int>(r0) : -1;
                    idx[2 * tid + 1] = t + 1 < prm.c ? static_cast<int>(r1) : -1;
                    // slot t is coarse iff t % 2 == 1 (ratio 2) and l > 0
                    sgn[2 * tid] = 1.0f;
                    sgn[2 * tid + 1] = prm.l > 0 ? -1.0f : 1.0f;
                }
                __syncthreads();
                if (*abort_s) {
                    aborted = true;
                    break;
                }
                // A tile: kRows rows x 64 slots; item = (row group of 4, slot group of 8)
                for (int it = tid; it < (C::kRows / 4) * 8; it += kThreads) {
                    const int g4 = it % (C::kRows / 4);
                    const int sg = it / (C::kRows / 4);
                    const int i = tm0 + 4 * g4;
                    float v[4][8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int k = idx[sg * 8 + u];
                        if (k >= 0 && i < prm.m) {
                            const uint4 w = philox4x32_10(
                                make_uint4(static_cast<uint32_t>(i >> 2), static_cast<uint32_t>(k), s_lo, lsw),
                                prm.keyA);
                            float z[4];
                            normals4_f32(w, z);
                            const float4* src = reinterpret_cast<const float4*>(
                                PA + (static_cast<int64_t>(k) * prm.m_pad + i) * 2);
                            const float4 p0 = __ldg(src);
                            const float4 p1 = __ldg(src + 1);
                            v[0][u] = fmaf(p0.y, z[0], p0.x);
                            v[1][u] = fmaf(p0.w, z[1], p0.z);
                            v[2][u] = fmaf(p1.y, z[2], p1.x);
                            v[3][u] = fmaf(p1.w, z[3], p1.z);
                        } else {
                            v[0][u] = v[1][u] = v[2][u] = v[3][u] = 0.0f;
                        }
                    }
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const uint4 packed = make_uint4(pack_bf16x2(v[r][0], v[r][1]), pack_bf16x2(v[r][2], v[r][3]),
                                                        pack_bf16x2(v[r][4], v[r][5]), pack_bf16x2(v[r][6], v[r][7]));
                        *reinterpret_cast<uint4*>(a_tile + tc::sw128_offset(4 * g4 + r, sg)) = packed;
                    }
                }
                // B tile (transposed: BN rows j x 64 slots), sign folded in
                for (int it = tid; it < (BN / 4) * 8; it += kThreads) {
                    const int g4 = it % (BN / 4);
                    const int sg = it / (BN / 4);
                    const int j = tp0 + 4 * g4;
                    float v[4][8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int k = idx[sg * 8 + u];
                        if (k >= 0 && j < prm.p) {
                            const uint4 w = philox4x32_10(
                                make_uint4(static_cast<uint32_t>(j >> 2), static_cast<uint32_t>(k), s_lo, lsw),
                                prm.keyB);
                            float z[4];
                            normals4_f32(w, z);
                            const float4* src = reinterpret_cast<const float4*>(
                                PB + (static_cast<int64_t>(k) * prm.p_pad + j) * 2);
                            const float4 p0 = __ldg(src);
                            const float4 p1 = __ldg(src + 1);
                            const float sg_t = sgn[sg * 8 + u];
                            v[0][u] = sg_t * fmaf(p0.y, z[0], p0.x);
                            v[1][u] = sg_t * fmaf(p0.w, z[1], p0.z);
                            v[2][u] = sg_t * fmaf(p1.y, z[2], p1.x);
                            v[3][u] = sg_t * fmaf(p1.w, z[3], p1.z);
                        } else {
                            v[0][u] = v[1][u] = v[2][u] = v[3][u] = 0.0f;
                        }
                    }
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const uint4 packed = make_uint4(pack_bf16x2(v[r][0], v[r][1]), pack_bf16x2(v[r][2], v[r][3]),
                                                        pack_bf16x2(v[r][4], v[r][5]), pack_bf16x2(v[r][6], v[r][7]));
                        *reinterpret_cast<uint4*>(b_tile + tc::sw128_offset(4 * g4 + r, sg)) = packed;
                    }
                }
                tc::fence_proxy_async_smem();
                __syncthreads();
                if (tid == 0) {
                    tc::tc_fence_after_sync();
                    const int kt = min(kKB, prm.c - kb * kKB);
                    const int ksteps = (kt + 15) / 16;
                    const uint32_t a_base = tc::smem_addr(a_tile);
                    const uint32_t b_base = tc::smem_addr(b_tile);
                    for (int kk = 0; kk < ksteps; ++kk) {
                        const uint64_t bdesc = tc::sw128_kmajor_desc(b_base + 32 * kk);
#pragma unroll
                        for (int h = 0; h < MH; ++h) {
                            const uint64_t adesc = tc::sw128_kmajor_desc(a_base + h * 128 * 128 + 32 * kk);
                            tc::mma_bf16(tmem + h * BN, adesc, bdesc, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
                        }
                    }
                    tc::mma_commit(tc::smem_addr(&bars[stage]));
                    if (kb == nkb - 1) tc::mma_commit(bar_done);
                }
            }
            if (aborted) break;
            // sample epilogue: wait for the accumulator, then drain it
            if (!tc::mbar_wait_bounded(bar_done, done_count & 1, tc::globaltimer() + ex.timeout_ns)) {
                *abort_s = 1;
                atomicExch(ex.err_flag, MLMC_ERR_TIMEOUT);
            }
            ++done_count;
            __syncthreads();
            if (*abort_s) {
                aborted = true;
                break;
            }
            tc::tc_fence_after_sync();
            {
                const int quarter = warp & 3;
                const int hgrp = warp >> 2;
                // MH == 2: warp group h drains M-half h (all BN columns); MH == 1: the two warp
                // groups split the columns, or group 0 takes all of them when BN < 64.
                const bool split = MH == 1 && BN >= 64;
                const int row_local = (MH == 2 ? hgrp * 128 : 0) + quarter * 32 + lane;
                const int col_tm = MH == 2 ? hgrp * BN : (split ? hgrp * (BN / 2) : 0);
                const int col_d = MH == 2 ? 0 : col_tm;
                const int ncols = MH == 2 ? BN : (split ? BN / 2 : (hgrp == 0 ? BN : 0));
                const int gi = tm0 + row_local;
                const bool first = (s == sa);
                for (int cb = 0; cb < ncols; cb += 32) {
                    float v[32];
                    tc::tmem_ld_32x32b_x32(tmem + (static_cast<uint32_t>(quarter * 32) << 16) +
                                               static_cast<uint32_t>(col_tm + cb),
                                           v);
                    float qs = 0.0f;
#pragma unroll
                    for (int e = 0; e < 32; ++e) {
                        v[e] *= ex.scale;
                        qs = fmaf(v[e], v[e], qs);
                    }
                    q += static_cast<double>(qs);
                    const int gj0 = tp0 + col_d + cb;
                    if (gi < prm.m && gj0 < prm.p) {
                        float* dst = part + static_cast<int64_t>(gi) * prm.p + gj0;
                        const int valid = min(32, prm.p - gj0);
                        if (valid == 32 && (prm.p & 3) == 0) {
                            float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
                            for (int e4 = 0; e4 < 8; ++e4) {
                                float4 o = first ? make_float4(0.f, 0.f, 0.f, 0.f) : d4[e4];
                                o.x += v[4 * e4];
                                o.y += v[4 * e4 + 1];
                                o.z += v[4 * e4 + 2];
                                o.w += v[4 * e4 + 3];
                                d4[e4] = o;
                            }
                        } else {
#pragma unroll
                            for (int e = 0; e < 32; ++e)
                                if (e < valid) dst[e] = first ? v[e] : dst[e] + v[e];
                        }
                    }
                }
            }
            tc::tc_fence_before_sync();
            __syncthreads();  // the accumulator may be overwritten by the next sample
        }
        if (aborted) break;
        // work-item epilogue: sum of ||D||^2 of this tile over the chunk, fixed-order reduction
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) q += __shfl_xor_sync(0xffffffffu, q, off);
        if (lane == 0) red_s[warp] = q;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) t += red_s[w];
            prm.partial_q[static_cast<int64_t>(cy) * tiles_n + tile] = t;
        }
        __syncthreads();
    }

    // teardown: after an abort make sure no MMA is still writing TMEM before freeing it
    if (aborted && tid == 0) {
        tc::mma_commit(bar_done);
        tc::mbar_wait_bounded(bar_done, done_count & 1, tc::globaltimer() + ex.timeout_ns);
    }
    tc::tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, C::kTmemCols);
}

template <int MH, int BN>
cudaError_t launch_cfg(const LevelParams& prm, const TcLaunch& tl, cudaStream_t st)
{
    using C = TcCfg<MH, BN>;
    static bool attr_set = false;  // per process; the attribute is per function
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(level_tc_bf16_kernel<MH, BN>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int items = prm.nchunks * prm.tiles_m * prm.tiles_p;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, level_tc_bf16_kernel<MH, BN>, kThreads,
                                                                  C::kSmemBytes);
    if (e != cudaSuccess) return e;
    per_sm = max(1, min(per_sm, 512 / C::kTmemCols));
    const int grid = max(1, min(items, per_sm * tl.num_sms));
    TcExtra ex{tl.err_flag, tl.timeout_ns, items, tl.scale};
    level_tc_bf16_kernel<MH, BN><<<grid, kThreads, C::kSmemBytes, st>>>(prm, ex);
    return cudaGetLastError();
}

}  // namespace

TcTile tc_tile_for(int64_t m, int64_t p)
{
    TcTile t;
    t.mh = m <= 128 ? 1 : 2;
    t.bn = p <= 32 ? 32 : p <= 64 ? 64 : p <= 128 ? 128 : 256;
    t.rows = 128 * t.mh;
    return t;
}

cudaError_t launch_level_tc_bf16(const LevelParams& prm, const TcLaunch& tl, cudaStream_t st)
{
    const TcTile t = tc_tile_for(prm.m, prm.p);
    if (t.mh == 1) {
        switch (t.bn) {
            case 32: return launch_cfg<1, 32>(prm, tl, st);
            case 64: return launch_cfg<1, 64>(prm, tl, st);
            case 128: return launch_cfg<1, 128>(prm, tl, st);
            default: return launch_cfg<1, 256>(prm, tl, st);
        }
    }
    switch (t.bn) {
        case 32: return launch_cfg<2, 32>(prm, tl, st);
        case 64: return launch_cfg<2, 64>(prm, tl, st);
        case 128: return launch_cfg<2, 128>(prm, tl, st);
        default: return launch_cfg<2, 256>(prm, tl, st);
    }
}

}  // namespace mlmc
