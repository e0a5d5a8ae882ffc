// level_tc_bf16.cu -- fused level kernel on the 5th-generation tensor cores (BF16 operands,
// FP32 accumulation in tensor memory).
//
// Per sample s of level l the kernel forms D = (n/c_l) sum_t sigma_t a_t b_t^T, the coupled
// difference P_l - P_{l-1} of Alg. 1 for ratio R = 2: every slot carries weight n/c_l and the
// odd (coarse, r_{2j}) slots additionally -2 n/c_l, i.e. sigma_t = +1 for even and -1 for odd
// slots at l >= 1 (sigma = +1 at l = 0).  sigma is folded into the B operand before rounding
// (exact); the magnitude n/c_l is applied to the FP32 accumulator.
//
// Persistent CTAs of 9 warps walk (chunk of samples, output tile) work items; a sample's slots
// are processed in sub-blocks of 16 or 32 slots:
//   * producer warp (warp 8): draws the sub-block's slot indices from Philox and stages the
//     sampled (M, S) column pairs of A and (M', S') row pairs of B with TMA row gathers
//     (cp.async.bulk.tensor ... tile::gather4, four sampled rows of the interleaved parameter
//     table per instruction; plain cp.async.bulk per row when no tensor map fits the tile) into
//     a double-buffered staging area, completing on the buffer's mbarrier;
//   * generator warps (0-7): wait for the staged pairs, generate A = M + S Z and
//     sigma (M' + S' Z') with Philox and a special-function-unit Box-Muller, round them to bf16
//     (or block-quantise them to E4M3) and write them into a swizzled K-major tile; thread 0 then
//     issues tcgen05.mma into tensor memory and commits to the slice's mbarrier.  Tiles of at most
//     256 accumulator columns issue each MMA twice: into D (this sample) and into S (the running
//     sum of the chunk's samples);
//   * after the last sub-block of a sample the generator warps read D and S back with
//     tcgen05.ld and grow the chunk's M2 by Welford's update ((k + 1) D - S is k times the
//     deviation of D from the mean of the k samples before it); S is stored once per chunk as the
//     chunk partial.  The 256 x 256 single-CTA tile keeps only D in tensor memory and folds each
//     sample into the chunk partial in global memory (one owner thread per element, read back
//     and rewritten in sample order).
// CTA pairs (tiles 3256, 4256): a cluster of two CTAs shares one 256 x 256 tile, each generating
// its 128 rows of A and half of B and sending that half to the peer with a shared-to-shared bulk
// copy; in batched launches each cluster walks its own item list.
// Forms selected by template parameters: Q (bfloat16 or block-scaled E4M3 with stochastic
// rounding), F (the targeted function: fine and coarse sums in two accumulators, f applied in the
// drain), XI (the xi** law: inverse-CDF draws, per-slot weights folded into B), W (8 or 16
// generator warps), kBatch (a batched launch over many problems and levels).
// Every mbarrier wait is bounded by a %globaltimer deadline; on timeout the kernel records
// MLMC_ERR_TIMEOUT, waits (bounded) for its own copies and MMAs in flight and frees its tensor
// memory before leaving.
#include <cstring>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "rng.cuh"
#include "tc_ptx.cuh"

namespace mlmc {
namespace {

constexpr int kGenBarrier = 1;              // named barrier of the generator warps
constexpr uint64_t kDrainNs = 100000000ull;   // bound on waiting for own copies in flight after an abort

// Operand formats: Q = 0 rounds the generated entries to bfloat16; Q = 1 quantises them to FP8
// E4M3 with a power-of-two scale per (row of A or column of B, 32-slot block) and stochastic
// rounding, and feeds the dequantised values (exact in bfloat16) to the same MMA.
// P = 1: a cluster pair of CTAs shares one 256-row x BN tile; each CTA owns 128 rows (MH = 1),
// generates its rows of A and half of the B columns, and copies that half into the peer's B tile
// (one bulk shared-to-shared copy per sub-block).  Pairs keep four slices of 32 K elements in
// 64-byte-swizzled tiles (one per slice), so each CTA's half of a slice is one contiguous run and
// the peer has three sub-blocks of slack before a slice is reused.
// W: generator warps, 8 (with 8-slot items) or 16 (pairs only, tile 4256: 4-slot items, so that
// every one of the 512 generator threads takes one item of a 32-slot sub-block); plus the producer.
// F: the targeted function (0: identity; 1: |x| H(2 - x)).  F != 0 keeps the fine and the coarse
// sums apart: each 32-slot sub-block holds the even slots at K positions 0-15 and the odd (coarse)
// slots at 16-31, the first K step accumulates into E and the second into O, and the drain forms
// D = f(n/c_l (E + O)) - f(n/c_{l-1} O) and keeps the chunk's running sum S in tensor memory.
template <int MH, int BN, int Q, int P = 0, int W = 8, int F = 0>
struct TcCfg {
    static constexpr int kGW = W;                         // generator warps
    static constexpr int kGT = 32 * W;                    // generator threads
    static constexpr int kThr = kGT + 32;                  // + the producer warp
    // slots per generator item: 4 where 8 would leave too few items per sub-block to keep the
    // generator warps busy (the 16-warp pair; BF16 single-CTA tiles of at most 64 columns: +4 to
    // +12 % at 64 x 1024 x 64, while E4M3 measured -5 % at level 0 and +0.5 to +4 % above)
    static constexpr int kNS = (W == 16 || (Q == 0 && P == 0 && MH == 1 && BN <= 64)) ? 4 : 8;
    // Slots per sub-block: 32 for E4M3 (one scale block), pairs, and small tiles whose 16-slot
    // sub-block would leave generator threads idle ((rows + BN) / 4 x 2 items for 256 threads)
    static constexpr int kSub = (Q || P || 128 * MH + BN <= 256) ? 32 : 16;
    static constexpr int kKSteps = kSub / 16;              // MMA K steps per sub-block
    static constexpr int kSlices = P ? 4 : 64 / kSub;      // sub-blocks in flight (128-byte atom: 64 bf16)
    static constexpr int kRows = 128 * MH;                 // output rows of a tile
    static constexpr int kASliceBytes = kRows * 64;        // pairs: one 64-byte-swizzled slice of A
    static constexpr int kBSliceBytes = BN * 64;           // pairs: one 64-byte-swizzled slice of B
    static constexpr int kABytes = P ? kSlices * kASliceBytes : kRows * 128;   // else kRows x 64 bf16, 128-B swizzle
    static constexpr int kBBytes = P ? kSlices * kBSliceBytes : BN * 128;      // B transposed, K-major
    static constexpr int kTileBytes = kABytes + kBBytes;
    static constexpr int kBGen = P ? BN / 2 : BN;           // B columns generated (and staged) by this CTA
    static constexpr int kSlotBytes = (kRows + kBGen) * 8;  // staged FP32 (M, S) pairs of A, then of B
    static constexpr int kStageBytes = kSub * kSlotBytes;
    static constexpr int kTileCols = MH * BN;
    // Tiles of at most 256 accumulator columns also keep the chunk's running sum of D in tensor
    // memory (a second accumulator S after D); the 256 x 256 tile adds each D to global memory.
    static constexpr bool kAccS = kTileCols <= 256;
    static constexpr int kSOff = F ? 2 * kTileCols : kTileCols;   // tensor-memory column of S
    static constexpr int kAccCols = F ? 3 * kTileCols : kAccS ? 2 * kTileCols : kTileCols;
    static constexpr int kTmemCols = kAccCols <= 32 ? 32 : kAccCols <= 64 ? 64 : kAccCols <= 128 ? 128
                                     : kAccCols <= 256 ? 256 : 512;
    // barriers: full[2], empty[2], slice[kSlices], done, and for pairs peer[kSlices] (the peer's B half landed)
    static constexpr int kNumBars = 2 + 2 + kSlices + 1 + (P ? kSlices : 0) + 1 /*abort drain*/;
    static constexpr int kBookBytes = 2 * kSub * 4 /*idx*/ + 2 * 2 * kSub * 4 /*idx per packed half*/ +
                                      2 * kSub * 4 /*xi** slot weights*/ +
                                      kNumBars * 8 + 16 /*tmem, abort*/ + kGW * 8 +
                                      (P ? 0 : 2 * static_cast<int>(sizeof(LevelParams)) +
                                                   static_cast<int>(alignof(LevelParams)))
                                      /*job copies of batched launches (pairs read the job table)*/;
    static constexpr int kSmemBytes = 1024 /*align slack*/ + kTileBytes + 2 * kStageBytes + kBookBytes;
    static_assert(kAccCols <= 512, "tile exceeds tensor memory");
    static_assert(kTmemCols >= kAccCols, "the allocation holds the accumulators");
    static_assert(kKSteps * 16 == kSub, "a sub-block is a whole number of K = 16 MMA steps");
    static_assert(BN % 16 == 0 && BN >= 32 && BN <= 256, "N of the MMA");
    static constexpr bool kFits = kSmemBytes <= 227 * 1024 &&   // E4M3's 32-slot staging rules out wide tiles
                                  (!P || (MH == 1 && BN == 256)) && (W == 8 || (W == 16 && P)) &&
                                  (F == 0 || (MH == 1 && BN <= 128 && Q == 0 && P == 0 && W == 8 && kSub == 32));

};

struct TcExtra {
    int* err_flag;
    uint64_t timeout_ns;
    int total_items;  // nchunks * tiles
    float scale;      // n / c_l
};

// The targeted function in FP32: F = 1 is |x| H(2 - x) with H(0) = 1; F = 0 the identity.
template <int F>
__device__ __forceinline__ float tc_targeted(float x)
{
    if constexpr (F == 1) return (2.0f - x >= 0.0f) ? fabsf(x) : 0.0f;
    return x;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

// Generate one block of (4 rows of A, or 4 columns of B) x (NS = 8 or 4 slots) entries from staged
// (M, S) pairs and write them as bf16 into the swizzled tile: tile rows row0 .. row0+3, 16-byte
// chunk `chunk` (NS = 4: its half `sub`, 8 bytes).  Staged pairs of slot u start at
// stage + u * stride (8 floats: (M,S) x 4).  kSw: the tile's swizzle, 128 or 64 bytes per row.
template <int kSw>
__device__ __forceinline__ uint32_t tile_offset(int row, int chunk)
{
    return kSw == 128 ? tc::sw128_offset(row, chunk) : tc::sw64_offset(row, chunk);
}

// kWt: each slot's entries are also multiplied by its weight gw[slot] (xi**: Q_{n-1} / q_k) before
// rounding.  kSkip: an item without any slot writes zeros without drawing (tiles that pack samples).
template <int kSw = 128, int NS = 8, bool kWt = false, bool kSkip = false>
__device__ __forceinline__ void gen_block(const int* idx, int slot0, bool valid_rows, uint32_t rowgrp,
                                          uint32_t s_lo, uint32_t lsw, const PhiloxRoundKeys& rk,
                                          const unsigned char* stage,
                                          int stride, bool odd_negative, unsigned char* tile, int row0, int chunk,
                                          int sub = 0, const float* gw = nullptr)
{
    static_assert(NS == 8 || NS == 4, "slots per item");
    if (!valid_rows) {
        // padding rows (or columns) of the tile: zeros, no random numbers needed
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            if constexpr (NS == 8)
                *reinterpret_cast<uint4*>(tile + tile_offset<kSw>(row0 + r, chunk)) = make_uint4(0, 0, 0, 0);
            else
                *reinterpret_cast<uint2*>(tile + tile_offset<kSw>(row0 + r, chunk) + sub) = make_uint2(0, 0);
        }
        return;
    }
    // Branch-free: the Philox blocks are independent dependency chains, computed for every slot
    // (a missing slot uses k = 0) and zeroed afterwards, so they can interleave.  With kSkip, an
    // item without any slot (a packed half's K positions of the other sample, the tail of the last
    // sub-block) only writes zeros.
    int ks[NS];
    uint4 w[NS];
    if constexpr (kSkip) {
        bool any = false;
#pragma unroll
        for (int u = 0; u < NS; ++u) {
            ks[u] = idx[slot0 + u];
            any |= ks[u] >= 0;
        }
        if (!any) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                if constexpr (NS == 8)
                    *reinterpret_cast<uint4*>(tile + tile_offset<kSw>(row0 + r, chunk)) = make_uint4(0, 0, 0, 0);
                else
                    *reinterpret_cast<uint2*>(tile + tile_offset<kSw>(row0 + r, chunk) + sub) = make_uint2(0, 0);
            }
            return;
        }
#pragma unroll
        for (int u = 0; u < NS; ++u)
            w[u] = philox4x32_10_rk(make_uint4(rowgrp, static_cast<uint32_t>(max(ks[u], 0)), s_lo, lsw), rk);
    } else {
#pragma unroll
        for (int u = 0; u < NS; ++u) {
            ks[u] = idx[slot0 + u];
            w[u] = philox4x32_10_rk(make_uint4(rowgrp, static_cast<uint32_t>(max(ks[u], 0)), s_lo, lsw), rk);
        }
    }
    float v[4][NS];
#pragma unroll
    for (int u = 0; u < NS; ++u) {
        float z[4];
        normals4_mufu(w[u], z);
        const float4* src = reinterpret_cast<const float4*>(stage + u * stride);
        const float4 p0 = src[0];
        const float4 p1 = src[1];
        const bool use = ks[u] >= 0;
        float sg = (odd_negative && (u & 1)) ? -1.0f : 1.0f;
        if constexpr (kWt) sg *= gw[slot0 + u];
        v[0][u] = use ? sg * fmaf(p0.y, z[0], p0.x) : 0.0f;
        v[1][u] = use ? sg * fmaf(p0.w, z[1], p0.z) : 0.0f;
        v[2][u] = use ? sg * fmaf(p1.y, z[2], p1.x) : 0.0f;
        v[3][u] = use ? sg * fmaf(p1.w, z[3], p1.z) : 0.0f;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        if constexpr (NS == 8) {
            const uint4 packed = make_uint4(pack_bf16x2(v[r][0], v[r][1]), pack_bf16x2(v[r][2], v[r][3]),
                                            pack_bf16x2(v[r][4], v[r][5]), pack_bf16x2(v[r][6], v[r][7]));
            *reinterpret_cast<uint4*>(tile + tile_offset<kSw>(row0 + r, chunk)) = packed;
        } else {
            const uint2 packed = make_uint2(pack_bf16x2(v[r][0], v[r][1]), pack_bf16x2(v[r][2], v[r][3]));
            *reinterpret_cast<uint2*>(tile + tile_offset<kSw>(row0 + r, chunk) + sub) = packed;
        }
    }
}

// E4M3 form of gen_block for 32-slot sub-blocks: the four adjacent lanes of one row group hold
// the row's 32 slots (8 each).  Each row's block maximum |x| gives the scale 2^e, e the
// smallest integer with max <= 448 * 2^e (1 for an all-zero block); x / 2^e is rounded to E4M3
// stochastically (e4m3_round_sr, with the entry's 16-bit dither) and the dequantised value,
// exact in bfloat16, is stored.  Every lane of the warp must call this together (shuffles).
__device__ __forceinline__ float e4m3_block_scale(float absmax)
{
    if (!(absmax > 0.0f)) return 1.0f;
    int e = ((__float_as_uint(absmax) >> 23) & 0xFF) - 127 - 9;   // absmax is a normal float here
    while (absmax > ldexpf(448.0f, e)) ++e;
    return ldexpf(1.0f, e);
}

// Stochastic rounding of y (|y| <= 448) to the E4M3 grid: with lo <= |y| < lo + h the two grid
// neighbours (h the spacing: 2^(e-3) for |y| in [2^e, 2^(e+1)), e >= -6; 2^-9 below 2^-6), the
// result is lo + h when (d + 1/2) 2^-16 < (|y| - lo) / h, else lo, with the sign of y -- unbiased
// over a uniform 16-bit dither d up to 2^-17 h.  Every step is exact in FP32 (h is a power of
// two, (|y| - lo) / h has at most 20 fraction bits).
__device__ __forceinline__ float e4m3_round_sr(float y, uint32_t d)
{
    const float ay = fabsf(y);
    int e = static_cast<int>((__float_as_uint(ay) >> 23) & 0xFFu) - 127;
    e = max(e, -6);
    const float h = __uint_as_float(static_cast<uint32_t>(e - 3 + 127) << 23);
    const float inv_h = __uint_as_float(static_cast<uint32_t>(127 - (e - 3)) << 23);
    const float t = ay * inv_h;
    const float fl = floorf(t);
    const float up = ((t - fl) * 65536.0f > static_cast<float>(d) + 0.5f) ? 1.0f : 0.0f;
    return copysignf((fl + up) * h, y);
}

// kTglob0: the absolute slot of the first of the 8 slots (even), for the dither counters
// (row group, 2^31 + slot / 2, s_lo, level word): word r of the block serves row r of the group,
// its low half the even slot and its high half the odd one.
template <int kSw = 128, int NS = 8>
__device__ __forceinline__ void gen_block_e4m3(const int* idx, int slot0, bool valid_rows, uint32_t rowgrp,
                                               uint32_t s_lo, uint32_t lsw, const PhiloxRoundKeys& rk,
                                               const unsigned char* stage, int stride, bool odd_negative,
                                               unsigned char* tile, int row0, int chunk, int tglob0,
                                               bool split16 = false, int sub = 0)
{
    // NS slots per lane: the 32 slots of a row's block sit in 32 / NS adjacent lanes
    static_assert(NS == 8 || NS == 4, "slots per item");
    float v[4][NS];
    if (valid_rows) {
        int ks[NS];
        uint4 w[NS];
#pragma unroll
        for (int u = 0; u < NS; ++u) {
            ks[u] = idx[slot0 + u];
            w[u] = philox4x32_10_rk(make_uint4(rowgrp, static_cast<uint32_t>(max(ks[u], 0)), s_lo, lsw), rk);
        }
#pragma unroll
        for (int u = 0; u < NS; ++u) {
            float z[4];
            normals4_mufu(w[u], z);
            const float4* src = reinterpret_cast<const float4*>(stage + u * stride);
            const float4 p0 = src[0];
            const float4 p1 = src[1];
            const bool use = ks[u] >= 0;
            const float sg = (odd_negative && (u & 1)) ? -1.0f : 1.0f;
            v[0][u] = use ? sg * fmaf(p0.y, z[0], p0.x) : 0.0f;
            v[1][u] = use ? sg * fmaf(p0.w, z[1], p0.z) : 0.0f;
            v[2][u] = use ? sg * fmaf(p1.y, z[2], p1.x) : 0.0f;
            v[3][u] = use ? sg * fmaf(p1.w, z[3], p1.z) : 0.0f;
        }
    } else {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int u = 0; u < NS; ++u) v[r][u] = 0.0f;
    }
    // dithers of the 4 rows x NS slots: one Philox block per slot pair
    uint4 dith[NS / 2];
#pragma unroll
    for (int u2 = 0; u2 < NS / 2; ++u2)
        dith[u2] = valid_rows ? philox4x32_10_rk(make_uint4(rowgrp, 0x80000000u | static_cast<uint32_t>((tglob0 >> 1) + u2),
                                                            s_lo, lsw),
                                                 rk)
                              : make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        float am = 0.0f;
#pragma unroll
        for (int u = 0; u < NS; ++u) am = fmaxf(am, fabsf(v[r][u]));
        // the block's maximum over its lanes (split16: slots 0-15 and 16-31 are blocks of two samples)
        constexpr int kLanes = 32 / NS;
#pragma unroll
        for (int x = 1; x < kLanes; x <<= 1) {
            const float other = __shfl_xor_sync(0xffffffffu, am, x);
            if (!split16 || 2 * x < kLanes) am = fmaxf(am, other);
        }
        const float sc = e4m3_block_scale(am);
        const float inv = 1.0f / sc;   // exact: a power of two
        uint32_t packed[NS / 2];
#pragma unroll
        for (int u2 = 0; u2 < NS / 2; ++u2) {
            const uint32_t word = r == 0 ? dith[u2].x : r == 1 ? dith[u2].y : r == 2 ? dith[u2].z : dith[u2].w;
            const float q0 = e4m3_round_sr(v[r][2 * u2] * inv, word & 0xFFFFu);
            const float q1 = e4m3_round_sr(v[r][2 * u2 + 1] * inv, word >> 16);
            packed[u2] = pack_bf16x2(q0 * sc, q1 * sc);
        }
        if constexpr (NS == 8)
            *reinterpret_cast<uint4*>(tile + tile_offset<kSw>(row0 + r, chunk)) =
                make_uint4(packed[0], packed[1], packed[2], packed[3]);
        else
            *reinterpret_cast<uint2*>(tile + tile_offset<kSw>(row0 + r, chunk) + sub) = make_uint2(packed[0], packed[1]);
    }
}

// prm.pack: two samples share one accumulator (problems with m <= 64 on a 128-row tile): rows 0-63
// hold the first sample of a group and rows 64-127 the second; the group's K positions are the
// first sample's c_l slots followed by the second's, and each half of A is zero on the other
// sample's positions, so one MMA chain forms both samples' D.  Each half keeps its own running
// sum (rows of S) and Welford M2; at the end of a chunk the halves are combined by Chan's update.
// Needs c_l % 16 == 0 (a group of 8 slots, and an E4M3 block, never straddles two samples).
// XI: the xi** law (Thm 3.1): the producer draws each slot by inverse CDF and stores its weight
// Q_{n-1} / q_k, which the generators fold into B; the accumulator is scaled by 1 / c_l.
template <int MH, int BN, int Q, bool kBatch, int P = 0, int W = 8, int F = 0, bool XI = false>
__global__ void __launch_bounds__(TcCfg<MH, BN, Q, P, W, F>::kThr, 1)
level_tc_bf16_kernel(const __grid_constant__ LevelParams prm_arg, const TcExtra ex, const TcBatch bt)
{
    using C = TcCfg<MH, BN, Q, P, W, F>;
    static_assert(!XI || (Q == 0 && !kBatch), "xi** runs BF16 single-problem launches");
    // tiles that pack two samples per accumulator skip the items of the other sample's positions
    constexpr bool kSkip = P == 0 && MH == 1 && BN <= 64;
    constexpr int kGenWarps = C::kGW;
    constexpr int kGenThreads = C::kGT;
    constexpr int kNS = C::kNS;
    // columns per TMEM read in the drains: the 16-warp form has fewer registers a thread
    constexpr int kCW = W == 16 ? 32 : 64;
    static_assert(C::kFits, "shared memory");
    constexpr int kSub = C::kSub;
    constexpr int kSlices = C::kSlices;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~static_cast<uintptr_t>(1023));
    unsigned char* a_tile = smem;
    unsigned char* b_tile = smem + C::kABytes;
    unsigned char* staging = smem + C::kTileBytes;  // [2][kStageBytes]
    int* idx_s = reinterpret_cast<int*>(staging + 2 * C::kStageBytes);  // [2][kSub]
    int* idxh_s = idx_s + 2 * kSub;   // PK: [2 buffers][2 halves][kSub], -1 on the other sample's slots
    uint64_t* bars = reinterpret_cast<uint64_t*>(idxh_s + 4 * kSub);
    uint32_t* tmem_s = reinterpret_cast<uint32_t*>(bars + C::kNumBars);
    volatile int* abort_s = reinterpret_cast<volatile int*>(tmem_s + 1);
    double* red_s = reinterpret_cast<double*>(tmem_s + 4);
    float* gw_s = reinterpret_cast<float*>(red_s + kGenWarps);   // xi**: [2][kSub] slot weights Q_{n-1} / q_k
    // batched launches: each role keeps its own copy of the current job's parameters (aligned as
    // the type requires: it embeds tensor maps)
    LevelParams* job_prod = reinterpret_cast<LevelParams*>(
        (reinterpret_cast<uintptr_t>(gw_s + 2 * kSub) + alignof(LevelParams) - 1) &
        ~static_cast<uintptr_t>(alignof(LevelParams) - 1));
    LevelParams* job_gen = job_prod + 1;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const uint32_t bars0 = tc::smem_addr(bars);
    const uint32_t bar_done = bars0 + 8 * (4 + kSlices);
    auto bar_full = [&](int b) { return bars0 + 8 * b; };
    auto bar_empty = [&](int b) { return bars0 + 8 * (2 + b); };
    auto bar_slice = [&](int kk) { return bars0 + 8 * (4 + kk); };
    auto bar_peer = [&](int kk) { return bars0 + 8 * (4 + kSlices + 1 + kk); };
    const uint32_t bar_quiesce = bars0 + 8 * (C::kNumBars - 1);   // used once, after an abort
    const uint32_t crank = P ? tc::cluster_ctarank() : 0u;   // this CTA's half of a pair
    const uint32_t peer = crank ^ 1u;

    if (warp == 0) tc::tmem_alloc(tc::smem_addr(tmem_s), C::kTmemCols);
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(bar_full(b), 1);
            tc::mbar_init(bar_empty(b), kGenWarps);
        }
        // a slice is free again once this CTA's MMA and, for pairs, the peer's MMA have read it
        for (int kk = 0; kk < kSlices; ++kk) tc::mbar_init(bar_slice(kk), P ? 2 : 1);
        tc::mbar_init(bar_done, 1);
        tc::mbar_init(bar_quiesce, 1);
        if constexpr (P)
            for (int kk = 0; kk < kSlices; ++kk) tc::mbar_init(bar_peer(kk), 1);
        tc::mbar_init_fence();
        *abort_s = 0;
    }
    tc::tc_fence_before_sync();
    __syncthreads();
    if constexpr (P) tc::cluster_sync();   // the peer's barriers exist before anything reaches them
    tc::tc_fence_after_sync();
    const uint32_t tmem = *tmem_s;
    // pairs: the peer's B tile in the cluster's shared window
    const uint32_t peer_b_tile = P ? tc::map_to_cta(tc::smem_addr(b_tile), peer) : 0u;

    // Work items: (chunk cy, output tile) of the launch's level, or, in a batched launch, the
    // CTA's list of (job, chunk, tile) items prepared by the host.
    auto for_each_item = [&](LevelParams* copy, auto&& body_fn, bool whole_cta) {
        if constexpr (kBatch) {
            int cur = -1;
            // pairs: both CTAs of a cluster walk the cluster's list (the same items in the same
            // order); an item's tile is then a pair of row tiles and a column tile
            const int unit = P ? static_cast<int>(blockIdx.x >> 1) : static_cast<int>(blockIdx.x);
            const int i0 = bt.cta_begin[unit], i1 = bt.cta_begin[unit + 1];
            for (int i = i0; i < i1; ++i) {
                const uint64_t it = bt.items[i];
                const int job = static_cast<int>(it & 0xFFFFu);
                if (!P && job != cur) {
                    const uint32_t* src = reinterpret_cast<const uint32_t*>(bt.jobs + job);
                    uint32_t* dst = reinterpret_cast<uint32_t*>(copy);
                    const int nthr = whole_cta ? kGenThreads : 32;
                    const int me = whole_cta ? tid : lane;
                    for (int w = me; w < static_cast<int>(sizeof(LevelParams) / 4); w += nthr) dst[w] = src[w];
                    if (whole_cta)
                        tc::named_barrier(kGenBarrier, kGenThreads);
                    else
                        __syncwarp();
                    cur = job;
                }
                // chunk run: first chunk in bits 16-39, run length in bits 40-47
                const int cy0 = static_cast<int>((it >> 16) & 0xFFFFFFu);
                const int ncy = static_cast<int>((it >> 40) & 0xFFu);
                const int tile = static_cast<int>(it >> 48);
                bool go = true;
                // tensor maps are read from the job table in global memory (not the shared copy)
                const TcMaps* maps = &bt.jobs[job].maps;
                // pairs keep no shared copy (their shared memory is full): they read the job's
                // parameters from the table in global memory
                const LevelParams& jp = P ? bt.jobs[job] : *copy;
                for (int cy = cy0; cy < cy0 + ncy && go; ++cy) go = body_fn(jp, cy, tile, maps);
                if (!go) break;
            }
        } else if constexpr (P) {
            // both CTAs of a cluster walk the same (chunk, pair of row tiles, column tile) items
            const int pair_tiles = ((prm_arg.tiles_m + 1) / 2) * prm_arg.tiles_p;
            const int total = prm_arg.nchunks * pair_tiles;
            const int cid = static_cast<int>(blockIdx.x >> 1), ncl = static_cast<int>(gridDim.x >> 1);
            for (int item = cid; item < total; item += ncl)
                if (!body_fn(prm_arg, item / pair_tiles, item % pair_tiles, &prm_arg.maps)) break;
        } else {
            const int tiles_n = prm_arg.tiles_m * prm_arg.tiles_p;
            const int total = prm_arg.nchunks * tiles_n;
            for (int item = blockIdx.x; item < total; item += gridDim.x)
                if (!body_fn(prm_arg, item / tiles_n, item % tiles_n, &prm_arg.maps)) break;
        }
    };

    // Tile geometry of an item: first row and column, the column of this CTA's generated B part,
    // and the (chunk, tile) index of its sum of squares (-1: a pair's row tile beyond m).
    struct Geo {
        int tm0, tp0, bcol0, qtile;
    };
    auto geometry = [&](const LevelParams& prm, int tile) {
        Geo g;
        if constexpr (P) {
            const int prow = tile / prm.tiles_p, col = tile % prm.tiles_p;
            const int row_idx = 2 * prow + static_cast<int>(crank);
            g.tm0 = row_idx * C::kRows;
            g.tp0 = col * BN;
            g.bcol0 = g.tp0 + static_cast<int>(crank) * C::kBGen;
            g.qtile = row_idx < prm.tiles_m ? row_idx * prm.tiles_p + col : -1;
        } else {
            g.tm0 = (tile / prm.tiles_p) * C::kRows;
            g.tp0 = (tile % prm.tiles_p) * BN;
            g.bcol0 = g.tp0;
            g.qtile = tile;
        }
        return g;
    };

    if (warp == kGenWarps) {
        // ---------------- producer warp: indices + TMA bulk copies of the sampled pairs ----------
        uint32_t g = 0;  // sub-blocks produced by this CTA
        bool aborted = false;
        const TcMaps* fenced = nullptr;   // batched: job-table maps already acquired by this warp
        for_each_item(job_prod, [&](const LevelParams& prm, int cy, int tile, const TcMaps* maps) -> bool {
            if constexpr (kBatch) {
                // the job table is rewritten between batched calls: reload cached descriptors
                if (maps != fenced && prm.maps.valid) {
                    tc::tensormap_acquire(&maps->a);
                    tc::tensormap_acquire(&maps->b);
                    fenced = maps;
                }
            }
            const int tiles_n = prm.tiles_m * prm.tiles_p;
            const float* PA = static_cast<const float*>(prm.PA);
            const float* PB = static_cast<const float*>(prm.PB);
            const int nsub = (prm.c + kSub - 1) / kSub;
            const Geo geo = geometry(prm, tile);
            const int tm0 = geo.tm0;
            const uint32_t a_bytes = static_cast<uint32_t>(max(0, min(C::kRows, prm.m_pad - tm0))) * 8u;
            const uint32_t b_bytes = static_cast<uint32_t>(max(0, min(C::kBGen, prm.p_pad - geo.bcol0))) * 8u;
            (void)tiles_n;
            (void)PB;
            // row gathers need maps encoded for exactly this tile's staging widths
            const bool gather = prm.maps.valid != 0 && prm.maps.wa == C::kRows && prm.maps.wb == C::kBGen;
            const uint64_t chunk = prm.chunk0 + static_cast<uint64_t>(cy);
            const uint64_t sa = max(prm.s_begin, chunk * static_cast<uint64_t>(prm.chunk));
            const uint64_t sb = min(prm.s_end, (chunk + 1) * static_cast<uint64_t>(prm.chunk));
            const bool PK = MH == 1 && P == 0 && F == 0 && prm.pack != 0;   // packed samples (uniform per item)
            const uint64_t kG = PK ? 2 : 1;                        // samples per accumulator
            for (uint64_t s = sa; s < sb && !aborted; s += kG) {
                const uint32_t lsw = level_sample_word(prm.l, s);
                const uint32_t s_lo = static_cast<uint32_t>(s);
                const int ngrp = (PK && sb - s >= 2) ? 2 : 1;   // samples in this group
                const int nK = prm.c * ngrp;                                             // K positions
                const int nsubg = PK ? (nK + kSub - 1) / kSub : nsub;
                for (int j = 0; j < nsubg; ++j, ++g) {
                    const int b = static_cast<int>(g & 1);
                    const int t0 = j * kSub;
                    // this sub-block's draws, made before waiting for staging buffer b (they do not
                    // touch it): the table walks of xi** and the Philox blocks of the indices run
                    // while the generators still use the buffer
                    int dr0 = -1, dr1 = -1, dh = 0;
                    float dg = 0.0f;
                    if (XI) {
                        // xi** (Thm 3.1): one slot per lane (a draw walks the tables with dependent
                        // loads: 32 walks in parallel), inverse-CDF index and weight Q_{n-1} / q_k.
                        // K position kp holds slot kp (PK: sample s + kp / c_l, slot kp mod c_l)
                        if (lane < kSub) {
                            const int kp = t0 + lane;
                            dh = (PK && kp < nK) ? kp / prm.c : 0;
                            const int t = kp - dh * prm.c;
                            if (kp < nK) {
                                const uint64_t sh = s + static_cast<uint64_t>(dh);
                                uint64_t w0, w1;
                                index_words(prm.keyI, level_sample_word(prm.l, sh), static_cast<uint32_t>(sh), t >> 1,
                                            w0, w1);
                                dr0 = static_cast<int>(index_from_cdf((t & 1) ? w1 : w0, prm.xi_Q, prm.xi_q, prm.xi_G,
                                                                      prm.n));
                                dg = static_cast<float>(__ddiv_rn(prm.xi_Qtot, prm.xi_q[dr0]));
                            }
                        }
                    } else if (PK) {
                        // K position kp -> sample s + h (h = kp / c_l), slot kp - h c_l; c_l is even, so a
                        // slot pair never straddles the two samples
                        if (lane < kSub / 2) {
                            const int kp = t0 + 2 * lane;
                            dh = kp < nK ? kp / prm.c : 0;
                            if (kp < nK) {
                                const uint64_t sh = s + static_cast<uint64_t>(dh);
                                int64_t r0, r1;
                                index_pair(prm.keyI, level_sample_word(prm.l, sh), static_cast<uint32_t>(sh),
                                           (kp - dh * prm.c) >> 1, static_cast<uint64_t>(prm.n), r0, r1);
                                dr0 = static_cast<int>(r0);
                                dr1 = static_cast<int>(r1);
                            }
                        }
                    } else if (lane < kSub / 2) {
                        const int t = t0 + 2 * lane;
                        if (t < prm.c) {
                            int64_t r0, r1;
                            index_pair(prm.keyI, lsw, s_lo, t >> 1, static_cast<uint64_t>(prm.n), r0, r1);
                            dr0 = static_cast<int>(r0);
                            dr1 = t + 1 < prm.c ? static_cast<int>(r1) : -1;
                        }
                    }
                    if (g >= 2 && !tc::mbar_wait_bounded(bar_empty(b), ((g >> 1) - 1) & 1,
                                                         tc::globaltimer() + ex.timeout_ns)) {
                        *abort_s = 1;
                        atomicExch(ex.err_flag, MLMC_ERR_TIMEOUT);
                    }
                    if (__any_sync(0xffffffffu, *abort_s != 0)) {
                        aborted = true;
                        break;
                    }
                    int* idx = idx_s + b * kSub;
                    if (XI) {
                        // F != 0: even slots at positions 0-15, odd slots at 16-31
                        if (lane < kSub) {
                            const int pos = F ? ((lane & 1) ? kSub / 2 + (lane >> 1) : (lane >> 1)) : lane;
                            idx[pos] = dr0;
                            gw_s[b * kSub + pos] = dg;
                            if (PK) {
                                int* ih = idxh_s + b * 2 * kSub;
                                ih[lane] = dh == 0 ? dr0 : -1;
                                ih[kSub + lane] = dh == 1 ? dr0 : -1;
                            }
                        }
                    } else if (PK) {
                        if (lane < kSub / 2) {
                            idx[2 * lane] = dr0;
                            idx[2 * lane + 1] = dr1;
                            int* ih = idxh_s + b * 2 * kSub;
                            ih[2 * lane] = dh == 0 ? dr0 : -1;
                            ih[2 * lane + 1] = dh == 0 ? dr1 : -1;
                            ih[kSub + 2 * lane] = dh == 1 ? dr0 : -1;
                            ih[kSub + 2 * lane + 1] = dh == 1 ? dr1 : -1;
                        }
                    } else if (lane < kSub / 2) {
                        // F != 0: even slot t at K position lane, odd slot t + 1 at 16 + lane
                        const int p0 = F ? lane : 2 * lane, p1 = F ? kSub / 2 + lane : 2 * lane + 1;
                        idx[p0] = dr0;
                        idx[p1] = dr1;
                    }
                    __syncwarp();
                    const int nvalid = min(kSub, nK - t0);
                    // staging buffer b: the A parts of the kSub slots, then their B parts
                    unsigned char* stg = staging + b * C::kStageBytes;
                    const uint32_t a_region = tc::smem_addr(stg);
                    const uint32_t b_region = a_region + static_cast<uint32_t>(kSub * C::kRows * 8);
                    if (gather) {
                        // TMA row gathers, four slots per instruction (boxes of kRows and kBGen pairs);
                        // F != 0: the valid K positions are a prefix of each 16-position half
                        const int ga = F ? (min(kSub / 2, (nvalid + 1) / 2) + 3) / 4 : (nvalid + 3) / 4;
                        const int groups = F ? ga + (min(kSub / 2, nvalid / 2) + 3) / 4 : ga;
                        if (lane == 0)
                            tc::mbar_arrive_expect_tx(bar_full(b),
                                                      static_cast<uint32_t>(groups * 4 * (C::kRows + C::kBGen) * 8));
                        __syncwarp();
                        if (lane < groups) {
                            const int gq = (F && lane >= ga) ? kSub / 8 + (lane - ga) : lane;   // group of 4 positions
                            const int r0 = max(idx[4 * gq], 0), r1 = max(idx[4 * gq + 1], 0);
                            const int r2 = max(idx[4 * gq + 2], 0), r3 = max(idx[4 * gq + 3], 0);
                            tc::tma_gather4(a_region + static_cast<uint32_t>(4 * gq * C::kRows * 8), &maps->a, tm0,
                                            r0, r1, r2, r3, bar_full(b));
                            tc::tma_gather4(b_region + static_cast<uint32_t>(4 * gq * C::kBGen * 8), &maps->b,
                                            prm.m_pad + geo.bcol0, r0, r1, r2, r3, bar_full(b));
                        }
                    } else {
                        if (lane == 0)
                            tc::mbar_arrive_expect_tx(bar_full(b), static_cast<uint32_t>(nvalid) * (a_bytes + b_bytes));
                        __syncwarp();
                        if (F ? (lane < kSub && idx[lane] >= 0) : lane < nvalid) {
                            const int k = idx[lane];
                            const float* row = PA + static_cast<int64_t>(k) * prm.ldPA;
                            if (a_bytes)
                                tc::bulk_copy_g2s(a_region + static_cast<uint32_t>(lane * C::kRows * 8), row + 2 * tm0,
                                                  a_bytes, bar_full(b));
                            if (b_bytes)
                                tc::bulk_copy_g2s(b_region + static_cast<uint32_t>(lane * C::kBGen * 8),
                                                  row + 2 * (prm.m_pad + geo.bcol0), b_bytes, bar_full(b));
                        }
                    }
                    __syncwarp();
                }
            }
            return !aborted;
        }, false);
        if (aborted) {
            // copies issued for the last two sub-blocks may still be landing in the staging buffers:
            // wait for them (bounded) before this CTA can exit
            for (uint32_t gp = g >= 2 ? g - 2 : 0; gp < g; ++gp)
                tc::mbar_wait_bounded(bar_full(static_cast<int>(gp & 1)), (gp >> 1) & 1,
                                      tc::globaltimer() + kDrainNs);
        }
    } else if (warp < kGenWarps) {
        // ---------------- generator warps: entries, MMA issue, drain ----------------------------
        constexpr uint32_t idesc = tc::idesc_bf16_f32(128, BN);
        constexpr int kItemsA = (C::kRows / 4) * (kSub / kNS);
        constexpr int kItemsB = (C::kBGen / 4) * (kSub / kNS);
        uint32_t g = 0;  // sub-blocks consumed
        uint32_t peer_par = 0;    // bit kk: parity of the peer's arrivals on peer barrier kk (pairs)
        int peer_armed = -1;      // pairs, thread 0: slice whose peer copy is expected but not yet waited for
        uint32_t slice_par = 0;   // bit kk: parity of the MMAs issued on slice kk so far
        uint32_t slice_seen = 0;  // bit kk: slice kk has been used
        uint32_t done_count = 0;
        bool aborted = false;
        for_each_item(job_gen, [&](const LevelParams& prm, int cy, int tile, const TcMaps*) -> bool {
            const int tiles_n = prm.tiles_m * prm.tiles_p;
            const int nsub = (prm.c + kSub - 1) / kSub;
            const bool coarse_sign = F == 0 && prm.l > 0;   // F != 0 keeps the coarse sum apart instead
            // n / c_l; xi** folds Q_{n-1} / q_k into B and leaves 1 / c_l
            const float scale = XI ? static_cast<float>(1.0 / static_cast<double>(prm.c))
                                         : static_cast<float>(prm.w_fine);
            const Geo geo = geometry(prm, tile);
            const int tm0 = geo.tm0;
            const int tp0 = geo.tp0;
            const int brow0 = geo.bcol0 - tp0;   // first row of this CTA's part of the transposed B tile
            const uint64_t chunk = prm.chunk0 + static_cast<uint64_t>(cy);
            const uint64_t sa = max(prm.s_begin, chunk * static_cast<uint64_t>(prm.chunk));
            const uint64_t sb = min(prm.s_end, (chunk + 1) * static_cast<uint64_t>(prm.chunk));
            float* part = static_cast<float*>(prm.partial_sum) + static_cast<int64_t>(cy) * prm.m * prm.p;
            double q = 0.0;    // chunk-level terms (scaled)
            float qw = 0.0f;   // Welford terms of the chunk's samples, FP32 (unscaled on tiles that keep S)
            const double scale_sq = static_cast<double>(scale) * static_cast<double>(scale);
            // Drain mapping.  MH == 2: warp group h reads M-half h (all BN columns); MH == 1: the two
            // warp groups split the columns, or group 0 takes all of them when BN < 64.
            struct Drain {
                int quarter, col_tm, col_d, ncols, gi;
                __device__ uint32_t taddr(uint32_t base, int cb) const
                {
                    return base + (static_cast<uint32_t>(quarter * 32) << 16) + static_cast<uint32_t>(col_tm + cb);
                }
            } dr;
            {
                const int hgrp = warp >> 2;                 // 0 .. kGenWarps / 4 - 1
                constexpr int kSplit = kGenWarps / 4;        // column groups of a 128-row tile
                const bool split = MH == 1 && BN >= 32 * kSplit;
                dr.quarter = warp & 3;
                dr.col_tm = MH == 2 ? hgrp * BN : (split ? hgrp * (BN / kSplit) : 0);
                dr.col_d = MH == 2 ? 0 : dr.col_tm;
                dr.ncols = MH == 2 ? BN : (split ? BN / kSplit : (hgrp == 0 ? BN : 0));
                dr.gi = tm0 + (MH == 2 ? hgrp * 128 : 0) + dr.quarter * 32 + lane;
            }
            const bool PK = MH == 1 && P == 0 && F == 0 && prm.pack != 0;   // packed samples (uniform per item)
            const uint64_t kG = PK ? 2 : 1;
            if (PK) dr.gi = (dr.quarter & 1) * 32 + lane;          // rows 64-127: the second sample
            const int pk_half = PK ? (warp & 3) >> 1 : 0;           // the sample of this warp's drained rows
            // Write (first sample of the chunk) or fold 64 drained, scaled columns starting at column
            // cb of this thread's row into the chunk partial: each element has one owner thread, so
            // the partial is read back and rewritten in a fixed order.  Folding returns the sum of
            // (k D - sum_k)^2 over the columns (k samples folded before: Welford's update of the
            // chunk's M2, the caller divides by k (k + 1)).
            auto store_cols = [&](const float* v, int cb, int nv, int kbefore) -> float {
                float qs = 0.0f;
                const float kf = static_cast<float>(kbefore);
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const int gj0 = tp0 + dr.col_d + cb + 32 * half;
                    if (32 * half >= nv || dr.gi >= prm.m || gj0 >= prm.p) continue;
                    float* dst = part + static_cast<int64_t>(dr.gi) * prm.p + gj0;
                    const float* w = v + 32 * half;
                    const int valid = min(32, prm.p - gj0);
                    if (valid == 32 && (prm.p & 3) == 0) {
#pragma unroll
                        for (int e4 = 0; e4 < 8; ++e4) {
                            float4 x = make_float4(w[4 * e4], w[4 * e4 + 1], w[4 * e4 + 2], w[4 * e4 + 3]);
                            if (kbefore > 0) {
                                const float4 pv = reinterpret_cast<const float4*>(dst)[e4];
                                const float d0 = fmaf(kf, x.x, -pv.x), d1 = fmaf(kf, x.y, -pv.y);
                                const float d2 = fmaf(kf, x.z, -pv.z), d3 = fmaf(kf, x.w, -pv.w);
                                qs = fmaf(d0, d0, fmaf(d1, d1, fmaf(d2, d2, fmaf(d3, d3, qs))));
                                x = make_float4(pv.x + x.x, pv.y + x.y, pv.z + x.z, pv.w + x.w);
                            }
                            reinterpret_cast<float4*>(dst)[e4] = x;
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < 32; ++e)
                            if (e < valid) {
                                float x = w[e];
                                if (kbefore > 0) {
                                    const float pv = dst[e];
                                    const float d = fmaf(kf, x, -pv);
                                    qs = fmaf(d, d, qs);
                                    x += pv;
                                }
                                dst[e] = x;
                            }
                    }
                }
                return qs;
            };
            for (uint64_t s = sa; s < sb && !aborted; s += kG) {
                const uint32_t lsw = level_sample_word(prm.l, s);
                const uint32_t s_lo = static_cast<uint32_t>(s);
                const int ngrp = (PK && sb - s >= 2) ? 2 : 1;
                const int nK = prm.c * ngrp;
                const int nsubg = PK ? (nK + kSub - 1) / kSub : nsub;
                for (int j = 0; j < nsubg; ++j, ++g) {
                    const int b = static_cast<int>(g & 1);
                    const int kk = j % kSlices;
                    bool ok = tc::mbar_wait_bounded(bar_full(b), (g >> 1) & 1, tc::globaltimer() + ex.timeout_ns);
                    if (ok && ((slice_seen >> kk) & 1u))
                        ok = tc::mbar_wait_bounded(bar_slice(kk), ((slice_par >> kk) & 1u) ^ 1u,
                                                   tc::globaltimer() + ex.timeout_ns);
                    if (!ok) {
                        *abort_s = 1;
                        atomicExch(ex.err_flag, MLMC_ERR_TIMEOUT);
                    }
                    const int* idx = idx_s + b * kSub;
                    const unsigned char* st = staging + b * C::kStageBytes;   // A parts of the slots
                    const unsigned char* stB = st + kSub * C::kRows * 8;          // then their B parts
                    ok = __all_sync(0xffffffffu, ok);   // whole warps generate or skip (E4M3 uses shuffles)
                    if (ok) {
                        constexpr int kGroups = kSub / kNS;   // items (kNS slots) per row group and sub-block
                        for (int it = tid; it < kItemsA + kItemsB; it += kGenThreads) {
                            if (PK) {
                                // packed samples: A rows 0-63 belong to sample s, rows 64-127 to s + 1 (zero
                                // on the other sample's K positions); B's K positions to whichever owns them.
                                // BF16 takes the A items of half 0, then the B items, then the A items of
                                // half 1, so that a thread's items (it, it + 256) hold one of the active
                                // half's A items or one B item, not both
                                // (4-slot tiles: there the items outnumber the threads)
                                int itA = -1, itB = -1;
                                if constexpr (Q == 0 && kNS == 4) {
                                    constexpr int kAH = kItemsA / 2;
                                    if (it < kAH)
                                        itA = it;
                                    else if (it < kAH + kItemsB)
                                        itB = it - kAH;
                                    else
                                        itA = it - kItemsB;
                                } else {
                                    if (it < kItemsA)
                                        itA = it;
                                    else
                                        itB = it - kItemsA;
                                }
                                if (itA >= 0) {
                                    // BF16: items ordered (half, slot group, row group), so a warp's items
                                    // belong to one half and skip the other sample's positions together
                                    const int rest = itA >> 4;
                                    const int g4 = Q == 0 ? (rest / kGroups) * 16 + (itA & 15) : itA / kGroups;
                                    const int sg = Q == 0 ? rest % kGroups : itA % kGroups;
                                    const int h = g4 >> 4;
                                    const int i = 4 * (g4 & 15);
                                    const uint64_t sh = s + static_cast<uint64_t>(h);
                                    const bool vr = i < prm.m && h < ngrp;
                                    const int* ih = idxh_s + b * 2 * kSub + h * kSub;
                                    const unsigned char* src = st + (sg * kNS) * (C::kRows * 8) + (g4 & 15) * 32;
                                    if constexpr (Q == 0)
                                        gen_block<128, kNS, false, kSkip>(ih, sg * kNS, vr, static_cast<uint32_t>(i >> 2),
                                                            static_cast<uint32_t>(sh), level_sample_word(prm.l, sh),
                                                            prm.rkA, src, C::kRows * 8, false, a_tile, 4 * g4,
                                                            (kSub / 8) * kk + (sg * kNS) / 8, ((sg * kNS) % 8) * 2);
                                    else
                                        gen_block_e4m3<128, kNS>(ih, sg * kNS, vr, static_cast<uint32_t>(i >> 2),
                                                                 static_cast<uint32_t>(sh), level_sample_word(prm.l, sh),
                                                                 prm.rkA, src, C::kRows * 8, false, a_tile, 4 * g4,
                                                                 (kSub / 8) * kk + (sg * kNS) / 8,
                                                                 j * kSub + sg * kNS - h * prm.c, false, ((sg * kNS) % 8) * 2);
                                } else {
                                    const int it2 = itB;
                                    const int g4 = Q == 0 ? it2 % (C::kBGen / 4) : it2 / kGroups;
                                    const int sg = Q == 0 ? it2 / (C::kBGen / 4) : it2 % kGroups;
                                    const int jc = geo.bcol0 + 4 * g4;
                                    const int kp0 = j * kSub + sg * kNS;   // first K position of the item's slots
                                    const int h = kp0 < nK ? kp0 / prm.c : 0;
                                    const uint64_t sh = s + static_cast<uint64_t>(h);
                                    const unsigned char* src = stB + (sg * kNS) * (C::kBGen * 8) + g4 * 32;
                                    if constexpr (Q == 0)
                                        gen_block<128, kNS, XI, kSkip>(idx, sg * kNS, jc < prm.p, static_cast<uint32_t>(jc >> 2),
                                                            static_cast<uint32_t>(sh), level_sample_word(prm.l, sh),
                                                            prm.rkB, src, C::kBGen * 8, coarse_sign, b_tile, brow0 + 4 * g4,
                                                            (kSub / 8) * kk + (sg * kNS) / 8, ((sg * kNS) % 8) * 2,
                                                            gw_s + b * kSub);
                                    else
                                        gen_block_e4m3<128, kNS>(idx, sg * kNS, jc < prm.p, static_cast<uint32_t>(jc >> 2),
                                                                 static_cast<uint32_t>(sh), level_sample_word(prm.l, sh),
                                                                 prm.rkB, src, C::kBGen * 8, coarse_sign, b_tile,
                                                                 brow0 + 4 * g4, (kSub / 8) * kk + (sg * kNS) / 8,
                                                                 kp0 - h * prm.c, prm.c == 16, ((sg * kNS) % 8) * 2);
                                }
                            } else if constexpr (Q == 0) {
                                // consecutive threads take consecutive row groups.  Single-CTA 4-slot tiles
                                // (more items than threads) take the A items of rows 0-63, then the B
                                // items, then the A items of rows 64-127, so that with at most 64 rows
                                // (64-127 are padding, drawn for nothing) no thread holds two drawn items
                                constexpr bool kSplitA = P == 0 && MH == 1 && kNS == 4;
                                constexpr int kAH = kItemsA / 2;
                                const bool isA = kSplitA ? (it < kAH || it >= kAH + kItemsB) : it < kItemsA;
                                const int itA = kSplitA ? (it < kAH ? it : it - kItemsB) : it;
                                const int itB = kSplitA ? it - kAH : it - kItemsA;
                                if (isA) {
                                    // 4 rows of A x kNS slots
                                    const int g4 = kSplitA ? (itA / kAH) * 16 + itA % 16 : itA % (C::kRows / 4);
                                    const int sg = kSplitA ? (itA % kAH) / 16 : itA / (C::kRows / 4);
                                    const int i = tm0 + 4 * g4;
                                    if constexpr (P)
                                        gen_block<64, kNS>(idx, sg * kNS, i < prm.m, static_cast<uint32_t>(i >> 2), s_lo,
                                                           lsw, prm.rkA, st + (sg * kNS) * (C::kRows * 8) + g4 * 32,
                                                           C::kRows * 8, false, a_tile + kk * C::kASliceBytes, 4 * g4,
                                                           (sg * kNS) / 8, ((sg * kNS) % 8) * 2);
                                    else
                                        gen_block<128, kNS, false, kSkip>(idx, sg * kNS, i < prm.m, static_cast<uint32_t>(i >> 2), s_lo,
                                                            lsw, prm.rkA, st + (sg * kNS) * (C::kRows * 8) + g4 * 32,
                                                            C::kRows * 8, false, a_tile, 4 * g4,
                                                            (kSub / 8) * kk + (sg * kNS) / 8, ((sg * kNS) % 8) * 2);
                                } else {
                                    // 4 columns of B (rows of the transposed tile) x kNS slots, sign folded in;
                                    // a pair also writes them into the peer's B tile
                                    const int it2 = itB;
                                    const int g4 = it2 % (C::kBGen / 4);
                                    const int sg = it2 / (C::kBGen / 4);
                                    const int jc = geo.bcol0 + 4 * g4;
                                    const unsigned char* srcB = stB + (sg * kNS) * (C::kBGen * 8) + g4 * 32;
                                    const float* gw = gw_s + b * kSub;
                                    // xi**: the slot weights are folded in too
                                    if constexpr (P) {
                                        if constexpr (XI)
                                            gen_block<64, kNS, true>(idx, sg * kNS, jc < prm.p, static_cast<uint32_t>(jc >> 2),
                                                                     s_lo, lsw, prm.rkB, srcB, C::kBGen * 8, coarse_sign,
                                                                     b_tile + kk * C::kBSliceBytes, brow0 + 4 * g4,
                                                                     (sg * kNS) / 8, ((sg * kNS) % 8) * 2, gw);
                                        else
                                            gen_block<64, kNS>(idx, sg * kNS, jc < prm.p, static_cast<uint32_t>(jc >> 2), s_lo,
                                                               lsw, prm.rkB, srcB, C::kBGen * 8, coarse_sign,
                                                               b_tile + kk * C::kBSliceBytes, brow0 + 4 * g4,
                                                               (sg * kNS) / 8, ((sg * kNS) % 8) * 2);
                                    } else {
                                        if constexpr (XI)
                                            gen_block<128, kNS, true, kSkip>(idx, sg * kNS, jc < prm.p, static_cast<uint32_t>(jc >> 2),
                                                                      s_lo, lsw, prm.rkB, srcB, C::kBGen * 8, coarse_sign,
                                                                      b_tile, brow0 + 4 * g4,
                                                                      (kSub / 8) * kk + (sg * kNS) / 8,
                                                                      ((sg * kNS) % 8) * 2, gw);
                                        else
                                            gen_block<128, kNS, false, kSkip>(idx, sg * kNS, jc < prm.p,
                                                                static_cast<uint32_t>(jc >> 2), s_lo,
                                                                lsw, prm.rkB, srcB, C::kBGen * 8, coarse_sign, b_tile,
                                                                brow0 + 4 * g4, (kSub / 8) * kk + (sg * kNS) / 8,
                                                                ((sg * kNS) % 8) * 2);
                                    }
                                }
                            } else {
                                // E4M3: the kGroups threads of one row group are adjacent lanes, so the
                                // block maximum is a shuffle; a warp is all-A or all-B (kItemsA % 32 == 0)
                                // (pairs: slice tiles in the 64-byte swizzle, as for bfloat16)
                                if (it < kItemsA) {
                                    const int g4 = it / kGroups, sg = it % kGroups;
                                    const int i = tm0 + 4 * g4;
                                    if constexpr (P)
                                        gen_block_e4m3<64, kNS>(idx, sg * kNS, i < prm.m, static_cast<uint32_t>(i >> 2),
                                                                s_lo, lsw, prm.rkA,
                                                                st + (sg * kNS) * (C::kRows * 8) + g4 * 32, C::kRows * 8,
                                                                false, a_tile + kk * C::kASliceBytes, 4 * g4,
                                                                (sg * kNS) / 8, j * kSub + sg * kNS, false,
                                                                ((sg * kNS) % 8) * 2);
                                    else
                                        gen_block_e4m3<128, kNS>(idx, sg * kNS, i < prm.m, static_cast<uint32_t>(i >> 2),
                                                                 s_lo, lsw, prm.rkA,
                                                                 st + (sg * kNS) * (C::kRows * 8) + g4 * 32, C::kRows * 8,
                                                                 false, a_tile, 4 * g4, (kSub / 8) * kk + (sg * kNS) / 8,
                                                                 j * kSub + sg * kNS, false, ((sg * kNS) % 8) * 2);
                                } else {
                                    const int it2 = it - kItemsA;
                                    const int g4 = it2 / kGroups, sg = it2 % kGroups;
                                    const int jc = geo.bcol0 + 4 * g4;
                                    if constexpr (P)
                                        gen_block_e4m3<64, kNS>(idx, sg * kNS, jc < prm.p, static_cast<uint32_t>(jc >> 2),
                                                                s_lo, lsw, prm.rkB,
                                                                stB + (sg * kNS) * (C::kBGen * 8) + g4 * 32, C::kBGen * 8,
                                                                coarse_sign, b_tile + kk * C::kBSliceBytes, brow0 + 4 * g4,
                                                                (sg * kNS) / 8, j * kSub + sg * kNS, false,
                                                                ((sg * kNS) % 8) * 2);
                                    else
                                        gen_block_e4m3<128, kNS>(idx, sg * kNS, jc < prm.p, static_cast<uint32_t>(jc >> 2),
                                                                 s_lo, lsw, prm.rkB,
                                                                 stB + (sg * kNS) * (C::kBGen * 8) + g4 * 32, C::kBGen * 8,
                                                                 coarse_sign, b_tile, brow0 + 4 * g4,
                                                                 (kSub / 8) * kk + (sg * kNS) / 8, j * kSub + sg * kNS,
                                                                 false, ((sg * kNS) % 8) * 2);
                                }
                            }
                        }
                    }
                    // staging buffer b fully read by this warp
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(bar_empty(b));
                    tc::fence_proxy_async_smem();
                    tc::named_barrier(kGenBarrier, kGenThreads);
                    if (*abort_s) {
                        aborted = true;
                        break;
                    }
                    // MMAs of sub-block jj (slice kj) into D and, for tiles that keep it, the chunk sum S
                    auto issue_mma = [&](int jj, int kj) {
                        tc::tc_fence_after_sync();
#pragma unroll
                        for (int ks = 0; ks < C::kKSteps; ++ks) {
                            const int koff = 32 * (kj * C::kKSteps + ks);   // bytes into the swizzle atom
                            if constexpr (F != 0) {
                                // even slots (K step 0) into E, odd (coarse) slots (K step 1) into O
                                tc::mma_bf16(tmem + ks * C::kTileCols, tc::sw128_kmajor_desc(tc::smem_addr(a_tile) + koff),
                                             tc::sw128_kmajor_desc(tc::smem_addr(b_tile) + koff), idesc,
                                             jj > 0 ? 1u : 0u);
                                continue;
                            }
                            const bool acc = jj > 0 || ks > 0;
#pragma unroll
                            for (int h = 0; h < MH; ++h) {
                                // pairs: slice kj has its own 64-byte-swizzled A and B tiles
                                const uint64_t adesc =
                                    P ? tc::sw64_kmajor_desc(tc::smem_addr(a_tile) + kj * C::kASliceBytes + 32 * ks)
                                      : tc::sw128_kmajor_desc(tc::smem_addr(a_tile) + h * 128 * 128 + koff);
                                const uint64_t bdesc =
                                    P ? tc::sw64_kmajor_desc(tc::smem_addr(b_tile) + kj * C::kBSliceBytes + 32 * ks)
                                      : tc::sw128_kmajor_desc(tc::smem_addr(b_tile) + koff);
                                tc::mma_bf16(tmem + h * BN, adesc, bdesc, idesc, acc ? 1u : 0u);
                                if constexpr (C::kAccS)   // running sum of the chunk's samples
                                    tc::mma_bf16(tmem + C::kTileCols + h * BN, adesc, bdesc, idesc,
                                                 (acc || s != sa) ? 1u : 0u);
                            }
                        }
                        if constexpr (P)
                            tc::mma_commit_multicast(bar_slice(kj), 0x3);   // both CTAs wait for this slice
                        else
                            tc::mma_commit(bar_slice(kj));
                        if (jj == nsubg - 1) tc::mma_commit(bar_done);
                    };
                    if constexpr (P) {
                        // Pairs: send our half of this slice of B to the peer (async proxy, counted on its
                        // barrier); the MMAs of a sub-block are issued one sub-block later, once the
                        // peer's half has had a sub-block's time to land, and at the sample's end.
                        if (tid == 0) {
                            const uint32_t off = static_cast<uint32_t>(kk * C::kBSliceBytes + brow0 * 64);
                            const uint32_t bytes = static_cast<uint32_t>(C::kBGen * 64);
                            tc::bulk_copy_s2s_cluster(peer_b_tile + off, tc::smem_addr(b_tile) + off, bytes,
                                                      tc::map_to_cta(bar_peer(kk), peer));
                            tc::mbar_arrive_expect_tx(bar_peer(kk), bytes);
                            peer_armed = kk;
                            auto wait_peer = [&](int kj) {
                                if (!tc::mbar_wait_cluster_bounded(bar_peer(kj), (peer_par >> kj) & 1u,
                                                                   tc::globaltimer() + ex.timeout_ns)) {
                                    *abort_s = 1;
                                    atomicExch(ex.err_flag, MLMC_ERR_TIMEOUT);
                                }
                                peer_par ^= 1u << kj;
                                if (kj == peer_armed) peer_armed = -1;
                            };
                            if (j > 0) {
                                const int kprev = (j - 1) % kSlices;
                                wait_peer(kprev);
                                issue_mma(j - 1, kprev);
                            }
                            if (j == nsubg - 1) {
                                wait_peer(kk);
                                issue_mma(j, kk);
                            }
                        }
                    } else if (tid == 0) {
                        issue_mma(j, kk);
                    }
                    slice_par ^= 1u << kk;
                    slice_seen |= 1u << kk;
                }
                if (aborted) break;
                // sample epilogue: wait for the accumulator, then drain it
                if (!tc::mbar_wait_bounded(bar_done, done_count & 1, tc::globaltimer() + ex.timeout_ns)) {
                    *abort_s = 1;
                    atomicExch(ex.err_flag, MLMC_ERR_TIMEOUT);
                }
                ++done_count;
                tc::named_barrier(kGenBarrier, kGenThreads);
                if (*abort_s) {
                    aborted = true;
                    break;
                }
                tc::tc_fence_after_sync();
                // Welford's update of the chunk's M2 with k = s - sa samples folded before: the
                // deviation of D from the mean of those k is (k D - sum_k) / k, and M2 grows by
                // ||k D - sum_k||^2 / (k (k + 1)) (nothing for the chunk's first sample)
                const int kbefore = static_cast<int>((s - sa) / kG);
                // FP32 throughout (FP64 runs at 1/64 of the FP32 rate here); exact for k (k + 1) <= 2^24
                const float wk = kbefore > 0 ? 1.0f / static_cast<float>(kbefore * (kbefore + 1)) : 0.0f;
                if constexpr (F != 0) {
                    // fine = n/c_l (E + O), coarse = n/c_{l-1} O (the odd slots t = 1 mod 2 are the
                    // coarse ones), D = f(fine) - f(coarse) (level 0: f(fine)); the chunk's running sum
                    // S of D is read, grown by Welford's update and written back in tensor memory
                    const float sc = 2.0f * scale;
                    const float kf = static_cast<float>(kbefore);
                    const bool coarse = prm.l > 0;
                    float qsamp = 0.0f;
                    for (int cb = 0; cb < dr.ncols; cb += 16) {   // ncols is a multiple of 32
                        float ve[16], vo[16], vs[16];
                        tc::tmem_ld_32x32b_x16_nowait(dr.taddr(tmem, cb), ve);
                        tc::tmem_ld_32x32b_x16_nowait(dr.taddr(tmem + C::kTileCols, cb), vo);
                        if (kbefore > 0) tc::tmem_ld_32x32b_x16_nowait(dr.taddr(tmem + C::kSOff, cb), vs);
                        tc::tmem_ld_wait();
                        float qs = 0.0f;
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            float d = tc_targeted<F>(scale * (ve[e] + vo[e]));
                            if (coarse) d -= tc_targeted<F>(sc * vo[e]);
                            if (kbefore > 0) {
                                const float dk = fmaf(kf, d, -vs[e]);
                                qs = fmaf(dk, dk, qs);
                                vs[e] += d;
                            } else {
                                vs[e] = d;
                            }
                        }
                        tc::tmem_st_32x32b_x16(dr.taddr(tmem + C::kSOff, cb), vs);
                        qsamp += qs;
                    }
                    tc::tmem_st_wait();
                    qw = fmaf(qsamp, wk, qw);
                } else if constexpr (C::kAccS) {
                    // the running sum S (after this sample) sits beside D in tensor memory:
                    // k D - sum_k = (k + 1) D - S, one fused rounding per element (PK: per half,
                    // and a group without a second sample has nothing in rows 64-127).  Levels
                    // whose mean is zero by construction (prm.welford == 0) keep the raw sum of
                    // ||D||^2 instead; the chunk's M2 follows from it and ||S||^2 at the chunk's end.
                    if (!prm.welford) {
                        if (pk_half < ngrp) {
                            float qsamp = 0.0f;
                            for (int cb = 0; cb < dr.ncols; cb += kCW) {
                                float v[kCW];
                                const uint32_t ta = dr.taddr(tmem, cb);
                                tc::tmem_ld_32x32b_x32_nowait(ta, v);
                                if constexpr (kCW == 64)
                                    if (cb + 32 < dr.ncols) tc::tmem_ld_32x32b_x32_nowait(ta + 32, v + kCW / 2);
                                tc::tmem_ld_wait();
                                const int nv = min(kCW, dr.ncols - cb);
                                float qs = 0.0f;
#pragma unroll
                                for (int e = 0; e < kCW; ++e)
                                    if (e < nv) qs = fmaf(v[e], v[e], qs);
                                qsamp += qs;
                            }
                            qw += qsamp;
                        }
                    } else if (kbefore > 0 && pk_half < ngrp) {
                        const float kp1 = static_cast<float>(kbefore + 1);
                        float qsamp = 0.0f;
                        // columns per wait: 32 where the registers allow it (pairs, narrow tiles), else 16
                        constexpr int kW = (W == 8 && (P || (BN <= 64 && MH == 1))) ? 32 : 16;
                        for (int cb = 0; cb < dr.ncols; cb += kW) {   // ncols is a multiple of 32
                            float vd[kW], vs[kW];
#pragma unroll
                            for (int h16 = 0; h16 < kW; h16 += 16) {
                                tc::tmem_ld_32x32b_x16_nowait(dr.taddr(tmem, cb + h16), vd + h16);
                                tc::tmem_ld_32x32b_x16_nowait(dr.taddr(tmem + C::kTileCols, cb + h16), vs + h16);
                            }
                            tc::tmem_ld_wait();
                            float qs = 0.0f;
#pragma unroll
                            for (int e = 0; e < kW; ++e) {
                                const float dk = fmaf(kp1, vd[e], -vs[e]);
                                qs = fmaf(dk, dk, qs);
                            }
                            qsamp += qs;
                        }
                        qw = fmaf(qsamp, wk, qw);
                    }
                } else {
                    // two 32-column loads in flight per wait
                    float qsamp = 0.0f;
                    for (int cb = 0; cb < dr.ncols; cb += 64) {
                        float v[64];
                        const uint32_t ta = dr.taddr(tmem, cb);
                        tc::tmem_ld_32x32b_x32_nowait(ta, v);
                        if (cb + 32 < dr.ncols) tc::tmem_ld_32x32b_x32_nowait(ta + 32, v + 32);
                        tc::tmem_ld_wait();
                        const int nv = min(64, dr.ncols - cb);
#pragma unroll
                        for (int e = 0; e < 64; ++e) v[e] *= scale;
                        qsamp += store_cols(v, cb, nv, kbefore);
                    }
                    qw = fmaf(qsamp, wk, qw);
                }
                tc::tc_fence_before_sync();
                tc::named_barrier(kGenBarrier, kGenThreads);  // the accumulator may now be overwritten
            }
            if (aborted) return false;
            if (PK) {
                // the two halves' running sums and M2 combine into the chunk's: the second half's sum
                // is stored first, then the first half adds its own and Chan's cross term
                // n_t n_b / (n_t + n_b) ||S_t / n_t - S_b / n_b||^2
                tc::tc_fence_after_sync();
                const int nc = static_cast<int>(sb - sa), nt = (nc + 1) / 2, nb = nc / 2;
                if (pk_half == 1 && nb > 0) {
                    float ssq = 0.0f;   // raw form: ||S_b||^2 (unscaled)
                    for (int cb = 0; cb < dr.ncols; cb += 64) {
                        float v[64];
                        const uint32_t ta = dr.taddr(tmem + C::kTileCols, cb);
                        tc::tmem_ld_32x32b_x32_nowait(ta, v);
                        if (cb + 32 < dr.ncols) tc::tmem_ld_32x32b_x32_nowait(ta + 32, v + 32);
                        tc::tmem_ld_wait();
                        float qs = 0.0f;   // grouped as in the drain, so one sample gives exactly zero
#pragma unroll
                        for (int e = 0; e < 64; ++e) {
                            if (e < min(64, dr.ncols - cb)) qs = fmaf(v[e], v[e], qs);
                            v[e] *= scale;
                        }
                        ssq += qs;
                        store_cols(v, cb, min(64, dr.ncols - cb), 0);
                    }
                    if (!prm.welford) q -= static_cast<double>(ssq) * scale_sq / static_cast<double>(nb);
                }
                tc::named_barrier(kGenBarrier, kGenThreads);   // orders the stores before the reads below
                if (pk_half == 0) {
                    const float inv_nt = 1.0f / static_cast<float>(nt);
                    const float inv_nb = nb > 0 ? 1.0f / static_cast<float>(nb) : 0.0f;
                    double cross = 0.0;
                    float ssq = 0.0f;   // raw form: ||S_t||^2 (unscaled)
                    for (int cb = 0; cb < dr.ncols; cb += 64) {
                        float v[64];
                        const uint32_t ta = dr.taddr(tmem + C::kTileCols, cb);
                        tc::tmem_ld_32x32b_x32_nowait(ta, v);
                        if (cb + 32 < dr.ncols) tc::tmem_ld_32x32b_x32_nowait(ta + 32, v + 32);
                        tc::tmem_ld_wait();
                        const int nv = min(64, dr.ncols - cb);
                        {
                            float qs = 0.0f;
#pragma unroll
                            for (int e = 0; e < 64; ++e)
                                if (e < nv) qs = fmaf(v[e], v[e], qs);
                            ssq += qs;
                        }
                        float cq = 0.0f;
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh) {
                            const int gj0 = tp0 + dr.col_d + cb + 32 * hh;
                            if (32 * hh >= nv || dr.gi >= prm.m || gj0 >= prm.p) continue;
                            float* dst = part + static_cast<int64_t>(dr.gi) * prm.p + gj0;
                            const int valid = min(32, prm.p - gj0);
#pragma unroll
                            for (int e = 0; e < 32; ++e) {
                                if (e < valid) {
                                    const float x = v[32 * hh + e] * scale;
                                    const float pb = nb > 0 ? dst[e] : 0.0f;
                                    if (nb > 0) {
                                        const float d = x * inv_nt - pb * inv_nb;
                                        cq = fmaf(d, d, cq);
                                    }
                                    dst[e] = x + pb;
                                }
                            }
                        }
                        cross += static_cast<double>(cq);
                    }
                    if (nb > 0)
                        q += cross * (static_cast<double>(nt) * static_cast<double>(nb) / static_cast<double>(nt + nb));
                    if (!prm.welford) q -= static_cast<double>(ssq) * scale_sq / static_cast<double>(nt);
                }
                tc::tc_fence_before_sync();
            } else if constexpr (C::kAccS) {
                // the chunk's sum of D: one store per element of the tile (raw form: also ||S||^2)
                tc::tc_fence_after_sync();
                float ssq = 0.0f;
                const float sscale = F ? 1.0f : scale;   // F != 0: S holds scaled values already
                for (int cb = 0; cb < dr.ncols; cb += kCW) {
                    float v[64];   // store_cols reads up to 64; the 16-warp form fills the first 32
                    const uint32_t ta = dr.taddr(tmem + C::kSOff, cb);
                    tc::tmem_ld_32x32b_x32_nowait(ta, v);
                    if (kCW == 64 && cb + 32 < dr.ncols) tc::tmem_ld_32x32b_x32_nowait(ta + 32, v + 32);
                    tc::tmem_ld_wait();
                    const int nv = min(kCW, dr.ncols - cb);
                    float qs = 0.0f;
#pragma unroll
                    for (int e = 0; e < kCW; ++e) {
                        if (e < nv) qs = fmaf(v[e], v[e], qs);
                        v[e] *= sscale;
                    }
                    ssq += qs;
                    store_cols(v, cb, nv, 0);
                }
                if (!prm.welford) q -= static_cast<double>(ssq) * scale_sq / static_cast<double>(sb - sa);
                tc::tc_fence_before_sync();
            }
            if (aborted) return false;
            // the Welford terms in FP64 (tiles that keep S drained unscaled values)
            q += static_cast<double>(qw) * (C::kAccS && F == 0 ? scale_sq : 1.0);
            // work-item epilogue: the chunk's M2 over this tile, fixed-order reduction
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) q += __shfl_xor_sync(0xffffffffu, q, off);
            if (lane == 0) red_s[warp] = q;
            tc::named_barrier(kGenBarrier, kGenThreads);
            if (tid == 0) {
                double t = 0.0;
                for (int w = 0; w < kGenWarps; ++w) t += red_s[w];
                if (geo.qtile >= 0) prm.partial_q[static_cast<int64_t>(cy) * tiles_n + geo.qtile] = t;
            }
            tc::named_barrier(kGenBarrier, kGenThreads);
            return true;
        }, true);
        // after an abort make sure no MMA is still writing TMEM before it is freed: a barrier used
        // for nothing else completes its first phase once every MMA issued so far has completed
        if (aborted && tid == 0) {
            tc::mma_commit(bar_quiesce);
            tc::mbar_wait_bounded(bar_quiesce, 0, tc::globaltimer() + kDrainNs);
            // pairs: the peer's half of the last slice may still be arriving in our B tile
            if (P && peer_armed >= 0)
                tc::mbar_wait_cluster_bounded(bar_peer(peer_armed), (peer_par >> peer_armed) & 1u,
                                              tc::globaltimer() + kDrainNs);
        }
    }
    tc::tc_fence_before_sync();
    __syncthreads();
    if constexpr (P) {
        tc::cluster_sync();   // no remote copy or arrival can reach a CTA that left
        if (*abort_s) {
            // after an abort a copy the peer sent for a sub-block we never reached may still be in
            // flight (it cannot be waited for): give it time to land before the CTA exits
            const uint64_t until = tc::globaltimer() + 50000;
            while (tc::globaltimer() < until) __nanosleep(1000);
        }
    }
    if (warp == 0) tc::tmem_dealloc(tmem, C::kTmemCols);
}

template <int MH, int BN, int Q, bool kBatch>
cudaError_t prepare(int* per_sm)
{
    using C = TcCfg<MH, BN, Q>;
    // the attribute is per function and device; setting it again is cheap
    cudaError_t e = cudaFuncSetAttribute(level_tc_bf16_kernel<MH, BN, Q, kBatch>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, level_tc_bf16_kernel<MH, BN, Q, kBatch>, C::kThr,
                                                      C::kSmemBytes);
    if (e != cudaSuccess) return e;
    *per_sm = max(1, min(occ, 512 / C::kTmemCols));
    return cudaSuccess;
}

// One single-problem launch of the single-CTA kernel (F: targeted function, XI: xi** law).
template <int MH, int BN, int Q, int F, bool XI>
cudaError_t launch_single(const LevelParams& prm, const TcLaunch& tl, cudaStream_t st)
{
    using C = TcCfg<MH, BN, Q, 0, 8, F>;
    if constexpr (!C::kFits) {
        return cudaErrorInvalidValue;
    } else {
        auto kern = level_tc_bf16_kernel<MH, BN, Q, false, 0, 8, F, XI>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
        if (e != cudaSuccess) return e;
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, C::kThr, C::kSmemBytes);
        if (e != cudaSuccess) return e;
        const int per_sm = max(1, min(occ, 512 / C::kTmemCols));
        const int items = prm.nchunks * prm.tiles_m * prm.tiles_p;
        const int grid = max(1, min(items, per_sm * tl.num_sms));
        TcExtra ex{tl.err_flag, tl.timeout_ns, items, tl.scale};
        kern<<<grid, C::kThr, C::kSmemBytes, st>>>(prm, ex, TcBatch{});
        return cudaGetLastError();
    }
}

template <int MH, int BN, int Q>
struct SingleF {
    static cudaError_t run(const LevelParams& prm, const TcLaunch& tl, cudaStream_t st)
    {
        return launch_single<MH, BN, Q, 0, false>(prm, tl, st);
    }
};

template <int MH, int BN, int Q>
struct BatchF {
    static cudaError_t run(const TcBatch& bt, int grid, const TcLaunch& tl, cudaStream_t st)
    {
        using C = TcCfg<MH, BN, Q>;
        if constexpr (!C::kFits) {
            return cudaErrorInvalidValue;
        } else {
            // the function attributes were set by tc_batch_grid (no attribute calls while a graph is captured)
            TcExtra ex{tl.err_flag, tl.timeout_ns, 0, 0.0f};
            LevelParams none{};
            level_tc_bf16_kernel<MH, BN, Q, true><<<grid, C::kThr, C::kSmemBytes, st>>>(none, ex, bt);
            return cudaGetLastError();
        }
    }
};

template <int MH, int BN, int Q>
struct GridF {
    static int run(int num_sms)
    {
        if constexpr (!TcCfg<MH, BN, Q>::kFits) {
            return 0;
        } else {
            int per_sm = 1;
            if (prepare<MH, BN, Q, true>(&per_sm) != cudaSuccess) return 0;
            return per_sm * num_sms;
        }
    }
};

// A cluster pair (two CTAs, 128 rows each) on one 256 x 256 output tile; W generator warps.
template <int Q, int W, bool XI = false>
cudaError_t launch_pair(const LevelParams& prm, const TcLaunch& tl, cudaStream_t st)
{
    using C = TcCfg<1, 256, Q, 1, W>;
    auto kern = level_tc_bf16_kernel<1, 256, Q, false, 1, W, 0, XI>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(C::kThr);
    cfg.dynamicSmemBytes = C::kSmemBytes;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(2 * static_cast<unsigned>(tl.num_sms / 2));
    int max_clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&max_clusters, kern, &cfg);
    if (e != cudaSuccess) return e;
    const int pair_items = prm.nchunks * ((prm.tiles_m + 1) / 2) * prm.tiles_p;
    const int clusters = max(1, min(pair_items, max(1, max_clusters)));
    cfg.gridDim = dim3(2 * static_cast<unsigned>(clusters));
    TcExtra ex{tl.err_flag, tl.timeout_ns, pair_items, tl.scale};
    e = cudaLaunchKernelEx(&cfg, kern, prm, ex, TcBatch{});
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// Batched launches of the CTA pair (tile 3256): `clusters` clusters of two CTAs, each cluster
// walking its own item list.  The function attributes were set by pair_batch_grid (no attribute
// calls while a graph is captured).
template <int Q>
cudaError_t launch_pair_batch(const TcBatch& bt, int clusters, const TcLaunch& tl, cudaStream_t st)
{
    using C = TcCfg<1, 256, Q, 1, 8>;
    auto kern = level_tc_bf16_kernel<1, 256, Q, true, 1, 8>;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(C::kThr);
    cfg.dynamicSmemBytes = C::kSmemBytes;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(2 * static_cast<unsigned>(max(1, clusters)));
    TcExtra ex{tl.err_flag, tl.timeout_ns, 0, 0.0f};
    LevelParams none{};
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, none, ex, bt);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// Clusters of the batched CTA pair that fit on the GPU at once (the units its item lists are cut
// into); sets the kernel's shared-memory attribute.
template <int Q>
int pair_batch_grid(int num_sms)
{
    using C = TcCfg<1, 256, Q, 1, 8>;
    auto kern = level_tc_bf16_kernel<1, 256, Q, true, 1, 8>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes) != cudaSuccess)
        return 0;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(C::kThr);
    cfg.dynamicSmemBytes = C::kSmemBytes;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(2 * static_cast<unsigned>(num_sms / 2));
    int max_clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&max_clusters, kern, &cfg) != cudaSuccess) return 0;
    return max(0, max_clusters);
}

template <int MH, int BN, int Q>
struct FitsF {
    static bool run() { return TcCfg<MH, BN, Q>::kFits; }
};

template <template <int, int, int> class F, int Q, typename... Args>
auto dispatch_bn(int mh, int bn, Args&&... args)
{
    if (mh == 1) {
        switch (bn) {
            case 32: return F<1, 32, Q>::run(args...);
            case 64: return F<1, 64, Q>::run(args...);
            case 128: return F<1, 128, Q>::run(args...);
            default: return F<1, 256, Q>::run(args...);
        }
    }
    switch (bn) {
        case 32: return F<2, 32, Q>::run(args...);
        case 64: return F<2, 64, Q>::run(args...);
        case 128: return F<2, 128, Q>::run(args...);
        default: return F<2, 256, Q>::run(args...);
    }
}

template <template <int, int, int> class F, typename... Args>
auto dispatch_tile(const TcTile& t, int q, Args&&... args)
{
    return q ? dispatch_bn<F, 1>(t.mh, t.bn, args...) : dispatch_bn<F, 0>(t.mh, t.bn, args...);
}

// Verification of the bounded waits: one warp waits on an mbarrier that nothing arrives on;
// when the wait gives up it records MLMC_ERR_TIMEOUT in the error word, as the level kernels do.
__global__ void bounded_wait_probe_kernel(int* err_flag, uint64_t timeout_ns)
{
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = tc::smem_addr(&bar);
    if (threadIdx.x == 0) {
        tc::mbar_init(b, 1);
        tc::mbar_init_fence();
    }
    __syncthreads();
    const bool ok = tc::mbar_wait_bounded(b, 0, tc::globaltimer() + timeout_ns);
    if (!ok && threadIdx.x == 0) atomicExch(err_flag, MLMC_ERR_TIMEOUT);
}

}  // namespace

cudaError_t launch_bounded_wait_probe(int* err_flag, uint64_t timeout_ns, cudaStream_t st)
{
    bounded_wait_probe_kernel<<<1, 32, 0, st>>>(err_flag, timeout_ns);
    return cudaGetLastError();
}

// E4M3 blocks are 32 consecutive slots of a sample: packed K positions keep them apart when c is a
// multiple of 32 (a sub-block never straddles two samples) or c = 16 (each sample's slots form one
// block, the two halves of a sub-block)
bool tc_pack(const TcTile& t, int q, int64_t m, int64_t c)
{
    if (t.mh != 1 || t.pair || m > 64 || c % 16 != 0) return false;
    return q == 0 || c == 16 || c % 32 == 0;
}

int tc_stage_width_a(const TcTile& t) { return t.pair ? 128 : 128 * t.mh; }
int tc_stage_width_b(const TcTile& t) { return t.pair ? t.bn / 2 : t.bn; }

bool tc_encode_maps(TcMaps* maps, const void* base, int64_t n, int64_t ld, int wa, int wb)
{
    std::memset(maps, 0, sizeof(TcMaps));
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Encode encode = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<Encode>(fn);
        looked_up = true;
    }
    if (!encode || wa < 2 || wb < 2 || wa > 256 || wb > 256 || (ld % 2) != 0) return false;
    // n rows of ld / 2 eight-byte (M, S) pairs; rows ld * 4 bytes apart; boxes of one row
    const cuuint64_t dims[2] = {static_cast<cuuint64_t>(ld / 2), static_cast<cuuint64_t>(n)};
    const cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * 4};
    const cuuint32_t estr[2] = {1, 1};
    if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (strides[0] & 15) != 0) return false;
    const cuuint32_t box_a[2] = {static_cast<cuuint32_t>(wa), 1};
    const cuuint32_t box_b[2] = {static_cast<cuuint32_t>(wb), 1};
    void* g = const_cast<void*>(base);
    if (encode(&maps->a, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, g, dims, strides, box_a, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    if (encode(&maps->b, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, g, dims, strides, box_b, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    maps->wa = wa;
    maps->wb = wb;
    maps->valid = 1;
    return true;
}

bool tc_tile_valid(const TcTile& t, int q)
{
    if (t.pair) return t.mh == 1 && t.bn == 256 && (q == 0 || q == 1);
    if (!((t.mh == 1 || t.mh == 2) && (t.bn == 32 || t.bn == 64 || t.bn == 128 || t.bn == 256))) return false;
    return dispatch_tile<FitsF>(t, q);
}

TcTile tc_tile_for(int64_t m, int64_t p, int q, bool allow_pair)
{
    TcTile t{};
    // cluster pair; E4M3 (the heavier generation of stochastic rounding) with 16 generator warps,
    // measured 10 % faster than 8 on the 256 x 65536 x 256 workload, BF16 with 8 (7 % faster)
    if (allow_pair && m > 128 && p > 128) return TcTile{1, 256, 128, q == 1 ? 2 : 1};
    t.mh = m <= 128 ? 1 : 2;
    t.bn = p <= 32 ? 32 : p <= 64 ? 64 : p <= 128 ? 128 : 256;
    while (!tc_tile_valid(t, q) && t.bn > 32) t.bn /= 2;   // E4M3: narrower column tiles
    t.rows = 128 * t.mh;
    t.pair = 0;
    return t;
}

cudaError_t launch_level_tc(const LevelParams& prm, const TcTile& tile, int q, const TcLaunch& tl, cudaStream_t st)
{
    if (!tc_tile_valid(tile, q)) return cudaErrorInvalidValue;
    if (prm.xi_Q) {
        // xi**: BF16, the CTA pair or single-CTA tiles of 128 rows and at most 128 columns
        if (q != 0 || !tc_tile_valid_xi(tile)) return cudaErrorInvalidValue;
        if (tile.pair) return launch_pair<0, 8, true>(prm, tl, st);
        switch (tile.bn) {
        case 32: return launch_single<1, 32, 0, 0, true>(prm, tl, st);
        case 64: return launch_single<1, 64, 0, 0, true>(prm, tl, st);
        default: return launch_single<1, 128, 0, 0, true>(prm, tl, st);
        }
    }
    if (tile.pair == 2) return q ? launch_pair<1, 16>(prm, tl, st) : launch_pair<0, 16>(prm, tl, st);
    if (tile.pair) return q ? launch_pair<1, 8>(prm, tl, st) : launch_pair<0, 8>(prm, tl, st);
    return dispatch_tile<SingleF>(tile, q, prm, tl, st);
}

TcTile tc_tile_for_f(int64_t p)
{
    const int bn = p <= 32 ? 32 : p <= 64 ? 64 : 128;
    return TcTile{1, bn, 128, 0};
}

bool tc_tile_valid_f(const TcTile& t) { return t.mh == 1 && !t.pair && (t.bn == 32 || t.bn == 64 || t.bn == 128); }

TcTile tc_tile_for_xi(int64_t m, int64_t p)
{
    if (m > 128 && p > 128) return TcTile{1, 256, 128, 1};
    return tc_tile_for_f(p);
}

bool tc_tile_valid_xi(const TcTile& t) { return (t.pair == 1 && t.mh == 1 && t.bn == 256) || tc_tile_valid_f(t); }

cudaError_t launch_level_tc_f(const LevelParams& prm, const TcTile& tile, int f, const TcLaunch& tl, cudaStream_t st)
{
    if (f != 1 || !tc_tile_valid_f(tile)) return cudaErrorInvalidValue;
    const bool xi = prm.xi_Q != nullptr;
    switch (tile.bn) {
    case 32: return xi ? launch_single<1, 32, 0, 1, true>(prm, tl, st) : launch_single<1, 32, 0, 1, false>(prm, tl, st);
    case 64: return xi ? launch_single<1, 64, 0, 1, true>(prm, tl, st) : launch_single<1, 64, 0, 1, false>(prm, tl, st);
    default:
        return xi ? launch_single<1, 128, 0, 1, true>(prm, tl, st) : launch_single<1, 128, 0, 1, false>(prm, tl, st);
    }
}

int tc_batch_grid(const TcTile& tile, int q, int num_sms)
{
    if (!tc_tile_valid(tile, q) || tile.pair == 2) return 0;
    if (tile.pair) return q ? pair_batch_grid<1>(num_sms) : pair_batch_grid<0>(num_sms);
    return dispatch_tile<GridF>(tile, q, num_sms);
}

cudaError_t launch_level_tc_batch(const TcBatch& bt, const TcTile& tile, int q, int grid, const TcLaunch& tl,
                                  cudaStream_t st)
{
    if (!tc_tile_valid(tile, q) || tile.pair == 2) return cudaErrorInvalidValue;
    if (tile.pair) return q ? launch_pair_batch<1>(bt, grid, tl, st) : launch_pair_batch<0>(bt, grid, tl, st);
    return dispatch_tile<BatchF>(tile, q, bt, grid, tl, st);
}

}  // namespace mlmc
