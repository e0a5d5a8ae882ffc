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
// are processed in sub-blocks of 16 (one MMA K step):
//   * producer warp (warp 8): draws the 16 slot indices of a sub-block from Philox and issues
//     TMA bulk copies (cp.async.bulk) of the sampled (M, S) column and (M', S') row pairs of the
//     tile into a double-buffered staging area, completing on the buffer's mbarrier;
//   * generator warps (0-7): wait for the staged pairs, generate A = M + S Z and
//     sigma (M' + S' Z') with Philox and a special-function-unit Box-Muller, round to bf16 and
//     write them into one 16-slot slice of a 128-byte-swizzled K-major tile (four slices form
//     one swizzle atom); thread 0 then issues tcgen05.mma (M = 128 per half, N = tile width,
//     K = 16) into TMEM and commits to the slice's mbarrier;
//   * after the last sub-block of a sample the generator warps drain the accumulator with
//     tcgen05.ld, add the sample's D to the chunk partial in global memory (store for the first
//     sample of the chunk, then red.global.add: each element has one owner thread, so the
//     order is fixed) and accumulate ||D||_F^2.
// Every mbarrier wait is bounded by a %globaltimer deadline; on timeout the kernel records
// MLMC_ERR_TIMEOUT and leaves after freeing its tensor memory.
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

constexpr int kGenWarps = 8;
constexpr int kGenThreads = kGenWarps * 32;
constexpr int kThreads = kGenThreads + 32;  // + producer warp
constexpr int kGenBarrier = 1;              // named barrier of the generator warps
constexpr uint64_t kDrainNs = 100000000ull;   // bound on waiting for own copies in flight after an abort

// Operand formats: Q = 0 rounds the generated entries to bfloat16; Q = 1 quantises them to FP8
// E4M3 with a power-of-two scale per (row of A or column of B, 32-slot block) and feeds the
// dequantised values (exact in bfloat16) to the same MMA.
// P = 1: a cluster pair of CTAs shares one 256-row x BN tile; each CTA owns 128 rows (MH = 1),
// generates its rows of A and half of the B columns, and copies that half into the peer's B tile
// (one bulk shared-to-shared copy per sub-block).  Pairs keep four slices of 32 K elements in
// 64-byte-swizzled tiles (one per slice), so each CTA's half of a slice is one contiguous run and
// the peer has three sub-blocks of slack before a slice is reused.
template <int MH, int BN, int Q, int P = 0>
struct TcCfg {
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
    static constexpr int kAccCols = kAccS ? 2 * kTileCols : kTileCols;
    static constexpr int kTmemCols = kAccCols <= 32 ? 32 : kAccCols <= 64 ? 64 : kAccCols <= 128 ? 128
                                     : kAccCols <= 256 ? 256 : 512;
    // barriers: full[2], empty[2], slice[kSlices], done, and for pairs peer[kSlices] (the peer's B half landed)
    static constexpr int kNumBars = 2 + 2 + kSlices + 1 + (P ? kSlices : 0) + 1 /*abort drain*/;
    static constexpr int kBookBytes = 2 * kSub * 4 /*idx*/ + kNumBars * 8 + 16 /*tmem, abort*/ + kGenWarps * 8 +
                                      (P ? 0 : 2 * static_cast<int>(sizeof(LevelParams)) +
                                                   static_cast<int>(alignof(LevelParams)))
                                      /*job copies of batched launches (pairs run single-problem launches)*/;
    static constexpr int kSmemBytes = 1024 /*align slack*/ + kTileBytes + 2 * kStageBytes + kBookBytes;
    static_assert(kAccCols <= 512, "tile exceeds tensor memory");
    static_assert(kTmemCols >= kAccCols, "the allocation holds the accumulators");
    static_assert(kKSteps * 16 == kSub, "a sub-block is a whole number of K = 16 MMA steps");
    static_assert(BN % 16 == 0 && BN >= 32 && BN <= 256, "N of the MMA");
    static constexpr bool kFits = kSmemBytes <= 227 * 1024 &&   // E4M3's 32-slot staging rules out wide tiles
                                  (!P || (MH == 1 && BN == 256));
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

// Generate one block of (4 rows of A, or 4 columns of B) x (8 slots) entries from staged (M, S)
// pairs and write them as bf16 into the swizzled tile: tile rows row0 .. row0+3, 16-byte chunk
// `chunk`.  Staged pairs of slot u start at stage + u * stride (8 floats: (M,S) x 4).
// kSw: the tile's swizzle, 128 or 64 bytes per row.
template <int kSw>
__device__ __forceinline__ uint32_t tile_offset(int row, int chunk)
{
    return kSw == 128 ? tc::sw128_offset(row, chunk) : tc::sw64_offset(row, chunk);
}

template <int kSw = 128>
__device__ __forceinline__ void gen_block(const int* idx, int slot0, bool valid_rows, uint32_t rowgrp,
                                          uint32_t s_lo, uint32_t lsw, const PhiloxRoundKeys& rk,
                                          const unsigned char* stage,
                                          int stride, bool odd_negative, unsigned char* tile, int row0, int chunk)
{
    if (!valid_rows) {
        // padding rows (or columns) of the tile: zeros, no random numbers needed
#pragma unroll
        for (int r = 0; r < 4; ++r)
            *reinterpret_cast<uint4*>(tile + tile_offset<kSw>(row0 + r, chunk)) = make_uint4(0, 0, 0, 0);
        return;
    }
    // Branch-free: the eight Philox blocks are independent dependency chains, computed for every
    // slot (a missing slot uses k = 0) and zeroed afterwards, so they can interleave.
    int ks[8];
    uint4 w[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        ks[u] = idx[slot0 + u];
        w[u] = philox4x32_10_rk(make_uint4(rowgrp, static_cast<uint32_t>(max(ks[u], 0)), s_lo, lsw), rk);
    }
    float v[4][8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
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
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const uint4 packed = make_uint4(pack_bf16x2(v[r][0], v[r][1]), pack_bf16x2(v[r][2], v[r][3]),
                                        pack_bf16x2(v[r][4], v[r][5]), pack_bf16x2(v[r][6], v[r][7]));
        *reinterpret_cast<uint4*>(tile + tile_offset<kSw>(row0 + r, chunk)) = packed;
    }
}

// E4M3 form of gen_block for 32-slot sub-blocks: the four adjacent lanes of one row group hold
// the row's 32 slots (8 each).  Each row's block maximum |x| gives the scale 2^e, e the
// smallest integer with max <= 448 * 2^e (1 for an all-zero block); x / 2^e is rounded to E4M3
// (nearest even, saturating at 448) and the dequantised value, exact in bfloat16, is stored.
// Every lane of the warp must call this together (shuffles).
__device__ __forceinline__ float e4m3_block_scale(float absmax)
{
    if (!(absmax > 0.0f)) return 1.0f;
    int e = ((__float_as_uint(absmax) >> 23) & 0xFF) - 127 - 9;   // absmax is a normal float here
    while (absmax > ldexpf(448.0f, e)) ++e;
    return ldexpf(1.0f, e);
}

template <int kSw = 128>
__device__ __forceinline__ void gen_block_e4m3(const int* idx, int slot0, bool valid_rows, uint32_t rowgrp,
                                               uint32_t s_lo, uint32_t lsw, const PhiloxRoundKeys& rk,
                                               const unsigned char* stage, int stride, bool odd_negative,
                                               unsigned char* tile, int row0, int chunk)
{
    float v[4][8];
    if (valid_rows) {
        int ks[8];
        uint4 w[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            ks[u] = idx[slot0 + u];
            w[u] = philox4x32_10_rk(make_uint4(rowgrp, static_cast<uint32_t>(max(ks[u], 0)), s_lo, lsw), rk);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
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
            for (int u = 0; u < 8; ++u) v[r][u] = 0.0f;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        float am = 0.0f;
#pragma unroll
        for (int u = 0; u < 8; ++u) am = fmaxf(am, fabsf(v[r][u]));
        am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, 1));
        am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, 2));
        const float sc = e4m3_block_scale(am);
        const float inv = 1.0f / sc;   // exact: a power of two
        uint32_t packed[4];
#pragma unroll
        for (int u2 = 0; u2 < 4; ++u2) {
            const __nv_fp8x2_storage_t q =
                __nv_cvt_float2_to_fp8x2(make_float2(v[r][2 * u2] * inv, v[r][2 * u2 + 1] * inv), __NV_SATFINITE,
                                         __NV_E4M3);
            const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(q, __NV_E4M3);
            const float2 d = __half22float2(*reinterpret_cast<const __half2*>(&hr));
            packed[u2] = pack_bf16x2(d.x * sc, d.y * sc);
        }
        *reinterpret_cast<uint4*>(tile + tile_offset<kSw>(row0 + r, chunk)) =
            make_uint4(packed[0], packed[1], packed[2], packed[3]);
    }
}

template <int MH, int BN, int Q, bool kBatch, int P = 0>
__global__ void __launch_bounds__(kThreads, 1)
level_tc_bf16_kernel(const __grid_constant__ LevelParams prm_arg, const TcExtra ex, const TcBatch bt)
{
    using C = TcCfg<MH, BN, Q, P>;
    static_assert(C::kFits, "shared memory");
    static_assert(!(P && kBatch), "pairs run single-problem launches");
    constexpr int kSub = C::kSub;
    constexpr int kSlices = C::kSlices;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~static_cast<uintptr_t>(1023));
    unsigned char* a_tile = smem;
    unsigned char* b_tile = smem + C::kABytes;
    unsigned char* staging = smem + C::kTileBytes;  // [2][kStageBytes]
    int* idx_s = reinterpret_cast<int*>(staging + 2 * C::kStageBytes);  // [2][kSub]
    uint64_t* bars = reinterpret_cast<uint64_t*>(idx_s + 2 * kSub);
    uint32_t* tmem_s = reinterpret_cast<uint32_t*>(bars + C::kNumBars);
    volatile int* abort_s = reinterpret_cast<volatile int*>(tmem_s + 1);
    double* red_s = reinterpret_cast<double*>(tmem_s + 4);
    // batched launches: each role keeps its own copy of the current job's parameters (aligned as
    // the type requires: it embeds tensor maps)
    LevelParams* job_prod = reinterpret_cast<LevelParams*>(
        (reinterpret_cast<uintptr_t>(red_s + kGenWarps) + alignof(LevelParams) - 1) &
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
            const int i0 = bt.cta_begin[blockIdx.x], i1 = bt.cta_begin[blockIdx.x + 1];
            for (int i = i0; i < i1; ++i) {
                const uint64_t it = bt.items[i];
                const int job = static_cast<int>(it & 0xFFFFu);
                if (job != cur) {
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
                for (int cy = cy0; cy < cy0 + ncy && go; ++cy) go = body_fn(*copy, cy, tile, maps);
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
            for (uint64_t s = sa; s < sb && !aborted; ++s) {
                const uint32_t lsw = level_sample_word(prm.l, s);
                const uint32_t s_lo = static_cast<uint32_t>(s);
                for (int j = 0; j < nsub; ++j, ++g) {
                    const int b = static_cast<int>(g & 1);
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
                    const int t0 = j * kSub;
                    if (lane < kSub / 2) {
                        const int t = t0 + 2 * lane;
                        int64_t r0 = -1, r1 = -1;
                        if (t < prm.c) index_pair(prm.keyI, lsw, s_lo, t >> 1, static_cast<uint64_t>(prm.n), r0, r1);
                        idx[2 * lane] = t < prm.c ? static_cast<int>(r0) : -1;
                        idx[2 * lane + 1] = t + 1 < prm.c ? static_cast<int>(r1) : -1;
                    }
                    __syncwarp();
                    const int nvalid = min(kSub, prm.c - t0);
                    // staging buffer b: the A parts of the kSub slots, then their B parts
                    unsigned char* stg = staging + b * C::kStageBytes;
                    const uint32_t a_region = tc::smem_addr(stg);
                    const uint32_t b_region = a_region + static_cast<uint32_t>(kSub * C::kRows * 8);
                    if (gather) {
                        // TMA row gathers, four slots per instruction (boxes of kRows and kBGen pairs)
                        const int groups = (nvalid + 3) / 4;
                        if (lane == 0)
                            tc::mbar_arrive_expect_tx(bar_full(b),
                                                      static_cast<uint32_t>(groups * 4 * (C::kRows + C::kBGen) * 8));
                        __syncwarp();
                        if (lane < groups) {
                            const int r0 = max(idx[4 * lane], 0), r1 = max(idx[4 * lane + 1], 0);
                            const int r2 = max(idx[4 * lane + 2], 0), r3 = max(idx[4 * lane + 3], 0);
                            tc::tma_gather4(a_region + static_cast<uint32_t>(4 * lane * C::kRows * 8), &maps->a, tm0,
                                            r0, r1, r2, r3, bar_full(b));
                            tc::tma_gather4(b_region + static_cast<uint32_t>(4 * lane * C::kBGen * 8), &maps->b,
                                            prm.m_pad + geo.bcol0, r0, r1, r2, r3, bar_full(b));
                        }
                    } else {
                        if (lane == 0)
                            tc::mbar_arrive_expect_tx(bar_full(b), static_cast<uint32_t>(nvalid) * (a_bytes + b_bytes));
                        __syncwarp();
                        if (lane < nvalid) {
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
    } else {
        // ---------------- generator warps: entries, MMA issue, drain ----------------------------
        constexpr uint32_t idesc = tc::idesc_bf16_f32(128, BN);
        constexpr int kItemsA = (C::kRows / 4) * (kSub / 8);
        constexpr int kItemsB = (C::kBGen / 4) * (kSub / 8);
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
            const bool coarse_sign = prm.l > 0;
            const float scale = static_cast<float>(prm.w_fine);
            const Geo geo = geometry(prm, tile);
            const int tm0 = geo.tm0;
            const int tp0 = geo.tp0;
            const int brow0 = geo.bcol0 - tp0;   // first row of this CTA's part of the transposed B tile
            const uint64_t chunk = prm.chunk0 + static_cast<uint64_t>(cy);
            const uint64_t sa = max(prm.s_begin, chunk * static_cast<uint64_t>(prm.chunk));
            const uint64_t sb = min(prm.s_end, (chunk + 1) * static_cast<uint64_t>(prm.chunk));
            float* part = static_cast<float*>(prm.partial_sum) + static_cast<int64_t>(cy) * prm.m * prm.p;
            double q = 0.0;
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
                const int hgrp = warp >> 2;
                const bool split = MH == 1 && BN >= 64;
                dr.quarter = warp & 3;
                dr.col_tm = MH == 2 ? hgrp * BN : (split ? hgrp * (BN / 2) : 0);
                dr.col_d = MH == 2 ? 0 : dr.col_tm;
                dr.ncols = MH == 2 ? BN : (split ? BN / 2 : (hgrp == 0 ? BN : 0));
                dr.gi = tm0 + (MH == 2 ? hgrp * 128 : 0) + dr.quarter * 32 + lane;
            }
            // Write (first) or add 64 drained columns starting at column cb of this thread's row.
            auto store_cols = [&](const float* v, int cb, int nv, bool first) {
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
                            if (first)
                                reinterpret_cast<float4*>(dst)[e4] =
                                    make_float4(w[4 * e4], w[4 * e4 + 1], w[4 * e4 + 2], w[4 * e4 + 3]);
                            else
                                tc::red_add_v4(dst + 4 * e4, w[4 * e4], w[4 * e4 + 1], w[4 * e4 + 2], w[4 * e4 + 3]);
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < 32; ++e)
                            if (e < valid) {
                                if (first)
                                    dst[e] = w[e];
                                else
                                    atomicAdd(dst + e, w[e]);
                            }
                    }
                }
            };
            for (uint64_t s = sa; s < sb && !aborted; ++s) {
                const uint32_t lsw = level_sample_word(prm.l, s);
                const uint32_t s_lo = static_cast<uint32_t>(s);
                for (int j = 0; j < nsub; ++j, ++g) {
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
                        constexpr int kGroups = kSub / 8;   // 8-slot groups per sub-block
                        for (int it = tid; it < kItemsA + kItemsB; it += kGenThreads) {
                            if constexpr (Q == 0) {
                                // consecutive threads take consecutive row groups
                                if (it < kItemsA) {
                                    // 4 rows of A x 8 slots
                                    const int g4 = it % (C::kRows / 4);
                                    const int sg = it / (C::kRows / 4);
                                    const int i = tm0 + 4 * g4;
                                    if constexpr (P)
                                        gen_block<64>(idx, sg * 8, i < prm.m, static_cast<uint32_t>(i >> 2), s_lo,
                                                      lsw, prm.rkA, st + (sg * 8) * (C::kRows * 8) + g4 * 32,
                                                      C::kRows * 8, false, a_tile + kk * C::kASliceBytes, 4 * g4, sg);
                                    else
                                        gen_block(idx, sg * 8, i < prm.m, static_cast<uint32_t>(i >> 2), s_lo, lsw,
                                                  prm.rkA, st + (sg * 8) * (C::kRows * 8) + g4 * 32, C::kRows * 8,
                                                  false, a_tile, 4 * g4, kGroups * kk + sg);
                                } else {
                                    // 4 columns of B (rows of the transposed tile) x 8 slots, sign folded in;
                                    // a pair also writes them into the peer's B tile
                                    const int it2 = it - kItemsA;
                                    const int g4 = it2 % (C::kBGen / 4);
                                    const int sg = it2 / (C::kBGen / 4);
                                    const int jc = geo.bcol0 + 4 * g4;
                                    if constexpr (P)
                                        gen_block<64>(idx, sg * 8, jc < prm.p, static_cast<uint32_t>(jc >> 2), s_lo,
                                                      lsw, prm.rkB, stB + (sg * 8) * (C::kBGen * 8) + g4 * 32,
                                                      C::kBGen * 8, coarse_sign, b_tile + kk * C::kBSliceBytes,
                                                      brow0 + 4 * g4, sg);
                                    else
                                        gen_block(idx, sg * 8, jc < prm.p, static_cast<uint32_t>(jc >> 2), s_lo, lsw,
                                                  prm.rkB, stB + (sg * 8) * (C::kBGen * 8) + g4 * 32,
                                                  C::kBGen * 8, coarse_sign, b_tile, brow0 + 4 * g4,
                                                  kGroups * kk + sg);
                                }
                            } else {
                                // E4M3: the kGroups threads of one row group are adjacent lanes, so the
                                // block maximum is a shuffle; a warp is all-A or all-B (kItemsA % 32 == 0)
                                // (pairs: slice tiles in the 64-byte swizzle, as for bfloat16)
                                if (it < kItemsA) {
                                    const int g4 = it / kGroups, sg = it % kGroups;
                                    const int i = tm0 + 4 * g4;
                                    if constexpr (P)
                                        gen_block_e4m3<64>(idx, sg * 8, i < prm.m, static_cast<uint32_t>(i >> 2), s_lo,
                                                           lsw, prm.rkA, st + (sg * 8) * (C::kRows * 8) + g4 * 32,
                                                           C::kRows * 8, false, a_tile + kk * C::kASliceBytes, 4 * g4,
                                                           sg);
                                    else
                                        gen_block_e4m3(idx, sg * 8, i < prm.m, static_cast<uint32_t>(i >> 2), s_lo, lsw,
                                                       prm.rkA, st + (sg * 8) * (C::kRows * 8) + g4 * 32, C::kRows * 8,
                                                       false, a_tile, 4 * g4, kGroups * kk + sg);
                                } else {
                                    const int it2 = it - kItemsA;
                                    const int g4 = it2 / kGroups, sg = it2 % kGroups;
                                    const int jc = geo.bcol0 + 4 * g4;
                                    if constexpr (P)
                                        gen_block_e4m3<64>(idx, sg * 8, jc < prm.p, static_cast<uint32_t>(jc >> 2), s_lo,
                                                           lsw, prm.rkB, stB + (sg * 8) * (C::kBGen * 8) + g4 * 32,
                                                           C::kBGen * 8, coarse_sign, b_tile + kk * C::kBSliceBytes,
                                                           brow0 + 4 * g4, sg);
                                    else
                                        gen_block_e4m3(idx, sg * 8, jc < prm.p, static_cast<uint32_t>(jc >> 2), s_lo, lsw,
                                                       prm.rkB, stB + (sg * 8) * (C::kBGen * 8) + g4 * 32,
                                                       C::kBGen * 8, coarse_sign, b_tile, brow0 + 4 * g4,
                                                       kGroups * kk + sg);
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
                        if (jj == nsub - 1) tc::mma_commit(bar_done);
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
                            if (j == nsub - 1) {
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
                if constexpr (C::kAccS) {
                    // ||D||^2 of the sample from its accumulator; the sum stays in tensor memory
                    for (int cb = 0; cb < dr.ncols; cb += 64) {
                        float v[64];
                        const uint32_t ta = dr.taddr(tmem, cb);
                        tc::tmem_ld_32x32b_x32_nowait(ta, v);
                        if (cb + 32 < dr.ncols) tc::tmem_ld_32x32b_x32_nowait(ta + 32, v + 32);
                        tc::tmem_ld_wait();
                        const int nv = min(64, dr.ncols - cb);
                        float qs = 0.0f;
#pragma unroll
                        for (int e = 0; e < 64; ++e)
                            if (e < nv) qs = fmaf(v[e], v[e], qs);
                        q += static_cast<double>(qs) * scale_sq;
                    }
                } else {
                    const bool first = (s == sa);
                    // two 32-column loads in flight per wait
                    for (int cb = 0; cb < dr.ncols; cb += 64) {
                        float v[64];
                        const uint32_t ta = dr.taddr(tmem, cb);
                        tc::tmem_ld_32x32b_x32_nowait(ta, v);
                        if (cb + 32 < dr.ncols) tc::tmem_ld_32x32b_x32_nowait(ta + 32, v + 32);
                        tc::tmem_ld_wait();
                        const int nv = min(64, dr.ncols - cb);
                        float qs = 0.0f;
#pragma unroll
                        for (int e = 0; e < 64; ++e) {
                            if (e < nv) {
                                v[e] *= scale;
                                qs = fmaf(v[e], v[e], qs);
                            }
                        }
                        q += static_cast<double>(qs);
                        store_cols(v, cb, nv, first);
                    }
                }
                tc::tc_fence_before_sync();
                tc::named_barrier(kGenBarrier, kGenThreads);  // the accumulator may now be overwritten
            }
            if (aborted) return false;
            if constexpr (C::kAccS) {
                // the chunk's sum of D: one store per element of the tile
                tc::tc_fence_after_sync();
                for (int cb = 0; cb < dr.ncols; cb += 64) {
                    float v[64];
                    const uint32_t ta = dr.taddr(tmem + C::kTileCols, cb);
                    tc::tmem_ld_32x32b_x32_nowait(ta, v);
                    if (cb + 32 < dr.ncols) tc::tmem_ld_32x32b_x32_nowait(ta + 32, v + 32);
                    tc::tmem_ld_wait();
                    const int nv = min(64, dr.ncols - cb);
#pragma unroll
                    for (int e = 0; e < 64; ++e) v[e] *= scale;
                    store_cols(v, cb, nv, true);
                }
                tc::tc_fence_before_sync();
            }
            if (aborted) return false;
            // work-item epilogue: sum of ||D||^2 of this tile over the chunk, fixed-order reduction
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
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, level_tc_bf16_kernel<MH, BN, Q, kBatch>, kThreads,
                                                      C::kSmemBytes);
    if (e != cudaSuccess) return e;
    *per_sm = max(1, min(occ, 512 / C::kTmemCols));
    return cudaSuccess;
}

template <int MH, int BN, int Q>
struct SingleF {
    static cudaError_t run(const LevelParams& prm, const TcLaunch& tl, cudaStream_t st)
    {
        using C = TcCfg<MH, BN, Q>;
        if constexpr (!C::kFits) {
            return cudaErrorInvalidValue;
        } else {
            int per_sm = 1;
            cudaError_t e = prepare<MH, BN, Q, false>(&per_sm);
            if (e != cudaSuccess) return e;
            const int items = prm.nchunks * prm.tiles_m * prm.tiles_p;
            const int grid = max(1, min(items, per_sm * tl.num_sms));
            TcExtra ex{tl.err_flag, tl.timeout_ns, items, tl.scale};
            level_tc_bf16_kernel<MH, BN, Q, false><<<grid, kThreads, C::kSmemBytes, st>>>(prm, ex, TcBatch{});
            return cudaGetLastError();
        }
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
            level_tc_bf16_kernel<MH, BN, Q, true><<<grid, kThreads, C::kSmemBytes, st>>>(none, ex, bt);
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

// A cluster pair (two CTAs, 128 rows each) on one 256 x 256 output tile.
template <int Q>
cudaError_t launch_pair(const LevelParams& prm, const TcLaunch& tl, cudaStream_t st)
{
    using C = TcCfg<1, 256, Q, 1>;
    auto kern = level_tc_bf16_kernel<1, 256, Q, false, 1>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kThreads);
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
    if (allow_pair && m > 128 && p > 128) return TcTile{1, 256, 128, 1};   // cluster pair
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
    if (tile.pair) return q ? launch_pair<1>(prm, tl, st) : launch_pair<0>(prm, tl, st);
    return dispatch_tile<SingleF>(tile, q, prm, tl, st);
}

int tc_batch_grid(const TcTile& tile, int q, int num_sms)
{
    if (!tc_tile_valid(tile, q) || tile.pair) return 0;
    return dispatch_tile<GridF>(tile, q, num_sms);
}

cudaError_t launch_level_tc_batch(const TcBatch& bt, const TcTile& tile, int q, int grid, const TcLaunch& tl,
                                  cudaStream_t st)
{
    if (!tc_tile_valid(tile, q) || tile.pair) return cudaErrorInvalidValue;
    return dispatch_tile<BatchF>(tile, q, bt, grid, tl, st);
}

}  // namespace mlmc
