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
// A CTA walks the chunks of its segments as one stream with two accumulators (128 TMEM columns)
// and two vector buffers: while the MMAs of chunk c run, the threads fold chunk c - 1 (regenerating
// its output-side normals) and build the vectors of chunk c + 1.
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
constexpr int kTcWarps = kTcThreads / 32;
constexpr int kTcGroups = kTcThreads / 128;   // record groups of the epilogue (4 warps each)
constexpr int kTcRec = 64;                    // records per chunk = MMA N
constexpr int kGroupRec = kTcRec / kTcGroups;
constexpr int kTcOut = 128;                   // outputs per CTA = MMA M
constexpr int kTcMaxAtoms = 4;                // contracted entries up to 4 x 64 (resident G block)
constexpr int kSegCache = 64;                 // segment bounds fetched per refill
static_assert(kGroupRec == 16, "one 16-column TMEM load per warp and chunk");
static_assert(2 * 64 * kTcMaxAtoms <= kTcThreads, "one parameter of a row per thread");

// Shared memory, bytes from the 1024-aligned base.  Vectors, records and weights are double
// buffered: the MMA of chunk c runs while the epilogue of chunk c - 1 and the vectors of chunk
// c + 1 are computed.
struct TcAdjSmem {
    size_t g_hi, g_lo, v, zslab, row, rec, omega, red, seg, wtab, bar, total;
    __host__ __device__ explicit TcAdjSmem(int atoms)
    {
        g_hi = 0;
        g_lo = g_hi + static_cast<size_t>(atoms) * kTcOut * 128;
        v = g_lo + static_cast<size_t>(atoms) * kTcOut * 128;                 // [2][atoms][64 rows][128 B]
        zslab = v + 2 * static_cast<size_t>(atoms) * kTcRec * 128;           // [warp][4 records][32 outputs]
        row = zslab + static_cast<size_t>(kTcWarps) * 4 * 32 * 4;            // (M, S) pairs of the segment's row
        rec = row + static_cast<size_t>(atoms) * 64 * 8;                      // [2][kTcRec]
        omega = rec + 2 * kTcRec * 8;                                         // [2][kTcRec]
        red = omega + 2 * kTcRec * 4;                                         // [group][M, S][outputs]
        seg = red + static_cast<size_t>(2 * kTcGroups) * kTcOut * 8;          // [kSegCache][begin, end]
        wtab = seg + static_cast<size_t>(kSegCache) * 16;                     // [coarse][level] weights
        bar = wtab + 2 * MLMC_MAX_LEVELS * 4;                                 // 4 mbarriers, tmem address, flag
        total = bar + 64;
    }
};

struct Chunk {
    int64_t k;    // segment (contracted row of the parameters)
    int64_t c0;   // first record
    int nc;       // records (1..64)
    bool last;    // last chunk of the segment
};

// PAIR: the CTAs of output blocks 2i and 2i + 1 form a cluster; each builds the vectors of half of
// every chunk's records and sends them to the other with one bulk copy per swizzle atom (rows
// 32 rank .. 32 rank + 31 of a 64-row atom are 4 contiguous KB), so a chunk's vectors are
// generated once per pair instead of once per output block.
template <int side, int ATOMS, bool PAIR>
__global__ void __launch_bounds__(kTcThreads, 1) segment_tc_kernel(const AdjSegmentParams prm, const TcLaunch tl)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~static_cast<uintptr_t>(1023));
    constexpr int kG8 = ATOMS * 8;   // 16-byte chunks (8 entries) per contracted vector
    const int kin = side == 0 ? prm.p : prm.m;
    const int kout = side == 0 ? prm.m : prm.p;
    const int o0 = blockIdx.y * kTcOut;
    const int ob = min(kTcOut, kout - o0);
    const TcAdjSmem L(ATOMS);
    unsigned char* g_hi = smem + L.g_hi;
    unsigned char* g_lo = smem + L.g_lo;
    unsigned char* vt = smem + L.v;
    float* zslab = reinterpret_cast<float*>(smem + L.zslab);
    float* row_s = reinterpret_cast<float*>(smem + L.row);
    uint64_t* rec_s = reinterpret_cast<uint64_t*>(smem + L.rec);
    float* omega = reinterpret_cast<float*>(smem + L.omega);
    double* red = reinterpret_cast<double*>(smem + L.red);
    int64_t* seg_s = reinterpret_cast<int64_t*>(smem + L.seg);
    float* wtab = reinterpret_cast<float*>(smem + L.wtab);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);   // [0, 1]: MMA commits; [2, 3]: peer vectors
    uint32_t* tmem_s = reinterpret_cast<uint32_t*>(smem + L.bar + 32);
    volatile int* abort_s = reinterpret_cast<volatile int*>(smem + L.bar + 36);
    const uint32_t rank = PAIR ? tc::cluster_ctarank() : 0u;
    const uint32_t peer = rank ^ 1u;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::tmem_alloc(tc::smem_addr(tmem_s), 2 * kTcRec);
    if (tid == 0) {
        for (int b = 0; b < 4; ++b) tc::mbar_init(tc::smem_addr(&bar[b]), 1);
        tc::mbar_init_fence();
        *abort_s = 0;
    }
    // on a timeout both CTAs of a pair leave at the same chunk
    auto set_abort = [&]() {
        *abort_s = 1;
        if constexpr (PAIR) tc::st_cluster_u32(tc::map_to_cta(tc::smem_addr(const_cast<int*>(abort_s)), peer), 1u);
        atomicExch(tl.err_flag, MLMC_ERR_TIMEOUT);
    };
    // weight omega of a record by (coarse, level): (n / c_l - [coarse] n / c_{l-1}) / N_l
    if (tid < 2 * MLMC_MAX_LEVELS) {
        const int l = tid % MLMC_MAX_LEVELS;
        const bool coarse = tid >= MLMC_MAX_LEVELS;
        wtab[tid] = static_cast<float>((prm.w_fine[l] + (coarse ? prm.w_coarse_extra[l] : 0.0)) * prm.inv_N[l]);
    }
    // the CTA's block of G as bfloat16 hi and lo parts, K-major (K = contracted index), 128-byte swizzle
    for (int e = tid; e < kTcOut * ATOMS * 64; e += kTcThreads) {
        const int r = e / (ATOMS * 64), x = e % (ATOMS * 64);
        double g = 0.0;
        if (r < ob && x < kin)
            g = side == 0 ? prm.G[static_cast<int64_t>(o0 + r) * prm.p + x] : prm.G[static_cast<int64_t>(x) * prm.p + o0 + r];
        const float gf = static_cast<float>(g);
        const __nv_bfloat16 hi = __float2bfloat16_rn(gf);
        const __nv_bfloat16 lo = __float2bfloat16_rn(gf - __bfloat162float(hi));
        const uint32_t off = static_cast<uint32_t>((x >> 6) * kTcOut * 128) + tc::sw128_offset(r, (x & 63) >> 3) +
                             2u * static_cast<uint32_t>(x & 7);
        *reinterpret_cast<__nv_bfloat16*>(g_hi + off) = hi;
        *reinterpret_cast<__nv_bfloat16*>(g_lo + off) = lo;
    }
    tc::fence_proxy_async_smem();
    tc::tc_fence_before_sync();
    __syncthreads();
    if constexpr (PAIR) tc::cluster_sync();   // the peer's barriers exist before anything reaches them
    tc::tc_fence_after_sync();
    const uint32_t tmem = *tmem_s;
    const uint32_t peer_vt = PAIR ? tc::map_to_cta(tc::smem_addr(vt), peer) : 0u;

    const float* P = static_cast<const float*>(prm.PAB);
    const int64_t in_off = side == 0 ? 2 * static_cast<int64_t>(prm.m_pad) : 0;
    const PhiloxRoundKeys& rk_in = side == 0 ? prm.rkB : prm.rkA;
    const PhiloxRoundKeys& rk_out = side == 0 ? prm.rkA : prm.rkB;
    constexpr uint32_t idesc = tc::idesc_bf16_f32(kTcOut, kTcRec);
    const int quarter = warp & 3;   // TMEM lanes (outputs) 32 * quarter ..
    const int group = warp >> 2;    // records kGroupRec * group ..
    const int o_loc = quarter * 32 + lane;
    float* zw = zslab + warp * 128;
    const uint64_t desc_hi = tc::sw128_kmajor_desc(tc::smem_addr(g_hi));
    const uint64_t desc_lo = tc::sw128_kmajor_desc(tc::smem_addr(g_lo));
    const uint64_t desc_v0 = tc::sw128_kmajor_desc(tc::smem_addr(vt));

    // chunks of this CTA's segments k = blockIdx.x + i gridDim.x, in order (uniform across the CTA;
    // the segment bounds are fetched kSegCache segments at a time)
    int64_t k_it = blockIdx.x, c_next = 0, seg_end = 0;
    int seg_i = kSegCache - 1;
    bool started = false;
    auto advance = [&](Chunk& ch) -> bool {
        while (c_next >= seg_end) {
            if (started) k_it += gridDim.x;
            started = true;
            if (k_it >= prm.n) return false;
            if (++seg_i == kSegCache) {
                __syncthreads();   // the cache is no longer read
                if (tid < kSegCache) {
                    const int64_t k = k_it + static_cast<int64_t>(tid) * gridDim.x;
                    int64_t b = 0, e = 0;
                    if (k < prm.n) {
                        b = prm.offsets[k];
                        e = k + 1 < prm.n ? prm.offsets[k + 1] : prm.total;
                    }
                    seg_s[2 * tid] = b;
                    seg_s[2 * tid + 1] = e;
                }
                __syncthreads();
                seg_i = 0;
            }
            c_next = seg_s[2 * seg_i];
            seg_end = seg_s[2 * seg_i + 1];
        }
        ch.k = k_it;
        ch.c0 = c_next;
        ch.nc = static_cast<int>(seg_end - c_next < kTcRec ? seg_end - c_next : kTcRec);
        c_next += kTcRec;
        ch.last = c_next >= seg_end;
        return true;
    };
    // the records of a chunk (one per thread < kTcRec) and the parameters of a row (one per thread)
    // are loaded one chunk ahead
    auto load_rec = [&](const Chunk& ch) -> uint64_t { return tid < ch.nc ? prm.records[ch.c0 + tid] : 0ull; };
    auto load_row = [&](int64_t k) -> float {
        return tid < 2 * kin ? P[k * prm.ld + in_off + tid] : 0.0f;
    };

    uint32_t phase = 0;   // bit b: parity of the next completion of bar[b]
    int last_b = -1;      // buffer of the most recent commit (thread 0)
    uint32_t last_par = 0;
    int peer_armed = -1;  // thread 0: buffer whose peer vectors are expected but not yet waited for
    bool have_prev = false, aborted = false;
    Chunk prev{0, 0, 0, false};
    Chunk cur{0, 0, 0, false};
    bool have = advance(cur);
    uint64_t rec_pf = have ? load_rec(cur) : 0ull;
    float row_pf = have ? load_row(cur.k) : 0.0f;
    int64_t row_k = -1;
    double accM = 0.0, accS = 0.0;

    for (int it = 0;; ++it) {
        tc::tc_fence_before_sync();
        // the epilogue of the previous chunk is done with its buffers (pairs: in both CTAs, so the
        // vector buffer of this chunk is free on both sides)
        if constexpr (PAIR)
            tc::cluster_sync();
        else
            __syncthreads();
        if (*abort_s) {
            aborted = true;
            break;
        }
        const int buf = it & 1;
        Chunk nxt{0, 0, 0, false};
        bool have_n = false;
        if (have) {
            if (tid < kTcRec) {
                rec_s[buf * kTcRec + tid] = rec_pf;
                omega[buf * kTcRec + tid] =
                    tid < cur.nc ? wtab[((rec_pf >> 5) & 1) * MLMC_MAX_LEVELS + (rec_pf & 31)] : 0.0f;
            }
            if (cur.k != row_k) {
                // float f of the row (pair f / 2) goes to float4 (f / 4 % 4) kG8 + f / 16, so that
                // threads of consecutive 8-entry chunks read consecutive float4s
                if (tid < 2 * ATOMS * 64) row_s[(((tid >> 2) & 3) * kG8 + (tid >> 4)) * 4 + (tid & 3)] = row_pf;
                row_k = cur.k;
            }
            have_n = advance(nxt);
            if (have_n) {
                rec_pf = load_rec(nxt);
                if (nxt.k != cur.k) row_pf = load_row(nxt.k);
            }
            __syncthreads();
            // the chunk's contracted vectors, bfloat16, as the K-major B operand (one row per record);
            // a thread builds one 16-byte swizzle chunk (8 entries, two Philox blocks) at a time
            unsigned char* vb = vt + buf * (ATOMS * kTcRec * 128);
            const uint64_t* rb = rec_s + buf * kTcRec;
            constexpr int kGenRec = PAIR ? kTcRec / 2 : kTcRec;
            const int j0 = PAIR ? static_cast<int>(rank) * kGenRec : 0;
#pragma unroll 1
            for (int e = tid; e < kGenRec * kG8; e += kTcThreads) {
                const int j = j0 + e / kG8, c8 = e % kG8;
                const int x = 8 * c8;
                uint4 packed = make_uint4(0u, 0u, 0u, 0u);
                if (j < cur.nc) {
                    const uint64_t rec = rb[j];
                    const uint64_t s = rec >> 6;
                    const uint32_t lsw = level_sample_word(static_cast<int>(rec & 31), s);
                    const uint4 w0 = philox4x32_10_rk(
                        make_uint4(static_cast<uint32_t>(2 * c8), static_cast<uint32_t>(cur.k), static_cast<uint32_t>(s), lsw),
                        rk_in);
                    const uint4 w1 = philox4x32_10_rk(
                        make_uint4(static_cast<uint32_t>(2 * c8 + 1), static_cast<uint32_t>(cur.k), static_cast<uint32_t>(s), lsw),
                        rk_in);
                    float z[8];
                    normals4_mufu(w0, z);
                    normals4_mufu(w1, z + 4);
                    const float4* rp = reinterpret_cast<const float4*>(row_s) + c8;
                    float v[8];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 pq = rp[q * kG8];   // (M, S) of entries x + 2q, x + 2q + 1
                        v[2 * q] = x + 2 * q < kin ? fmaf(pq.y, z[2 * q], pq.x) : 0.0f;
                        v[2 * q + 1] = x + 2 * q + 1 < kin ? fmaf(pq.w, z[2 * q + 1], pq.z) : 0.0f;
                    }
                    const __nv_bfloat162 b0 = __floats2bfloat162_rn(v[0], v[1]);
                    const __nv_bfloat162 b1 = __floats2bfloat162_rn(v[2], v[3]);
                    const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[4], v[5]);
                    const __nv_bfloat162 b3 = __floats2bfloat162_rn(v[6], v[7]);
                    packed = make_uint4(*reinterpret_cast<const uint32_t*>(&b0), *reinterpret_cast<const uint32_t*>(&b1),
                                        *reinterpret_cast<const uint32_t*>(&b2), *reinterpret_cast<const uint32_t*>(&b3));
                }
                *reinterpret_cast<uint4*>(vb + (x >> 6) * (kTcRec * 128) + tc::sw128_offset(j, (x & 63) >> 3)) = packed;
            }
            tc::fence_proxy_async_smem();
            tc::tc_fence_before_sync();
            __syncthreads();
            bool peer_ok = true;
            if (PAIR && tid == 0) {
                // our half to the peer (counted on its barrier), then wait for the peer's half
                const uint32_t boff = static_cast<uint32_t>(buf * ATOMS * kTcRec * 128);
#pragma unroll
                for (int a = 0; a < ATOMS; ++a) {
                    const uint32_t off = boff + static_cast<uint32_t>(a * kTcRec * 128) + rank * 4096u;
                    tc::bulk_copy_s2s_cluster(peer_vt + off, tc::smem_addr(vt) + off, 4096u,
                                              tc::map_to_cta(tc::smem_addr(&bar[2 + buf]), peer));
                }
                tc::mbar_arrive_expect_tx(tc::smem_addr(&bar[2 + buf]), static_cast<uint32_t>(ATOMS * 4096));
                peer_armed = buf;
                if (!tc::mbar_wait_cluster_bounded(tc::smem_addr(&bar[2 + buf]), (phase >> (2 + buf)) & 1u,
                                                   tc::globaltimer() + tl.timeout_ns)) {
                    set_abort();
                    peer_ok = false;
                } else {
                    peer_armed = -1;
                }
                phase ^= 1u << (2 + buf);
            }
            if (tid == 0 && peer_ok) {
                tc::tc_fence_after_sync();
                const uint32_t d = tmem + static_cast<uint32_t>(buf * kTcRec);
                // descriptors advance by (byte offset >> 4) in their start-address field
                const uint64_t bdesc0 = desc_v0 + static_cast<uint64_t>((buf * ATOMS * kTcRec * 128) >> 4);
#pragma unroll
                for (int part = 0; part < 2; ++part) {
#pragma unroll
                    for (int ks = 0; ks < ATOMS * 4; ++ks) {
                        const uint64_t adesc = (part ? desc_lo : desc_hi) +
                                               static_cast<uint64_t>(((ks >> 2) * kTcOut * 128 + 32 * (ks & 3)) >> 4);
                        const uint64_t bdesc = bdesc0 + static_cast<uint64_t>(((ks >> 2) * kTcRec * 128 + 32 * (ks & 3)) >> 4);
                        tc::mma_bf16(d, adesc, bdesc, idesc, (part > 0 || ks > 0) ? 1u : 0u);
                    }
                }
                tc::mma_commit(tc::smem_addr(&bar[buf]));
                last_b = buf;
                last_par = (phase >> buf) & 1u;
            }
        }
        if (have_prev) {
            // epilogue of the previous chunk while this chunk's MMAs run
            const int pb = buf ^ 1;
            if (!tc::mbar_wait_bounded(tc::smem_addr(&bar[pb]), (phase >> pb) & 1u, tc::globaltimer() + tl.timeout_ns))
                set_abort();
            phase ^= 1u << pb;
            __syncwarp();
            tc::tc_fence_after_sync();
            float u[kGroupRec];
            tc::tmem_ld_32x32b_x16_nowait(tmem + (static_cast<uint32_t>(quarter * 32) << 16) +
                                              static_cast<uint32_t>(pb * kTcRec + group * kGroupRec),
                                          u);
            tc::tmem_ld_wait();
            const uint64_t* rb = rec_s + pb * kTcRec;
            const float* wb = omega + pb * kTcRec;
            float sm = 0.0f, ss = 0.0f;
            if (group * kGroupRec < prev.nc) {   // uniform per warp; records past nc have omega = 0
                // normals of outputs o0 + 32 quarter + 4 (lane & 7) .. + 3 for records 4 r + lane / 8 of the
                // group, passed through the warp's slab so that lane L reads output 32 quarter + L
                const int oq = quarter * 32 + 4 * (lane & 7);
                float z[kGroupRec / 4][4];
#pragma unroll
                for (int r = 0; r < kGroupRec / 4; ++r) {
                    const uint64_t rec = rb[group * kGroupRec + 4 * r + (lane >> 3)];
                    const uint64_t s = rec >> 6;
                    const uint4 w = philox4x32_10_rk(
                        make_uint4(static_cast<uint32_t>((o0 + oq) >> 2), static_cast<uint32_t>(prev.k),
                                   static_cast<uint32_t>(s), level_sample_word(static_cast<int>(rec & 31), s)),
                        rk_out);
                    normals4_mufu(w, z[r]);
                }
#pragma unroll
                for (int r = 0; r < kGroupRec / 4; ++r) {
                    reinterpret_cast<float4*>(zw)[lane] = make_float4(z[r][0], z[r][1], z[r][2], z[r][3]);
                    __syncwarp();
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int jj = 4 * r + t;
                        const float wu = wb[group * kGroupRec + jj] * u[jj];
                        sm += wu;
                        ss = fmaf(wu, zw[t * 32 + lane], ss);
                    }
                    __syncwarp();
                }
            }
            accM += static_cast<double>(sm);
            accS += static_cast<double>(ss);
            if (prev.last) {
                // the record groups of every output, summed in a fixed order
                red[(group * 2 + 0) * kTcOut + o_loc] = accM;
                red[(group * 2 + 1) * kTcOut + o_loc] = accS;
                accM = accS = 0.0;
                __syncthreads();
                if (tid < ob) {
                    double tm = 0.0, ts = 0.0;
#pragma unroll
                    for (int g = 0; g < kTcGroups; ++g) {
                        tm += red[(2 * g) * kTcOut + tid];
                        ts += red[(2 * g + 1) * kTcOut + tid];
                    }
                    // one CTA owns (k, o) in a launch and launches are ordered, so the
                    // fire-and-forget additions are deterministic
                    const int o = o0 + tid;
                    if (side == 0) {
                        atomicAdd(&prm.gM_t[prev.k * prm.m + o], tm);
                        atomicAdd(&prm.gS_t[prev.k * prm.m + o], ts);
                    } else {
                        atomicAdd(&prm.gMp[prev.k * prm.p + o], tm);
                        atomicAdd(&prm.gSp[prev.k * prm.p + o], ts);
                    }
                }
            }
        }
        if (!have) break;
        prev = cur;
        have_prev = true;
        cur = nxt;
        have = have_n;
    }
    if (aborted && tid == 0) {
        // no MMA may still write tensor memory when it is freed: the last commit covers every
        // earlier MMA of this thread; pairs: the peer's vectors of the last chunk may still be landing
        if (last_b >= 0)
            tc::mbar_wait_bounded(tc::smem_addr(&bar[last_b]), last_par, tc::globaltimer() + 100000000ull);
        if (PAIR && peer_armed >= 0)
            tc::mbar_wait_cluster_bounded(tc::smem_addr(&bar[2 + peer_armed]), ((phase >> (2 + peer_armed)) & 1u) ^ 1u,
                                          tc::globaltimer() + 100000000ull);
    }
    tc::tc_fence_before_sync();
    __syncthreads();
    if constexpr (PAIR) tc::cluster_sync();   // no copy can reach a CTA that left
    if (warp == 0) tc::tmem_dealloc(tmem, 2 * kTcRec);
}

template <int side, int ATOMS, bool PAIR>
cudaError_t launch_side(const AdjSegmentParams& prm, const TcLaunch& tl, cudaStream_t st)
{
    const int kout = side == 0 ? prm.m : prm.p;
    const size_t smem = TcAdjSmem(ATOMS).total + 1024;
    auto kern = segment_tc_kernel<side, ATOMS, PAIR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int oblocks = (kout + kTcOut - 1) / kTcOut;
    if constexpr (!PAIR) {
        const int64_t want = (static_cast<int64_t>(tl.num_sms) + oblocks - 1) / oblocks;
        const unsigned batches = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(prm.n, want)));
        kern<<<dim3(batches, static_cast<unsigned>(oblocks)), kTcThreads, smem, st>>>(prm, tl);
        return cudaGetLastError();
    } else {
        // pairs of output blocks (an odd count gets an idle partner block); as many batches of
        // pairs as can be resident at once
        const unsigned ypad = static_cast<unsigned>((oblocks + 1) & ~1);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 1;
        attr[0].val.clusterDim.y = 2;
        attr[0].val.clusterDim.z = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.blockDim = dim3(kTcThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cfg.gridDim = dim3(1, ypad);
        int max_clusters = 0;
        e = cudaOccupancyMaxActiveClusters(&max_clusters, kern, &cfg);
        if (e != cudaSuccess) return e;
        const int64_t want = std::max<int64_t>(1, max_clusters / static_cast<int>(ypad / 2));
        cfg.gridDim = dim3(static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(prm.n, want))), ypad);
        e = cudaLaunchKernelEx(&cfg, kern, prm, tl);
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
}

template <int side>
cudaError_t launch_atoms(const AdjSegmentParams& prm, int atoms, const TcLaunch& tl, cudaStream_t st)
{
    const bool pair = (side == 0 ? prm.m : prm.p) > kTcOut;
    switch (atoms * 2 + (pair ? 1 : 0)) {
    case 2: return launch_side<side, 1, false>(prm, tl, st);
    case 3: return launch_side<side, 1, true>(prm, tl, st);
    case 4: return launch_side<side, 2, false>(prm, tl, st);
    case 5: return launch_side<side, 2, true>(prm, tl, st);
    case 6: return launch_side<side, 3, false>(prm, tl, st);
    case 7: return launch_side<side, 3, true>(prm, tl, st);
    case 8: return launch_side<side, 4, false>(prm, tl, st);
    case 9: return launch_side<side, 4, true>(prm, tl, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool adjoint_tc_supported(int kin)
{
    return kin >= 1 && kin <= 64 * kTcMaxAtoms && TcAdjSmem(kTcMaxAtoms).total + 1024 <= 227 * 1024;
}

cudaError_t adjoint_segments_tc(const AdjSegmentParams& prm, int side, const TcLaunch& tl, cudaStream_t st)
{
    const int kin = side == 0 ? prm.p : prm.m;
    if (!adjoint_tc_supported(kin)) return cudaErrorInvalidValue;
    const int atoms = (kin + 63) / 64;
    return side == 0 ? launch_atoms<0>(prm, atoms, tl, st) : launch_atoms<1>(prm, atoms, tl, st);
}

}  // namespace mlmc
