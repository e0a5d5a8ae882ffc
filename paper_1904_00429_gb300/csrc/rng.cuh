// rng.cuh -- device-side counter-based draws of the MLMC estimator.
//
// Every random number the estimator consumes is a pure function of its
// coordinates, so any thread can produce any draw without state:
//   * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): a 10-round keyed
//     bijection of a 128-bit counter; each round takes the double-width
//     products of words 0 and 2 with two odd multipliers and mixes their high
//     halves with the other words and the round key, which advances by two
//     Weyl increments between rounds.
//   * uniforms u = (w + 1/2) 2^-32 in (0, 1);
//   * normals by Box-Muller on word pairs: radius from the first word,
//     angle 2 pi u from the second, cosine for even and sine for odd entries
//     (four normals per block: entries 4q..4q+3 of one column);
//   * indices of the uniform law xi_j = 1/n (Eq. unique):
//     floor(word64 * n / 2^64).
// Counter layout (level l < 256, sample s < 2^56):
//   A entry (i, k): key (seed_A, problem), ctr (i/4, k, s_lo, s_hi << 8 | l)
//   B entry (k, j): key (seed_B, problem), ctr (j/4, k, s_lo, s_hi << 8 | l)
//   slot t index:   key (seed_idx, problem), ctr (t/2, 0xFFFFFFFF, s_lo, s_hi << 8 | l)
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mlmc {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;
constexpr uint32_t kIndexStream = 0xFFFFFFFFu;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k.x += kPhiloxW0;
            k.y += kPhiloxW1;
        }
        const uint32_t hi0 = __umulhi(kPhiloxM0, c.x);
        const uint32_t lo0 = kPhiloxM0 * c.x;
        const uint32_t hi1 = __umulhi(kPhiloxM1, c.z);
        const uint32_t lo1 = kPhiloxM1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Round keys of Philox4x32-10: k_r = key + r (W0, W1), r = 0..9 (the schedule above, precomputed
// once per launch so that the rounds read them as kernel-parameter operands).
struct PhiloxRoundKeys {
    uint2 k[10];
};

__host__ __device__ inline PhiloxRoundKeys philox_round_keys(uint2 key)
{
    PhiloxRoundKeys rk;
    for (int r = 0; r < 10; ++r) {
        rk.k[r] = make_uint2(key.x + static_cast<uint32_t>(r) * kPhiloxW0, key.y + static_cast<uint32_t>(r) * kPhiloxW1);
    }
    return rk;
}

__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const PhiloxRoundKeys& rk)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t hi0 = __umulhi(kPhiloxM0, c.x);
        const uint32_t lo0 = kPhiloxM0 * c.x;
        const uint32_t hi1 = __umulhi(kPhiloxM1, c.z);
        const uint32_t lo1 = kPhiloxM1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ rk.k[round].x, lo1, hi0 ^ c.w ^ rk.k[round].y, lo0);
    }
    return c;
}

__host__ __device__ __forceinline__ uint32_t level_sample_word(int l, uint64_t s)
{
    return static_cast<uint32_t>(((s >> 32) << 8) | static_cast<uint64_t>(l & 0xFF));
}

// Index r_t for slot pair (t & ~1, t | 1) of one sample: both from one block.
__device__ __forceinline__ void index_pair(uint2 key, uint32_t lsw, uint32_t s_lo, int64_t t_pair,
                                           uint64_t n, int64_t& r_even, int64_t& r_odd)
{
    const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(t_pair), kIndexStream, s_lo, lsw), key);
    const uint64_t even = (static_cast<uint64_t>(w.y) << 32) | w.x;
    const uint64_t odd = (static_cast<uint64_t>(w.w) << 32) | w.z;
    r_even = static_cast<int64_t>(__umul64hi(even, n));
    r_odd = static_cast<int64_t>(__umul64hi(odd, n));
}

// Index r_t for one slot's 64-bit word under a tabulated law (xi** of Thm 3.1): u = (word >> 11)
// 2^-53 in [0, 1), x = u Q[n-1], r = the smallest j with x < Q[j] (Q the running sums of the
// weights q), or the last j with q[j] > 0 when rounding put x at Q[n-1].  The guide table G (n
// buckets; G[b] = the smallest j with Q[j] > b Q[n-1] / n, see xi_guide_kernel) gives a start
// at or below the answer, from which a forward scan finds it: the same j as a full search.
__device__ __forceinline__ int64_t index_from_cdf(uint64_t word, const double* __restrict__ Q,
                                                  const double* __restrict__ q, const int* __restrict__ G,
                                                  int64_t n)
{
    const double Qtot = Q[n - 1];
    const double u = __ull2double_rn(word >> 11) * 0x1p-53;
    const double x = __dmul_rn(u, Qtot);
    if (!(x < Qtot)) {
        int64_t j = n - 1;
        while (j > 0 && !(q[j] > 0.0)) --j;
        return j;
    }
    // bucket of x, one bucket lower to absorb the rounding of u n and of the bucket bounds
    int64_t b = static_cast<int64_t>(u * static_cast<double>(n));
    b = b < 1 ? 0 : (b > n ? n - 1 : b - 1);
    int64_t j = G[b];
    while (!(x < Q[j])) ++j;   // ends: x < Q[n-1]
    return j;
}

// The two 64-bit index words of slot pair (t & ~1, t | 1) of one sample (even slot first).
__device__ __forceinline__ void index_words(uint2 key, uint32_t lsw, uint32_t s_lo, int64_t t_pair, uint64_t& even,
                                            uint64_t& odd)
{
    const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(t_pair), kIndexStream, s_lo, lsw), key);
    even = (static_cast<uint64_t>(w.y) << 32) | w.x;
    odd = (static_cast<uint64_t>(w.w) << 32) | w.z;
}

// ---- FP64 normals ---------------------------------------------------------

__device__ __forceinline__ double uniform_f64(uint32_t w)
{
    return (static_cast<double>(w) + 0.5) * 0x1p-32;
}

__device__ __forceinline__ void box_muller_f64(uint32_t wr, uint32_t wa, double& zc, double& zs)
{
    const double radius = sqrt(-2.0 * log(uniform_f64(wr)));
    double s, c;
    sincospi(2.0 * uniform_f64(wa), &s, &c);
    zc = radius * c;
    zs = radius * s;
}

__device__ __forceinline__ void normals4_f64(uint4 w, double z[4])
{
    box_muller_f64(w.x, w.y, z[0], z[1]);
    box_muller_f64(w.z, w.w, z[2], z[3]);
}

// ---- FP32 normals ---------------------------------------------------------
//
// -ln u with u = (w + 1/2) 2^-32 loses all relative accuracy near u = 1 if u
// is first rounded to FP32.  Writing v = 1 - u = (~w + 1/2) 2^-32 (both u and
// v are FP32-accurate to 2^-24 relatively) and -ln u = log1p(v / u) keeps a
// few ulps of relative accuracy over the whole range without a branch.

__device__ __forceinline__ float neg_log_uniform_f32(uint32_t w)
{
    const float u = fmaf(__uint2float_rn(w), 0x1p-32f, 0x1p-33f);
    const float v = fmaf(__uint2float_rn(~w), 0x1p-32f, 0x1p-33f);
    return log1pf(__fdividef(v, u));
}

__device__ __forceinline__ void box_muller_f32(uint32_t wr, uint32_t wa, float& zc, float& zs)
{
    const float radius = sqrtf(2.0f * neg_log_uniform_f32(wr));
    const float x = fmaf(__uint2float_rn(wa), 0x1p-31f, 0x1p-32f);  // 2u
    float s, c;
    sincospif(x, &s, &c);
    zc = radius * c;
    zs = radius * s;
}

__device__ __forceinline__ void normals4_f32(uint4 w, float z[4])
{
    box_muller_f32(w.x, w.y, z[0], z[1]);
    box_muller_f32(w.z, w.w, z[2], z[3]);
}

// ---- FP32 normals from the special-function units (reduced-precision paths) -----------
//
// For entries that are rounded to bfloat16 or FP8 right after generation, Box-Muller runs on
// the MUFU approximations: rho^2 = -2 ln 2 lg2(u) (absolute error of lg2 about 2^-22, so the
// radius keeps full relative accuracy except for rho < 2^-6, probability 2^-13, where its
// absolute error stays below 2^-11; u rounded to 1 for w >= 2^32 - 2^7 gives rho = 0 instead of
// at most 2^-12), and the angle 2 pi u = theta + pi with theta in [-pi, pi) so that
// sin.approx / cos.approx run inside their accurate range (absolute error about 2^-21);
// cos(theta + pi) = -cos(theta), sin(theta + pi) = -sin(theta).

__device__ __forceinline__ void box_muller_mufu(uint32_t wr, uint32_t wa, float& zc, float& zs)
{
    const float u = fmaf(__uint2float_rn(wr), 0x1p-32f, 0x1p-33f);
    float l2, radius, s, c;
    asm("lg2.approx.f32 %0, %1;" : "=f"(l2) : "f"(u));
    asm("sqrt.approx.f32 %0, %1;" : "=f"(radius) : "f"(-1.3862943611198906f * l2));
    const float theta = fmaf(__int2float_rn(static_cast<int>(wa ^ 0x80000000u)), 6.283185307179586f * 0x1p-32f,
                             3.141592653589793f * 0x1p-32f);
    asm("sin.approx.f32 %0, %1;" : "=f"(s) : "f"(theta));
    asm("cos.approx.f32 %0, %1;" : "=f"(c) : "f"(theta));
    zc = -radius * c;
    zs = -radius * s;
}

__device__ __forceinline__ void normals4_mufu(uint4 w, float z[4])
{
    box_muller_mufu(w.x, w.y, z[0], z[1]);
    box_muller_mufu(w.z, w.w, z[2], z[3]);
}

template <typename T>
struct Normals;

template <>
struct Normals<double> {
    static __device__ __forceinline__ void four(uint4 w, double z[4]) { normals4_f64(w, z); }
};

template <>
struct Normals<float> {
    static __device__ __forceinline__ void four(uint4 w, float z[4]) { normals4_f32(w, z); }
};

}  // namespace mlmc
