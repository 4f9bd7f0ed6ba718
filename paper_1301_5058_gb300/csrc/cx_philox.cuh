// cx_philox.cuh -- Philox4x32-10 counter-based generator (Salmon, Moraes,
// Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11) and
// the random perturbation Delta of the motility sigma (Eq. CoefCrsDif;
// Sec. 3 draws it "on every grid point and at each time step" from a
// triangular law on [-1,1]).
#pragma once

#include <stdint.h>

namespace cx {

// One Philox4x32 block, 10 rounds.  A round maps (c0,c1,c2,c3) to
//   (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
// and the key advances by the Weyl increments (W0, W1) between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
    constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += W0;
        k.y += W1;
    }
    return c;
}

// Delta of cell `idx` at time step `step`.  Two 53-bit integers are cut
// from the output words, k_a = (w0 << 21) | (w1 >> 11), k_b likewise from
// (w2, w3); U = k 2^-53 is uniform on [0,1).
//   dist 0:  Delta = 2 U_a - 1          uniform on [-1,1)
//   dist 1:  Delta = U_a + U_b - 1      triangular on (-1,1)
// The numerator is an exact integer below 2^53 in magnitude, so the
// conversion and the power-of-two scaling are exact.
__device__ __forceinline__ double noise_delta(uint64_t seed, uint64_t idx, uint64_t step, int dist)
{
    const uint4 w = philox4x32_10(
        make_uint4((uint32_t)idx, (uint32_t)(idx >> 32), (uint32_t)step, (uint32_t)(step >> 32)),
        make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const long long ka = (long long)(((unsigned long long)w.x << 21) | (unsigned long long)(w.y >> 11));
    const long long kb = (long long)(((unsigned long long)w.z << 21) | (unsigned long long)(w.w >> 11));
    const long long two53 = 1LL << 53;
    const long long num = dist == 0 ? 2 * ka - two53 : ka + kb - two53;
    return (double)num * 0x1p-53;
}

// sigma = sigma0 (1 + a Delta) by the FP64 recipe, each operation rounded
// on its own.
__device__ __forceinline__ double sigma_f64(uint64_t seed, uint64_t idx, uint64_t step, int dist,
                                            double sigma0, double amp)
{
    const double d = noise_delta(seed, idx, step, dist);
    return __dmul_rn(sigma0, __dadd_rn(1.0, __dmul_rn(amp, d)));
}

// FP32 recipe, for an FP32 state whose sigma is redrawn every step (GB300's
// FP64 pipe is too slow to run the FP64 recipe per cell per step).  One
// Philox block serves four consecutive cells: counter (q lo, q hi, step lo,
// step hi) with q = idx >> 2; cell idx takes word w[h], h = idx & 3, as the
// 16-bit integers j_a = w[h] >> 16, j_b = w[h] & 0xffff:
//   dist 0:  Delta = (2 j_a - 2^16) 2^-16,   dist 1:  Delta = (j_a + j_b - 2^16) 2^-16,
// exact in FP32, then sigma0 (1 + a Delta) with each operation rounded on
// its own.
__device__ __forceinline__ float sigma_from_word(uint32_t w, int dist, float sigma0, float amp)
{
    const int ja = (int)(w >> 16), jb = (int)(w & 0xffffu);
    const int num = dist == 0 ? 2 * ja - (1 << 16) : ja + jb - (1 << 16);
    const float d = (float)num * 0x1p-16f;
    return __fmul_rn(sigma0, __fadd_rn(1.0f, __fmul_rn(amp, d)));
}

// Philox4x32-10 with the key schedule given: round r uses (kx[r], ky[r]) =
// (k0 + r W0, k1 + r W1) mod 2^32, the keys the rounds above derive one by
// one.  The schedule is the same for every cell of a launch, so the host
// computes it once and the rounds read it as operands.
__device__ __forceinline__ uint4 philox4x32_10_ks(uint4 c, const uint32_t (&kx)[10],
                                                  const uint32_t (&ky)[10])
{
    constexpr uint64_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = M0 * (uint64_t)c.x, p1 = M1 * (uint64_t)c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ kx[r], (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ ky[r], (uint32_t)p0);
    }
    return c;
}

// the Philox block of cells 4q .. 4q+3
__device__ __forceinline__ uint4 sigma_block_f32(uint64_t seed, uint64_t q, uint64_t step)
{
    return philox4x32_10(
        make_uint4((uint32_t)q, (uint32_t)(q >> 32), (uint32_t)step, (uint32_t)(step >> 32)),
        make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

__device__ __forceinline__ uint32_t block_word(const uint4 &w, int h)
{
    return h == 0 ? w.x : h == 1 ? w.y : h == 2 ? w.z : w.w;
}

__device__ __forceinline__ float sigma_f32(uint64_t seed, uint64_t idx, uint64_t step, int dist,
                                           float sigma0, float amp)
{
    const uint4 w = sigma_block_f32(seed, idx >> 2, step);
    return sigma_from_word(block_word(w, (int)(idx & 3)), dist, sigma0, amp);
}

}  // namespace cx
