// sampler.cuh -- in-register counter-based Gaussian sampler for the Picard sweep.
//
// For each (state m, sweep k) the sampler defines one stream of standard normals: slot q
// is lane q % 6 of Philox4x32-10 block b = q / 6, drawn with counter (m, b_lo, k, b_hi)
// and key (seed_lo, seed_hi ^ instance) (Philox: Salmon et al., SC'11).  The block index
// sits in the words the first round does not multiply, so the products of the first
// rounds that depend only on (m, k) are the same for every sample of a state and sweep.
// Each block (words X, Y, Z, W) gives three Box-Muller pairs and every one of its 128 bits
// feeds exactly one uniform: pair j (slots 6b+2j, 6b+2j+1) takes its radius from the low
// 23 bits of X, Y, Z (u = ((r & (2^23-1)) + 0.5) 2^-23) and its angle from the high 23 bits
// of W (j = 0), the high 9 bits of X then of Y (j = 1, 18 bits), the high 9 bits of Z then
// the low 9 of W (j = 2, 18 bits), with u = (k + 0.5) 2^-bits.  Sample i of a game with n
// state dimensions reads slots i*S .. i*S + n - 1, S = n for n <= 8 (consecutive samples
// packed back to back, so every Philox output is used) and S = n rounded up to a multiple
// of 6 above.  Nothing is written to memory: the heat-kernel expectation of Prop. 2.1 /
// Cor. B.4 consumes each draw where it is made.
#pragma once
#include <cstdint>

namespace hjg {

// Philox4x32-10 round constants (multipliers and Weyl key increments).
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 ctr, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)kPhiloxM0 * ctr.x;   // IMAD.WIDE.U32
        const uint64_t p1 = (uint64_t)kPhiloxM1 * ctr.z;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        ctr = make_uint4(hi1 ^ ctr.y ^ k0, lo1, hi0 ^ ctr.w ^ k1, lo0);
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return ctr;
}

// ---- fast single-instruction approximations (PTX .approx forms) ------------------
__device__ __forceinline__ float ex2_approx(float x) {
    float y; asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y; asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
    float y; asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y;
}
__device__ __forceinline__ float sin_approx(float x) {
    float y; asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y;
}
__device__ __forceinline__ float cos_approx(float x) {
    float y; asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y;
}

// The low 23 bits of r as a float in [1, 2): 1 + (r & (2^23-1)) 2^-23 (exact): a single
// three-input logic operation (r & 0x7FFFFF) | one, with `one` held in a register.
__device__ __forceinline__ float mant_one_two(uint32_t r) {
    uint32_t one = 0x3F800000u, y;
    asm("lop3.b32 %0, %1, 0x007FFFFF, %2, 0xEA;" : "=r"(y) : "r"(r), "r"(one));
    return __uint_as_float(y);
}

// u = ((r & (2^23-1)) + 0.5) 2^-23, exactly (the sum below is exact in binary32).
__device__ __forceinline__ float u01(uint32_t r) {
    return mant_one_two(r) + (-1.0f + 0x1.0p-24f);
}

// Box-Muller phase phi = 2 pi u - pi in (-pi, pi) for the angle uniform u = (k + 0.5) 2^-b,
// one FMA from the mantissa float f = 1 + k 2^-b (the b-bit field k in the top bits of the
// mantissa): phi = 2 pi f - 3 pi + pi 2^-b.  The pair is (r cos 2 pi u, r sin 2 pi u) =
// (-r cos phi, -r sin phi).
constexpr float kTwoPi = 6.283185307179586f;
constexpr float kPhase23 = -9.42477798461914f;    // -3 pi + pi 2^-23 in binary32
constexpr float kPhase18 = -9.424765586853027f;   // -3 pi + pi 2^-18 in binary32

// Pair 0: the high 23 bits of W.
__device__ __forceinline__ float bm_phase0(const uint4& r) {
    return fmaf(mant_one_two(r.w >> 9), kTwoPi, kPhase23);
}
// Pair 1: k = (X >> 23) << 9 | (Y >> 23), placed in mantissa bits 22..5.
__device__ __forceinline__ float bm_phase1(const uint4& r) {
    const uint32_t f = ((r.x >> 9) & 0x007FC000u) | ((r.y >> 18) & 0x00003FE0u) | 0x3F800000u;
    return fmaf(__uint_as_float(f), kTwoPi, kPhase18);
}
// Pair 2: k = (Z >> 23) << 9 | (W & 511), placed in mantissa bits 22..5.
__device__ __forceinline__ float bm_phase2(const uint4& r) {
    const uint32_t f = ((r.z >> 9) & 0x007FC000u) | ((r.w << 5) & 0x00003FE0u) | 0x3F800000u;
    return fmaf(__uint_as_float(f), kTwoPi, kPhase18);
}

// Per-round Philox keys (k + r W for rounds r = 0..9), computed once on the host so that
// the rounds take them straight from the constant bank.
struct PhiloxKeys {
    uint32_t k0[10], k1[10];
};

__host__ __device__ inline PhiloxKeys philox_round_keys(uint32_t k0, uint32_t k1) {
    PhiloxKeys rk;
    for (int r = 0; r < 10; ++r) {
        rk.k0[r] = k0;
        rk.k1[r] = k1;
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return rk;
}

// High and low words of a 32 x 32 product as two separate multiplies: on this part the
// low half issues at twice the rate of a widening multiply (measured: mul.lo.u32 ~64,
// mul.hi.u32 ~32, 64-bit-result multiply ~32 per SM and clock), so a Philox block formed
// this way runs ~1.3x faster than with widening multiplies.
__device__ __forceinline__ uint32_t mulhi_u32(uint32_t a, uint32_t b) {
    uint32_t r; asm("mul.hi.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b)); return r;
}
__device__ __forceinline__ uint32_t mullo_u32(uint32_t a, uint32_t b) {
    uint32_t r; asm("mul.lo.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b)); return r;
}

__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 ctr, const PhiloxKeys& rk) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t h0 = mulhi_u32(kPhiloxM0, ctr.x), l0 = mullo_u32(kPhiloxM0, ctr.x);
        const uint32_t h1 = mulhi_u32(kPhiloxM1, ctr.z), l1 = mullo_u32(kPhiloxM1, ctr.z);
        ctr = make_uint4(h1 ^ ctr.y ^ rk.k0[r], l1, h0 ^ ctr.w ^ rk.k1[r], l0);
    }
    return ctr;
}

// Box-Muller without its constant factors: the normal pair is kBmScale * (r' cos phi,
// r' sin phi) with r' = sqrt(|log2 u0|) and phi the phase above, kBmScale = -sqrt(2 ln 2).
// The sweep keeps the scale out of the per-sample loop (it folds it into sigma, the tilt
// slope and the final gradient).
constexpr float kBmScale = -1.1774100225154747f;

// Box-Muller on the four words of one Philox block: up to six normals (constant factors
// left out, see above).
template <int NUSE>
__device__ __forceinline__ void bm_normals_raw(const uint4& r, float* z) {
    {
        const float ra = sqrt_approx(fabsf(lg2_approx(u01(r.x))));
        const float ph = bm_phase0(r);
        z[0] = ra * cos_approx(ph);
        if (NUSE > 1) z[1] = ra * sin_approx(ph);
    }
    if (NUSE > 2) {
        const float rb = sqrt_approx(fabsf(lg2_approx(u01(r.y))));
        const float ph = bm_phase1(r);
        z[2] = rb * cos_approx(ph);
        if (NUSE > 3) z[3] = rb * sin_approx(ph);
    }
    if (NUSE > 4) {
        const float rc = sqrt_approx(fabsf(lg2_approx(u01(r.z))));
        const float ph = bm_phase2(r);
        z[4] = rc * cos_approx(ph);
        if (NUSE > 5) z[5] = rc * sin_approx(ph);
    }
}

// Philox block b of the stream of (point, sweep).
__device__ __forceinline__ uint4 stream_block(uint32_t b, uint32_t point, uint32_t sweep,
                                              const PhiloxKeys& rk) {
    return philox4x32_10_rk(make_uint4(point, b, sweep, 0u), rk);
}

template <int NUSE>
__device__ __forceinline__ void block_normals_raw(uint32_t b, uint32_t point, uint32_t sweep,
                                                  const PhiloxKeys& rk, float* z) {
    bm_normals_raw<NUSE>(stream_block(b, point, sweep, rk), z);
}
template <int NUSE>
__device__ __forceinline__ void block_normals(uint32_t b, uint32_t point, uint32_t sweep,
                                              uint32_t k0, uint32_t k1, float* z) {
    const PhiloxKeys rk = philox_round_keys(k0, k1);
    block_normals_raw<NUSE>(b, point, sweep, rk, z);
#pragma unroll
    for (int j = 0; j < NUSE; ++j) z[j] *= kBmScale;
}

// Normals per Philox block, slots per sample and the sample grouping that makes a group
// end on a block boundary.
constexpr int kNormalsPerBlock = 6;
__host__ __device__ constexpr int slot_stride(int n) { return n <= 8 ? n : (n + 5) / 6 * 6; }
__host__ __device__ constexpr int gcd6(int a) {
    return (a % 6 == 0) ? 6 : (a % 3 == 0) ? 3 : (a % 2 == 0) ? 2 : 1;
}
__host__ __device__ constexpr int group_samples(int n) { return 6 / gcd6(slot_stride(n)); }

__host__ __device__ constexpr int group_blocks(int n) {
    return group_samples(n) * slot_stride(n) / 6;
}

// The kernels carry a stream's block index in one 32-bit counter word (the high word is
// 0), so the groups that hold N samples of an n-dimensional state may span at most 2^32
// blocks.
__host__ __device__ constexpr bool stream_blocks_fit(int n, int64_t N) {
    return n >= 1 && N >= 0 &&
           ((uint64_t)N + group_samples(n) - 1) / group_samples(n) * (uint64_t)group_blocks(n) <= 0x100000000ull;
}

}  // namespace hjg
