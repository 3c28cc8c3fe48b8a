// sampler.cuh -- in-register counter-based Gaussian sampler for the Picard sweep.
//
// For each (state m, sweep k) the sampler defines one stream of standard normals: slot q
// is lane q % 8 of Philox4x32-10 block b = q / 8, drawn with counter (m, b_lo, k, b_hi)
// and key (seed_lo, seed_hi ^ instance) (Philox: Salmon et al., SC'11).  The block index
// sits in the words the first round does not multiply, so the products of the first
// rounds that depend only on (m, k) are the same for every sample of a state and sweep.
// Each 32-bit word of a block (X, Y, Z, W) gives one Box-Muller pair, so a block gives
// eight normals and every one of its 128 bits feeds exactly one uniform: word j makes the
// pair in slots 8b+2j, 8b+2j+1 with its radius uniform from the low 20 bits,
// u = ((w & (2^20-1)) + 0.5) 2^-20, and its angle uniform from the high 12 bits,
// u = ((w >> 20) + 0.5) 2^-12.  Sample i of a game with n state dimensions reads slots
// i*S .. i*S + n - 1, S = n for n <= 8 (consecutive samples packed back to back, so every
// Philox output is used) and S = n rounded up to a multiple of 8 above.  Nothing is written
// to memory: the heat-kernel expectation of Prop. 2.1 / Cor. B.4 consumes each draw where
// it is made.
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

// Radius uniform of one word: u = ((w & (2^20-1)) + 0.5) 2^-20, exactly.  One three-input
// logic operation builds f = 1 + (w & (2^20-1)) 2^-23 (the field in the low mantissa bits,
// `one` held in a register), and one FMA gives 8 f - 8 + 2^-21 = u (exact in binary32).
__device__ __forceinline__ float mant_low20(uint32_t w) {
    uint32_t one = 0x3F800000u, y;
    asm("lop3.b32 %0, %1, 0x000FFFFF, %2, 0xEA;" : "=r"(y) : "r"(w), "r"(one));
    return __uint_as_float(y);
}
constexpr float kRadOff = -0x1.fffffep+2f;   // -8 + 2^-21
__device__ __forceinline__ float u_radius(uint32_t w) {
    return fmaf(mant_low20(w), 8.0f, kRadOff);
}

// Box-Muller phase phi = 2 pi u - pi in (-pi, pi) for the angle uniform u = (k + 0.5) 2^-12
// of the high 12 bits k of w: phi = pi ((k + 0.5) 2^-11 - 1).  The pair is
// (r cos 2 pi u, r sin 2 pi u) = (-r cos phi, -r sin phi).

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

// The rounds with the products in one of three instruction forms (identical results):
// MULF = 0 separate high and low multiplies, 1 one widening multiply per product, 2 one of
// each per round.  Which is fastest depends on the kernel's mix of pipes (the launch
// variants carry the choice and the autotuner measures it).
template <int MULF = 0>
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 ctr, const PhiloxKeys& rk) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t h0, l0, h1, l1;
        if (MULF == 1) {
            const uint64_t p0 = (uint64_t)kPhiloxM0 * ctr.x, p1 = (uint64_t)kPhiloxM1 * ctr.z;
            h0 = (uint32_t)(p0 >> 32); l0 = (uint32_t)p0; h1 = (uint32_t)(p1 >> 32); l1 = (uint32_t)p1;
        } else if (MULF == 2) {
            const uint64_t p0 = (uint64_t)kPhiloxM0 * ctr.x;
            h0 = (uint32_t)(p0 >> 32); l0 = (uint32_t)p0;
            h1 = mulhi_u32(kPhiloxM1, ctr.z); l1 = mullo_u32(kPhiloxM1, ctr.z);
        } else {
            h0 = mulhi_u32(kPhiloxM0, ctr.x); l0 = mullo_u32(kPhiloxM0, ctr.x);
            h1 = mulhi_u32(kPhiloxM1, ctr.z); l1 = mullo_u32(kPhiloxM1, ctr.z);
        }
        ctr = make_uint4(h1 ^ ctr.y ^ rk.k0[r], l1, h0 ^ ctr.w ^ rk.k1[r], l0);
    }
    return ctr;
}

// Box-Muller without its constant factors: the normal pair is kBmScale * (r' cos phi,
// r' sin phi) with r' = sqrt(|log2 u0|) and phi the phase above, kBmScale = -sqrt(2 ln 2).
// The sweep keeps the scale out of the per-sample loop (it folds it into sigma, the tilt
// slope and the final gradient).
constexpr float kBmScale = -1.1774100225154747f;

// Box-Muller on the four words of one Philox block: up to eight normals, pair j from word
// j (constant factors left out, see above).  The calling kernel must have filled the
// angle table.
// The angle field takes one of 4,096 values, so (cos phi, sin phi) of every phase sits in a
// 32 KB shared-memory table that each CTA of a sampling kernel fills once at its start
// (bm_table_fill, then a CTA barrier): one shared load per pair instead of two MUFU
// operations, and the entries are the FP32 roundings of sincospi of the exact phase.
constexpr int kBmTableSize = 4096;
__device__ __forceinline__ float2* bm_table() {
    __shared__ float2 tab[kBmTableSize];
    return tab;
}
// Every thread of the CTA (one-dimensional CTAs) takes part; entry k holds the phase of angle
// field k, phi_k = pi ((k + 0.5) 2^-11 - 1) (the argument of sincospi is exact in FP32).
__device__ __forceinline__ void bm_table_fill() {
    float2* t = bm_table();
    for (int k = threadIdx.x; k < kBmTableSize; k += blockDim.x) {
        float s, c;
        sincospif(fmaf((float)k + 0.5f, 1.0f / 2048.0f, -1.0f), &s, &c);
        t[k] = make_float2(c, s);
    }
}

__device__ __forceinline__ void bm_pair_raw(uint32_t w, float* z, bool both) {
    const float ra = sqrt_approx(fabsf(lg2_approx(u_radius(w))));
    const float2 cs = bm_table()[w >> 20];
    z[0] = ra * cs.x;
    if (both) z[1] = ra * cs.y;
}
template <int NUSE>
__device__ __forceinline__ void bm_normals_raw(const uint4& r, float* z) {
    bm_pair_raw(r.x, z, NUSE > 1);
    if (NUSE > 2) bm_pair_raw(r.y, z + 2, NUSE > 3);
    if (NUSE > 4) bm_pair_raw(r.z, z + 4, NUSE > 5);
    if (NUSE > 6) bm_pair_raw(r.w, z + 6, NUSE > 7);
}

// Philox block b of the stream of (point, sweep).
template <int MULF = 0>
__device__ __forceinline__ uint4 stream_block(uint32_t b, uint32_t point, uint32_t sweep,
                                              const PhiloxKeys& rk) {
    return philox4x32_10_rk<MULF>(make_uint4(point, b, sweep, 0u), rk);
}

template <int NUSE, int MULF = 0>
__device__ __forceinline__ void block_normals_raw(uint32_t b, uint32_t point, uint32_t sweep,
                                                  const PhiloxKeys& rk, float* z) {
    bm_normals_raw<NUSE>(stream_block<MULF>(b, point, sweep, rk), z);
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
constexpr int kNormalsPerBlock = 8;
__host__ __device__ constexpr int slot_stride(int n) { return n <= 8 ? n : (n + 7) / 8 * 8; }
__host__ __device__ constexpr int gcd8(int a) {
    return (a % 8 == 0) ? 8 : (a % 4 == 0) ? 4 : (a % 2 == 0) ? 2 : 1;
}
__host__ __device__ constexpr int group_samples(int n) { return 8 / gcd8(slot_stride(n)); }

__host__ __device__ constexpr int group_blocks(int n) {
    return group_samples(n) * slot_stride(n) / 8;
}

// The kernels carry a stream's block index in one 32-bit counter word (the high word is
// 0), so the groups that hold N samples of an n-dimensional state may span at most 2^32
// blocks.
__host__ __device__ constexpr bool stream_blocks_fit(int n, int64_t N) {
    return n >= 1 && N >= 0 &&
           ((uint64_t)N + group_samples(n) - 1) / group_samples(n) * (uint64_t)group_blocks(n) <= 0x100000000ull;
}

}  // namespace hjg
