// sampler.cuh -- in-register counter-based Gaussian sampler for the Picard sweep.
//
// Sample i of evaluation state m in sweep k, dims 4j..4j+3, is drawn from one
// Philox4x32-10 block (Salmon et al., SC'11) with counter (i, j, m, k) and key
// (seed_lo, seed_hi ^ instance).  Nothing is written to memory: the heat-kernel
// expectation of Prop. 2.1 / Cor. B.4 consumes each draw where it is made.
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

// The 23 high bits of r as a float in [1, 2): 1 + (r >> 9) 2^-23 (exact).
__device__ __forceinline__ float mant_one_two(uint32_t r) {
    return __uint_as_float((r >> 9) | 0x3F800000u);
}

// u = ((r >> 9) + 0.5) 2^-23, exactly (the sum below is exact in binary32).
__device__ __forceinline__ float u01(uint32_t r) {
    return mant_one_two(r) + (-1.0f + 0x1.0p-24f);
}

// Box-Muller radius sqrt(-2 ln u) from the radius word.
__device__ __forceinline__ float bm_radius(uint32_t r) {
    const float u = u01(r);
    // -2 ln u = -2 ln2 * log2 u; clamp: near u = 1 the approximate log2 may cross 0.
    const float t = fmaxf(-1.3862943611198906f * lg2_approx(u), 0.0f);
    return sqrt_approx(t);
}

// Box-Muller angle: returns phi = 2 pi (u - 1/2) in (-pi, pi); the pair is
// (r cos 2 pi u, r sin 2 pi u) = (-r cos phi, -r sin phi).
__device__ __forceinline__ float bm_phase(uint32_t r) {
    const float t = (mant_one_two(r) - 1.5f) + 0x1.0p-24f;   // u - 1/2, exact
    return t * 6.283185307179586f;
}

// Standard normals of dims [4*q0, 4*q0 + 4*NQ) for one sample, keeping only the first
// NUSE of them (the rest are never computed).
template <int NQ, int NUSE>
__device__ __forceinline__ void draw_normals(uint32_t sample, uint32_t q0, uint32_t point,
                                             uint32_t sweep, uint32_t k0, uint32_t k1,
                                             float* z) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int b = 4 * q;
        if (b >= NUSE) break;
        const uint4 r = philox4x32_10(make_uint4(sample, q0 + q, point, sweep), k0, k1);
        {
            const float ra = bm_radius(r.x);
            const float ph = bm_phase(r.y);
            z[b] = -ra * cos_approx(ph);
            if (b + 1 < NUSE) z[b + 1] = -ra * sin_approx(ph);
        }
        if (b + 2 < NUSE) {
            const float rb = bm_radius(r.z);
            const float ph = bm_phase(r.w);
            z[b + 2] = -rb * cos_approx(ph);
            if (b + 3 < NUSE) z[b + 3] = -rb * sin_approx(ph);
        }
    }
}

}  // namespace hjg
