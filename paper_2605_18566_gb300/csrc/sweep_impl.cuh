// sweep_impl.cuh -- the fused frozen-coefficient Picard sweep (Algorithm 1) on sm_103a.
//
// One CTA owns one evaluation state at a time and runs all requested sweeps for it:
// states are independent (c_m depends only on Dv at x_m; the map Gamma of Theorem 2.8 acts
// pointwise), so no grid-wide synchronisation is ever needed.  Per sweep:
//   a2  sampler    Philox4x32-10 -> uniforms -> Box-Muller, in registers (sampler.cuh)
//   a3  payoff     y = x + theta + sigma z, a = -c l(y) - <z, theta>/sigma   (base 2)
//   a4  LSE        running shift m, s = sum 2^(a-m), S_j = sum 2^(a-m) z_j, Q = sum 2^(2(a-m))
//   a5  merge      warp shuffle (FP32) -> shared-memory block combine in FP64
//   a6  recover    v = -(m ln2 - |theta|^2/2sigma^2 + ln(s/N)) / c        (Cor. B.4 / B.6)
//                  Dv = -(theta + sigma S/s) / (c sigma^2)                  (Cor. B.5 / B.6)
//                  ESS = s^2 / Q                                           (Section 2.4)
//   a7  Gamma      c = clip((2/delta) H(x, Dv) / (|Dv|^2 + eta))           (Eq. coeff_frozen)
// The incoming and outgoing v of every sweep go to a history buffer from which the
// residual kernel forms the relative L2 change of Algorithm 1.
#pragma once
#include <cuda_runtime.h>
#include <cmath>
#include <cstdint>

#include "games.cuh"
#include "sampler.cuh"

namespace hjg {

// Kernel width of one item: sigma = sqrt(delta t) for its horizon t.
struct Sig {
    double sigma_d, sigma2_d;
    float sigma, sk;          // sk = sigma kBmScale
};

struct SweepArgs {
    const float* x;           // [M][ldx] evaluation states
    float* p;                 // [M][ldp] Dv iterate (in: p^(k), out: p^(k+K))
    float* c;                 // [M] frozen coefficient (in: c^(k), out: c^(k+K))
    double* v;                // [M] value iterate (in: v^(k), out: v^(k+K))
    double* vhist;            // [K+1][M] value history (row 0 = incoming v); may be null
    float* ess;               // [M] ESS of the last sweep
    float* se;                // [M] Monte-Carlo standard error of v in the last sweep, or null
    unsigned long long* counters;  // [0] non-finite states, [1] clipped coefficients (last sweep)
    int64_t ldx, ldp, M, N;
    PhiloxKeys rk;            // Philox round keys of (seed_lo, seed_hi ^ instance)
    uint32_t k0;              // global index of the first sweep
    uint32_t pt0;             // global index of state 0 (Philox counter word 0 = pt0 + state)
    int32_t K;                // sweeps to run
    float sigma;              // sqrt(delta t)
    float sk;                 // sigma * kBmScale: y = x + theta + sk * (raw normal)
    double sigma_d, sigma2_d, delta, eta, c_min, c_max;
    const float* aux;         // [M][ldaux] per-state game data (flock neighbours), or null
    int64_t ldaux;
    const struct Sig* tsig;   // per-horizon kernel widths (item pt uses tsig[pt / m_base]), or null
    int64_t m_base;           //   states per horizon
    GameParams g;
};

// The kernel width of item pt: its horizon's entry of the table, else the solve's own.
__device__ __forceinline__ Sig item_sig(const SweepArgs& A, int64_t pt) {
    if (A.tsig) return A.tsig[pt / A.m_base];
    Sig g;
    g.sigma_d = A.sigma_d;
    g.sigma2_d = A.sigma2_d;
    g.sigma = A.sigma;
    g.sk = A.sk;
    return g;
}

// Threshold (base-2 units) above the running shift at which the sums are rescaled.
// Weights stay below 2^32 and Q below N 2^64, far inside FP32 range, while the rescale
// branch is taken only a handful of times per thread.
constexpr float kRescaleTau = 32.0f;
constexpr float kLog2e = 1.4426950408889634f;
constexpr double kLn2 = 0.69314718055994530942;

__device__ __forceinline__ float merge_factor(float m, float M) {
    return (m == -INFINITY) ? 0.0f : ex2_approx(m - M);
}

// Online accumulation of one sample with log2-weight a.
template <int NS>
__device__ __forceinline__ void lse_accumulate(float a, const float* z, float& m, float& s,
                                               float& q, float* S) {
    float d = a - m;
    if (d > kRescaleTau) {
        const float f = ex2_approx(-d);   // 2^(m_old - a); 0 on the first sample
        s *= f;
        q *= f * f;
#pragma unroll
        for (int j = 0; j < NS; ++j) S[j] *= f;
        m = a;
        d = 0.0f;
    }
    const float w = ex2_approx(d);
    s += w;
    q = fmaf(w, w, q);
#pragma unroll
    for (int j = 0; j < NS; ++j) S[j] = fmaf(w, z[j], S[j]);
}

// Butterfly merge of (m, s, q, S) across the lanes selected by the xor offsets [lo, 16].
template <int NS>
__device__ __forceinline__ void warp_merge(int lo, float& m, float& s, float& q, float* S) {
    for (int off = 16; off >= lo; off >>= 1) {
        const float mo = __shfl_xor_sync(0xffffffffu, m, off);
        const float so = __shfl_xor_sync(0xffffffffu, s, off);
        const float qo = __shfl_xor_sync(0xffffffffu, q, off);
        const float Mx = fmaxf(m, mo);
        const float f1 = merge_factor(m, Mx), f2 = merge_factor(mo, Mx);
        s = s * f1 + so * f2;
        q = q * (f1 * f1) + qo * (f2 * f2);
#pragma unroll
        for (int j = 0; j < NS; ++j) {
            const float So = __shfl_xor_sync(0xffffffffu, S[j], off);
            S[j] = S[j] * f1 + So * f2;
        }
        m = Mx;
    }
}

// Shared-memory state of one CTA.
template <int NPAD, int W, int NC>
struct SweepShared {
    double x[NPAD];       // state in FP64
    double pd[NPAD];      // Dv of the sweep just finished (FP64)
    double hc[NC > 0 ? NC : 1];  // per-state trigonometric cache of H
    double fw[W];         // block-combine factors 2^(m_w - max)
    double s, q, mx;      // combined sums and shift
    float xf[NPAD];       // state in FP32
    float p_cur[NPAD];    // Dv iterate in FP32 (the stored precision)
    float yoff[NPAD];     // x + theta (FP32), the sample mean
    float tq[NPAD];       // -theta_j log2e kBmScale / sigma (tilt slope per raw normal)
    float theta[NPAD];
    Sig sig;              // kernel width of the state's horizon
    float cneg2;          // -c log2e
    float cr;             // -cneg2 radius (0 for targets without a radius)
    float c;
    float red_m[W], red_s[W], red_q[W];
    float red_S[W][NPAD];
    // control variate: value guess, linear coefficient b (FP64, and times kBmScale in FP32
    // for the raw normals), per-warp unweighted sums of z and z (z.b), combined sums
    double v_cur, s_use, mu;
    double bd[NPAD], Sd[NPAD], z1d[NPAD], z2d[NPAD];
    float braw[NPAD];
    float red_Z1[W][NPAD], red_Z2[W][NPAD];
};

// Load state pt into shared memory (threads < NPAD) and its trigonometric cache.
template <class G, int NPAD, int W, int NC>
__device__ __forceinline__ void load_state(SweepShared<NPAD, W, NC>& sh, const SweepArgs& A,
                                           int64_t pt, int tid, float* s_aux) {
    constexpr int n = G::kN;
    if (G::kAux > 0 && tid < G::kAux) s_aux[tid] = A.aux[pt * A.ldaux + tid];
    if (tid < NPAD) {
        const float xv = tid < n ? A.x[pt * A.ldx + tid] : 0.0f;
        sh.xf[tid] = xv;
        sh.x[tid] = (double)xv;
        sh.p_cur[tid] = tid < n ? A.p[pt * A.ldp + tid] : 0.0f;
    }
    if (tid == 0) {
        if (A.vhist) A.vhist[pt] = A.v[pt];
        sh.sig = item_sig(A, pt);
        sh.v_cur = A.v[pt];
        sh.c = A.c[pt];
        sh.cneg2 = -sh.c * kLog2e;
        sh.cr = G::kRadius ? -sh.cneg2 * A.g.radius : 0.0f;
    }
    __syncthreads();
    if (NC > 0 && tid < NC) sh.hc[tid] = G::cache(sh.x, tid, s_aux);
}

// theta = -sigma^2 c p (Eq. tilt_shift) for the coming sweep and the FP32 constants the
// sample loop needs (threads < NPAD).
template <int NPAD, int W, int NC, bool TILT>
__device__ __forceinline__ void prepare_sweep(SweepShared<NPAD, W, NC>& sh, const SweepArgs& A,
                                              int n, int tid) {
    if (tid < NPAD) {
        float th = 0.0f;
        if (TILT && tid < n) th = (float)(-sh.sig.sigma2_d * (double)sh.c * (double)sh.p_cur[tid]);
        sh.theta[tid] = th;
        sh.yoff[tid] = sh.xf[tid] + th;
        sh.tq[tid] = -th * kLog2e * kBmScale / sh.sig.sigma;
        // control variate coefficient b = -c sigma Dv (0 in the tilted frame, where the
        // tilt has removed the weight's linear term)
        const double b = (!TILT && tid < n) ? -(double)sh.c * sh.sig.sigma_d * (double)sh.p_cur[tid] : 0.0;
        sh.bd[tid] = b;
        sh.braw[tid] = (float)(b * (double)kBmScale);
    }
}

// Block combine of the per-warp partials in FP64, recovery of v, Dv, ESS and the
// coefficient update.  Must be entered by all threads right after the partials are
// written; ends synchronised.
template <class G, int NPAD, int W, int NC, bool TILT, bool CV = false>
__device__ __forceinline__ void finish_sweep(SweepShared<NPAD, W, NC>& sh, const SweepArgs& A,
                                             int64_t pt, int k, int tid) {
    constexpr int n = G::kN;
    const bool last = (k + 1 == A.K);
    __syncthreads();
    if (tid < W) {
        double Mx = -INFINITY;
#pragma unroll
        for (int w = 0; w < W; ++w) Mx = fmax(Mx, (double)sh.red_m[w]);
        sh.fw[tid] = (sh.red_m[tid] == -INFINITY) ? 0.0 : exp2((double)sh.red_m[tid] - Mx);
        if (tid == 0) sh.mx = Mx;
    }
    __syncthreads();
    const double c = (double)sh.c;
    if constexpr (CV) {
        // Stein control variate (see the oracle): with mu = exp(-c v_guess) in the units of
        // the shifted weights, sum w -> sum w - mu b.(sum z) and sum w z -> sum w z - mu
        // (sum z + sum z (z.b) - N b); the uncorrected sums are kept when mu is more than a
        // factor 4 away from the sample mean weight or the corrected weight sum is not
        // positive.
        if (tid < n) {
            double s = 0.0, Sj = 0.0, z1 = 0.0, z2 = 0.0;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                s = fma(sh.fw[w], (double)sh.red_s[w], s);
                Sj = fma(sh.fw[w], (double)sh.red_S[w][tid], Sj);
                z1 += (double)sh.red_Z1[w][tid];
                z2 += (double)sh.red_Z2[w][tid];
            }
            sh.Sd[tid] = Sj * (double)kBmScale;
            sh.z1d[tid] = z1 * (double)kBmScale;
            sh.z2d[tid] = z2 * (double)kBmScale;
            if (tid == 0) {
                double q = 0.0;
#pragma unroll
                for (int w = 0; w < W; ++w) q = fma(sh.fw[w] * sh.fw[w], (double)sh.red_q[w], q);
                sh.s = s;
                sh.q = q;
            }
        }
        __syncthreads();
        if (tid == 0) {
            double th2 = 0.0, bz = 0.0;
            for (int j = 0; j < n; ++j) {
                th2 += (double)sh.theta[j] * (double)sh.theta[j];
                bz += sh.bd[j] * sh.z1d[j];
            }
            // the sampled log2-weights omit -|theta|^2 / (2 sigma^2) and are shifted by mx
            const double l2mu = (-c * sh.v_cur + th2 / (2.0 * sh.sig.sigma2_d)) * 1.4426950408889634 - sh.mx;
            const bool near = fabs(l2mu - log2(sh.s / (double)A.N)) <= 2.0;
            const double mu = near ? exp2(l2mu) : 0.0;
            const double s_cv = sh.s - mu * bz;
            const bool use = near && s_cv > 0.0 && isfinite(s_cv);
            sh.s_use = use ? s_cv : sh.s;
            sh.mu = use ? mu : 0.0;
        }
        __syncthreads();
        if (tid < n) {
            const double Sj = sh.Sd[tid] - sh.mu * (sh.z1d[tid] + sh.z2d[tid] - (double)A.N * sh.bd[tid]);
            const double pj = -((double)sh.theta[tid] + sh.sig.sigma_d * Sj / sh.s_use) / (c * sh.sig.sigma2_d);
            sh.pd[tid] = pj;
            sh.p_cur[tid] = (float)pj;
            if (last) A.p[pt * A.ldp + tid] = (float)pj;
        }
    } else {
        if (tid < n) {
            double s = 0.0, Sj = 0.0;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                s = fma(sh.fw[w], (double)sh.red_s[w], s);
                Sj = fma(sh.fw[w], (double)sh.red_S[w][tid], Sj);
            }
            Sj *= (double)kBmScale;   // the sample loop accumulates raw normals
            const double pj = -((double)sh.theta[tid] + sh.sig.sigma_d * Sj / s) / (c * sh.sig.sigma2_d);
            sh.pd[tid] = pj;
            sh.p_cur[tid] = (float)pj;
            if (last) A.p[pt * A.ldp + tid] = (float)pj;
            if (tid == 0) {
                double q = 0.0;
#pragma unroll
                for (int w = 0; w < W; ++w) q = fma(sh.fw[w] * sh.fw[w], (double)sh.red_q[w], q);
                sh.s = s;
                sh.q = q;
                sh.s_use = s;
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        double th2 = 0.0, pp = 0.0;
        bool finite = true;
        for (int j = 0; j < n; ++j) {
            th2 += (double)sh.theta[j] * (double)sh.theta[j];
            pp += sh.pd[j] * sh.pd[j];
            finite = finite && isfinite(sh.pd[j]);
        }
        const double s = sh.s;
        const double logmean = sh.mx * kLn2 - th2 / (2.0 * sh.sig.sigma2_d) + log(sh.s_use / (double)A.N);
        double v = -logmean / c;
        if (G::kObstacle && obstacle_project(sh.x, A.g, n, v, sh.pd)) {   // reach-avoid: v >= o(x)
            pp = 0.0;
            finite = true;
            for (int j = 0; j < n; ++j) {
                pp += sh.pd[j] * sh.pd[j];
                finite = finite && isfinite(sh.pd[j]);
                sh.p_cur[j] = (float)sh.pd[j];
                if (last) A.p[pt * A.ldp + j] = (float)sh.pd[j];
            }
        }
        sh.v_cur = v;
        finite = finite && isfinite(v);
        const double h = G::ham_c(sh.x, sh.hc, sh.pd, A.g);
        int clipped = 0;
        const float c_new = (float)coef_update(h, pp, A.delta, A.eta, A.c_min, A.c_max, A.g.tube, &clipped);
        if (A.vhist) A.vhist[(int64_t)(k + 1) * A.M + pt] = v;
        if (last) {
            A.v[pt] = v;
            A.c[pt] = c_new;
            A.ess[pt] = (float)(s * s / sh.q);
            if (A.se) A.se[pt] = (float)(sqrt(fmax(0.0, sh.q / (s * s) - 1.0 / (double)A.N)) / fabs(c));
            if (!finite) atomicAdd(&A.counters[0], 1ull);
            if (clipped) atomicAdd(&A.counters[1], 1ull);
        }
        sh.c = c_new;
        sh.cneg2 = -c_new * kLog2e;
        sh.cr = G::kRadius ? -sh.cneg2 * A.g.radius : 0.0f;
    }
    __syncthreads();
    if (!last) prepare_sweep<NPAD, W, NC, TILT>(sh, A, n, tid);
    __syncthreads();
}

// Last block of a group that sample t of the group reads (S slots per sample, eight
// normals per block): the sample can be consumed as soon as that block is drawn.
__host__ __device__ constexpr int last_block_of(int t, int S) { return (t * S + S - 1) / kNormalsPerBlock; }

// Box-Muller on block b of a group and every sample that block completes (compile-time
// selection once the loops are unrolled), so that the normals of a consumed sample need no
// register afterwards.
template <int GS, int S, class F>
__device__ __forceinline__ void consume_block(int b, const uint4& r, float* z, F&& sample) {
    bm_normals_raw<kNormalsPerBlock>(r, z + kNormalsPerBlock * b);
#pragma unroll
    for (int t = 0; t < GS; ++t)
        if (last_block_of(t, S) == b) sample(z + t * S);
}

// The full groups g = start, start + STRIDE, ... < full of one (state, sweep) stream, each
// turned into GB Philox blocks, 8 GB normals and GS samples of S slots handed to `sample`
// one by one as their blocks are drawn.  With PIPE the Philox block after the current one
// (the next block of this group, or the first block of the thread's next group) is drawn
// while the current block's Box-Muller and samples run (software pipelining one block
// ahead), so that each warp's instruction stream interleaves the integer multiplies of the
// generator with the transcendental and FP32 work of the samples; the one block drawn past
// the end is discarded.  With UNR2 two independent groups are drawn per iteration.  All
// forms consume identical draws.
template <int GS, int GB, int S, int STRIDE, bool PIPE, bool UNR2, int MULF, class F>
__device__ __forceinline__ void run_groups(uint32_t start, uint32_t full, uint32_t point, uint32_t sweep,
                                           const PhiloxKeys& rk, F&& sample) {
    if constexpr (PIPE) {
        uint4 r = stream_block<MULF>(start * GB, point, sweep, rk);
        for (uint32_t grp = start; grp < full; grp += STRIDE) {
            float z[kNormalsPerBlock * GB];
#pragma unroll
            for (int b = 0; b < GB; ++b) {
                const uint32_t nb = (b + 1 < GB) ? grp * GB + b + 1 : (grp + STRIDE) * GB;
                const uint4 rn = stream_block<MULF>(nb, point, sweep, rk);
                consume_block<GS, S>(b, r, z, sample);
                r = rn;
            }
        }
    } else {
        uint32_t grp = start;
        if constexpr (UNR2) {   // two independent groups per iteration (more work in flight)
            for (; grp + STRIDE < full; grp += 2 * STRIDE) {
                float z[kNormalsPerBlock * GB], y[kNormalsPerBlock * GB];
#pragma unroll
                for (int b = 0; b < GB; ++b) {
                    const uint4 ra = stream_block<MULF>(grp * GB + b, point, sweep, rk);
                    const uint4 rb = stream_block<MULF>((grp + STRIDE) * GB + b, point, sweep, rk);
                    consume_block<GS, S>(b, ra, z, sample);
                    consume_block<GS, S>(b, rb, y, sample);
                }
            }
        }
        for (; grp < full; grp += STRIDE) {
            float z[kNormalsPerBlock * GB];
#pragma unroll
            for (int b = 0; b < GB; ++b) consume_block<GS, S>(b, stream_block<MULF>(grp * GB + b, point, sweep, rk), z, sample);
        }
    }
}

// ------------------------------------------------------------------------------------
// One lane per sample stream (games with n <= 8).  A thread draws samples in groups of
// g = group_samples(n) that end on a Philox block boundary (n = 3: 2 samples from 1 block;
// n = 4: 3 samples from 2 blocks; n = 6: 1 sample from 1 block), so every normal drawn is used.
template <class G, int THREADS, int MINB, bool TILT, bool PIPE, bool CV = false, bool UNR2 = false, int MULF = 0>
__global__ void __launch_bounds__(THREADS, MINB) sweep_kernel(const SweepArgs A) {
    constexpr int n = G::kN;
    constexpr int NPAD = (n + 3) / 4 * 4;
    constexpr int W = THREADS / 32;
    constexpr int GS = group_samples(n);
    constexpr int GB = group_blocks(n);
    constexpr int KA = G::kAux > 0 ? G::kAux : 1;
    __shared__ SweepShared<NPAD, W, G::kCache> sh;
    __shared__ float s_aux[KA];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    bm_table_fill();
    __syncthreads();
    const uint32_t N32 = (uint32_t)A.N;
    const uint32_t full = N32 / GS;            // groups whose GS samples all lie inside N
    const uint32_t groups = (N32 + GS - 1) / GS;

    for (int64_t pt = blockIdx.x; pt < A.M; pt += gridDim.x) {
        load_state<G, NPAD, W, G::kCache>(sh, A, pt, tid, s_aux);
        __syncthreads();
        prepare_sweep<NPAD, W, G::kCache, TILT>(sh, A, n, tid);
        __syncthreads();

        for (int k = 0; k < A.K; ++k) {
            const uint32_t sweep = A.k0 + (uint32_t)k;
            const float cneg2 = sh.cneg2, cr = sh.cr, sk = sh.sig.sk;
            float yoff[n], tq[n];
#pragma unroll
            for (int j = 0; j < n; ++j) { yoff[j] = sh.yoff[j]; tq[j] = sh.tq[j]; }
            float auxr[KA];
#pragma unroll
            for (int j = 0; j < KA; ++j) auxr[j] = G::kAux > 0 ? s_aux[j] : 0.0f;
            float m = -INFINITY, s = 0.0f, q = 0.0f, S[n];
#pragma unroll
            for (int j = 0; j < n; ++j) S[j] = 0.0f;
            constexpr int NC1 = CV ? n : 1, NC2 = (CV && !TILT) ? n : 1;
            float Z1[NC1], Z2[NC2], braw[NC2];
#pragma unroll
            for (int j = 0; j < NC1; ++j) Z1[j] = 0.0f;
#pragma unroll
            for (int j = 0; j < NC2; ++j) { Z2[j] = 0.0f; braw[j] = (CV && !TILT) ? sh.braw[j] : 0.0f; }

            auto sample = [&](const float* zt) {
                float a = fmaf(cneg2, G::dist(zt, yoff, sk, A.g, auxr), cr);
                if (TILT) {
#pragma unroll
                    for (int j = 0; j < n; ++j) a = fmaf(zt[j], tq[j], a);
                }
                lse_accumulate<n>(a, zt, m, s, q, S);
                if constexpr (CV) {
#pragma unroll
                    for (int j = 0; j < n; ++j) Z1[j] += zt[j];
                    if constexpr (!TILT) {
                        float t = 0.0f;
#pragma unroll
                        for (int j = 0; j < n; ++j) t = fmaf(zt[j], braw[j], t);
#pragma unroll
                        for (int j = 0; j < n; ++j) Z2[j] = fmaf(zt[j], t, Z2[j]);
                    }
                }
            };
            run_groups<GS, GB, n, THREADS, PIPE, UNR2, MULF>((uint32_t)tid, full, A.pt0 + (uint32_t)pt, sweep, A.rk,
                                                            sample);
            if (GS > 1 && full < groups && tid == (int)(full % THREADS)) {   // ragged last group
                float z[kNormalsPerBlock * GB];
#pragma unroll
                for (int b = 0; b < GB; ++b)
                    block_normals_raw<kNormalsPerBlock>(full * GB + b, A.pt0 + (uint32_t)pt, sweep, A.rk,
                                                        z + kNormalsPerBlock * b);
                for (uint32_t t = 0; t < N32 - full * GS; ++t) sample(z + t * n);
            }

            warp_merge<n>(1, m, s, q, S);
            if constexpr (CV) {   // plain sums of the unweighted polynomials
#pragma unroll
                for (int off = 16; off >= 1; off >>= 1) {
#pragma unroll
                    for (int j = 0; j < NC1; ++j) Z1[j] += __shfl_xor_sync(0xffffffffu, Z1[j], off);
                    if constexpr (!TILT) {
#pragma unroll
                        for (int j = 0; j < NC2; ++j) Z2[j] += __shfl_xor_sync(0xffffffffu, Z2[j], off);
                    }
                }
            }
            if (lane == 0) {
                sh.red_m[warp] = m; sh.red_s[warp] = s; sh.red_q[warp] = q;
#pragma unroll
                for (int j = 0; j < n; ++j) sh.red_S[warp][j] = S[j];
                if constexpr (CV) {
#pragma unroll
                    for (int j = 0; j < n; ++j) {
                        sh.red_Z1[warp][j] = Z1[j];
                        sh.red_Z2[warp][j] = TILT ? 0.0f : Z2[j < NC2 ? j : 0];
                    }
                }
            }
            finish_sweep<G, NPAD, W, G::kCache, TILT, CV>(sh, A, pt, k, tid);
        }
    }
}

// Lane 0's FP64 recovery for the one-warp-per-state kernel (kept out of line so that its
// double-precision temporaries do not compete with the sample loop for registers):
// v, Dv, ESS from the merged sums, the coefficient update, and the outputs.  Updates
// p (FP32 Dv iterate) in place and returns the new FP32 coefficient.
template <class G, bool TILT>
__device__ __noinline__ float warp_recover(const SweepArgs& A, const Sig& sig, int64_t pt, int k, float c,
                                           float m, float s, float q, const double* xd, float* p,
                                           const float* S, double* pd, const float* aux) {
    constexpr int n = G::kN;
    const bool last = (k + 1 == A.K);
    const double cd = (double)c;
    const double sd = (double)s;
    double th2 = 0.0, pp = 0.0;
    bool finite = true;
    for (int j = 0; j < n; ++j) {
        const double th = TILT ? (double)(float)(-sig.sigma2_d * cd * (double)p[j]) : 0.0;
        th2 += th * th;
        const double pj = -(th + sig.sigma_d * (double)kBmScale * (double)S[j] / sd) / (cd * sig.sigma2_d);
        pd[j] = pj;
        pp += pj * pj;
        finite = finite && isfinite(pj);
    }
    double v = -((double)m * kLn2 - th2 / (2.0 * sig.sigma2_d) + log(sd / (double)A.N)) / cd;
    if (G::kObstacle && obstacle_project(xd, A.g, n, v, pd)) {   // reach-avoid: v >= o(x)
        pp = 0.0;
        finite = true;
        for (int j = 0; j < n; ++j) {
            pp += pd[j] * pd[j];
            finite = finite && isfinite(pd[j]);
        }
    }
    finite = finite && isfinite(v);
    int clipped = 0;
    const float c_new = (float)coef_update(G::ham_d(xd, pd, A.g, aux), pp, A.delta, A.eta, A.c_min,
                                           A.c_max, A.g.tube, &clipped);
    for (int j = 0; j < n; ++j) p[j] = (float)pd[j];
    if (A.vhist) A.vhist[(int64_t)(k + 1) * A.M + pt] = v;
    if (last) {
        A.v[pt] = v;
        A.c[pt] = c_new;
        A.ess[pt] = (float)(sd * sd / (double)q);
        if (A.se) A.se[pt] = (float)(sqrt(fmax(0.0, (double)q / (sd * sd) - 1.0 / (double)A.N)) / fabs(cd));
        for (int j = 0; j < n; ++j) A.p[pt * A.ldp + j] = p[j];
        if (!finite) atomicAdd(&A.counters[0], 1ull);
        if (clipped) atomicAdd(&A.counters[1], 1ull);
    }
    return c_new;
}

// ------------------------------------------------------------------------------------
// One warp per state (games with n <= 8): the 32 lanes of a warp share one state's N
// samples, the butterfly merge leaves the sums on every lane, and lane 0 alone does the
// FP64 recovery and coefficient update and broadcasts the new (c, Dv) with shuffles.
// No CTA barrier is involved, so a warp never waits for another state's epilogue.
// Chosen by the autotuner when there are many more states than warps in flight.
template <class G, int THREADS, int MINB, bool TILT, bool PIPE, bool UNR2 = false, int MULF = 0>
__global__ void __launch_bounds__(THREADS, MINB) sweep_kernel_warp(const SweepArgs A) {
    constexpr int n = G::kN;
    constexpr int GS = group_samples(n);
    constexpr int GB = group_blocks(n);
    constexpr int WPC = THREADS / 32;
    __shared__ float s_x[WPC][n];    // the warp's state and Dv iterate (FP32)
    __shared__ float s_p[WPC][n];
    __shared__ double s_xd[WPC][n];  // lane 0's FP64 work space for the recovery
    __shared__ double s_pd[WPC][n];
    __shared__ float s_S[WPC][n];
    constexpr int KA = G::kAux > 0 ? G::kAux : 1;
    __shared__ float s_aux[WPC][KA];
    bm_table_fill();
    __syncthreads();
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * WPC;
    const uint32_t N32 = (uint32_t)A.N;
    const uint32_t full = N32 / GS;
    const uint32_t groups = (N32 + GS - 1) / GS;

    for (int64_t pt = (int64_t)blockIdx.x * WPC + wl; pt < A.M; pt += nwarps) {
        if (lane < n) {
            const float xv = A.x[pt * A.ldx + lane];
            s_x[wl][lane] = xv;
            s_xd[wl][lane] = (double)xv;
            s_p[wl][lane] = A.p[pt * A.ldp + lane];
        }
        if (G::kAux > 0 && lane < G::kAux) s_aux[wl][lane] = A.aux[pt * A.ldaux + lane];
        if (lane == 0 && A.vhist) A.vhist[pt] = A.v[pt];
        float c = A.c[pt];
        const Sig sig = item_sig(A, pt);
        const float sk = sig.sk;
        __syncwarp();

        for (int k = 0; k < A.K; ++k) {
            const uint32_t sweep = A.k0 + (uint32_t)k;
            const float cneg2 = -c * kLog2e;
            const float cr = G::kRadius ? -cneg2 * A.g.radius : 0.0f;
            float yoff[n], tq[n];
#pragma unroll
            for (int j = 0; j < n; ++j) {
                const float th = TILT ? (float)(-sig.sigma2_d * (double)c * (double)s_p[wl][j]) : 0.0f;
                yoff[j] = s_x[wl][j] + th;
                tq[j] = -th * kLog2e * kBmScale / sig.sigma;
            }
            float auxr[KA];
#pragma unroll
            for (int j = 0; j < KA; ++j) auxr[j] = G::kAux > 0 ? s_aux[wl][j] : 0.0f;
            float m = -INFINITY, s = 0.0f, q = 0.0f, S[n];
#pragma unroll
            for (int j = 0; j < n; ++j) S[j] = 0.0f;
            auto sample = [&](const float* zt) {
                float a = fmaf(cneg2, G::dist(zt, yoff, sk, A.g, auxr), cr);
                if (TILT) {
#pragma unroll
                    for (int j = 0; j < n; ++j) a = fmaf(zt[j], tq[j], a);
                }
                lse_accumulate<n>(a, zt, m, s, q, S);
            };
            run_groups<GS, GB, n, 32, PIPE, UNR2, MULF>((uint32_t)lane, full, A.pt0 + (uint32_t)pt, sweep, A.rk,
                                                       sample);
            if (GS > 1 && full < groups && lane == (int)(full % 32)) {
                float z[kNormalsPerBlock * GB];
#pragma unroll
                for (int b = 0; b < GB; ++b)
                    block_normals_raw<kNormalsPerBlock>(full * GB + b, A.pt0 + (uint32_t)pt, sweep, A.rk,
                                                        z + kNormalsPerBlock * b);
                for (uint32_t t = 0; t < N32 - full * GS; ++t) sample(z + t * n);
            }
            warp_merge<n>(1, m, s, q, S);

            float c_new = 0.0f;
            if (lane == 0) {
#pragma unroll
                for (int j = 0; j < n; ++j) s_S[wl][j] = S[j];
                c_new = warp_recover<G, TILT>(A, sig, pt, k, c, m, s, q, s_xd[wl], s_p[wl], s_S[wl],
                                              s_pd[wl], s_aux[wl]);
            }
            c = __shfl_sync(0xffffffffu, c_new, 0);
            __syncwarp();
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------------------------
// 45-D multi-rocket game: two lanes per sample stream.  Lane h of a pair owns dims
// 24h..24h+23 (agents 8h..8h+7; dims 45..47 are padding), i.e. blocks 6 i + 3h + j of the
// stream (three blocks of eight normals).  The evader (agent 14, dims 42..44) sits on lane
// h = 1 as its local agent 6; its position goes to the other lane with two shuffles, each
// lane takes the minimum squared distance over its own pursuers (eight on h = 0, six on
// h = 1), and one shuffle finishes the pair's minimum.  Both lanes then hold the same
// log-weight and accumulate their own 24 S_j.
template <int THREADS, int MINB, bool TILT, bool CV = false, bool PIPE = false, int MULF = 0>
__global__ void __launch_bounds__(THREADS, MINB) sweep_kernel_r45(const SweepArgs A) {
    static_assert(!CV || TILT, "the 45-D control variate runs in the tilted frame");
    using G = Rockets45;
    constexpr int n = 45;
    constexpr int NPAD = 48;
    constexpr int W = THREADS / 32;
    constexpr int GROUPS = THREADS / 2;   // samples in flight per CTA
    constexpr int L = 24;                 // dims per lane
    __shared__ SweepShared<NPAD, W, G::kCache> sh;
    __shared__ float s_aux[1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    bm_table_fill();
    __syncthreads();
    const int h = lane & 1;
    const int grp = tid >> 1;
    const int src_e = lane | 1;
    const uint32_t N32 = (uint32_t)A.N;

    for (int64_t pt = blockIdx.x; pt < A.M; pt += gridDim.x) {
        load_state<G, NPAD, W, G::kCache>(sh, A, pt, tid, s_aux);
        __syncthreads();
        prepare_sweep<NPAD, W, G::kCache, TILT>(sh, A, n, tid);
        __syncthreads();

        for (int k = 0; k < A.K; ++k) {
            const uint32_t sweep = A.k0 + (uint32_t)k;
            const float cneg2 = sh.cneg2, cr = sh.cr, sk = sh.sig.sk;
            float yx0[8], yz0[8];
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                yx0[a] = sh.yoff[L * h + 3 * a];
                yz0[a] = sh.yoff[L * h + 3 * a + 1];
            }
            // the tilt's 24 coefficients of this lane stay in shared memory (the two lanes of
            // a pair read two addresses, broadcast to the warp): registers for the normals
            const float* tql = sh.tq + L * h;
            float m = -INFINITY, s = 0.0f, q = 0.0f, S[L];
#pragma unroll
            for (int j = 0; j < L; ++j) S[j] = 0.0f;
            float Z1[CV ? L : 1];   // control variate: plain sums of this lane's 24 normals
#pragma unroll
            for (int j = 0; j < (CV ? L : 1); ++j) Z1[j] = 0.0f;

            // The shuffles below take the whole warp, so every lane runs the trip count of
            // the warp's first group; a group whose sample index is past N draws (unused
            // blocks) and joins the shuffles but accumulates nothing.
            // With PIPE the three Philox blocks of the next sample are drawn while the
            // current sample's Box-Muller, distances and accumulation run (identical draws).
            const uint32_t g_first = (uint32_t)(grp & ~15);
            const uint32_t trips = N32 > g_first ? (N32 - g_first + GROUPS - 1) / GROUPS : 0u;
            const uint32_t point = A.pt0 + (uint32_t)pt;
            uint4 rb[3];
            if constexpr (PIPE) {
#pragma unroll
                for (int j = 0; j < 3; ++j) rb[j] = stream_block<MULF>(6u * (uint32_t)grp + 3u * h + j, point, sweep, A.rk);
            }
            for (uint32_t t = 0; t < trips; ++t) {
                const uint32_t i = (uint32_t)grp + t * (uint32_t)GROUPS;
                const bool live = i < N32;
                float z[L];
                if constexpr (PIPE) {
                    const uint32_t nx = i + (uint32_t)GROUPS;
                    uint4 rn[3];
#pragma unroll
                    for (int j = 0; j < 3; ++j) rn[j] = stream_block<MULF>(6u * nx + 3u * h + j, point, sweep, A.rk);
#pragma unroll
                    for (int j = 0; j < 3; ++j) bm_normals_raw<8>(rb[j], z + 8 * j);
#pragma unroll
                    for (int j = 0; j < 3; ++j) rb[j] = rn[j];
                } else {
#pragma unroll
                    for (int j = 0; j < 3; ++j) block_normals_raw<8, MULF>(6u * i + 3u * h + j, point, sweep, A.rk, z + 8 * j);
                }
                float yx[8], yz[8];
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    yx[a] = fmaf(sk, z[3 * a], yx0[a]);
                    yz[a] = fmaf(sk, z[3 * a + 1], yz0[a]);
                }
                const float ex = __shfl_sync(0xffffffffu, yx[6], src_e);
                const float ez = __shfl_sync(0xffffffffu, yz[6], src_e);
                float dd[8];
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    const float dx = yx[a] - ex, dz = yz[a] - ez;
                    dd[a] = fmaf(dx, dx, dz * dz);
                }
                float d2 = fminf(fminf(fminf(dd[0], dd[1]), fminf(dd[2], dd[3])), fminf(dd[4], dd[5]));
                const float d67 = fminf(dd[6], dd[7]);   // pursuers 6, 7 on h = 0; evader, padding on h = 1
                d2 = h ? d2 : fminf(d2, d67);
                d2 = fminf(d2, __shfl_xor_sync(0xffffffffu, d2, 1));
                float a2 = fmaf(cneg2, sqrt_approx(d2), cr);
                if (TILT) {
                    float part = 0.0f;
#pragma unroll
                    for (int j = 0; j < L; ++j) part = fmaf(z[j], tql[j], part);
                    part += __shfl_xor_sync(0xffffffffu, part, 1);
                    a2 += part;
                }
                if (live) {
                    lse_accumulate<L>(a2, z, m, s, q, S);
                    if constexpr (CV) {
#pragma unroll
                        for (int j = 0; j < L; ++j) Z1[j] += z[j];
                    }
                }
            }

            warp_merge<L>(2, m, s, q, S);
            if constexpr (CV) {
#pragma unroll
                for (int off = 16; off >= 2; off >>= 1) {
#pragma unroll
                    for (int j = 0; j < L; ++j) Z1[j] += __shfl_xor_sync(0xffffffffu, Z1[j], off);
                }
            }
            if (lane < 2) {
                if (lane == 0) { sh.red_m[warp] = m; sh.red_s[warp] = s; sh.red_q[warp] = q; }
#pragma unroll
                for (int j = 0; j < L; ++j) sh.red_S[warp][L * lane + j] = S[j];
                if constexpr (CV) {
#pragma unroll
                    for (int j = 0; j < L; ++j) {
                        sh.red_Z1[warp][L * lane + j] = Z1[j];
                        sh.red_Z2[warp][L * lane + j] = 0.0f;
                    }
                }
            }
            finish_sweep<G, NPAD, W, G::kCache, TILT, CV>(sh, A, pt, k, tid);
        }
    }
}

// ------------------------------------------------------------------------------------
// Initial iterate of Algorithm 1: v0 = l(x), p0 = Dl(x), c0 = Gamma(p0) (FP64 per state).
template <class G>
__global__ void init_kernel(const float* __restrict__ x, int64_t ldx, int64_t M, GameParams g,
                            double delta, double eta, double c_min, double c_max,
                            double* __restrict__ v, float* __restrict__ p, int64_t ldp,
                            float* __restrict__ c, float* __restrict__ ess,
                            const float* __restrict__ aux, int64_t ldaux) {
    constexpr int n = G::kN;
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double xd[n], gr[n];
    for (int j = 0; j < n; ++j) xd[j] = (double)x[m * ldx + j];
    const float* am = G::kAux > 0 ? aux + m * ldaux : nullptr;
    v[m] = G::ell_d(xd, g, am);
    G::grad_ell_d(xd, gr, g, am);
    double pp = 0.0;
    for (int j = 0; j < n; ++j) { p[m * ldp + j] = (float)gr[j]; pp += gr[j] * gr[j]; }
    int clipped;
    c[m] = (float)coef_update(G::ham_d(xd, gr, g, am), pp, delta, eta, c_min, c_max, g.tube, &clipped);
    ess[m] = 0.0f;
}

// Coefficient map Gamma at given (x, p) per state (FP64): used for warm starts, where Dv
// comes from outside the sweep (a surrogate) rather than from a sweep.
template <class G>
__global__ void coef_kernel(const float* __restrict__ x, int64_t ldx, int64_t M, const float* __restrict__ p,
                            int64_t ldp, GameParams g, double delta, double eta, double c_min, double c_max,
                            float* __restrict__ c, const float* __restrict__ aux, int64_t ldaux) {
    constexpr int n = G::kN;
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double xd[n], pd[n];
    double pp = 0.0;
    for (int j = 0; j < n; ++j) {
        xd[j] = (double)x[m * ldx + j];
        pd[j] = (double)p[m * ldp + j];
        pp += pd[j] * pd[j];
    }
    int clipped;
    c[m] = (float)coef_update(G::ham_d(xd, pd, g, G::kAux > 0 ? aux + m * ldaux : nullptr), pp, delta, eta,
                              c_min, c_max, g.tube, &clipped);
}

template <class G>
cudaError_t launch_coef(const float* x, int64_t ldx, int64_t M, const float* p, int64_t ldp,
                        const GameParams& g, double delta, double eta, double c_min, double c_max, float* c,
                        const float* aux, int64_t ldaux, cudaStream_t st) {
    const int T = 128;
    coef_kernel<G><<<(unsigned)((M + T - 1) / T), T, 0, st>>>(x, ldx, M, p, ldp, g, delta, eta, c_min, c_max,
                                                              c, aux, ldaux);
    return cudaGetLastError();
}

// The iterate relative to Algorithm 1's initial one, for a surrogate that learns the
// correction to it (FP64 per state).  warm = false: d[m] = (v - l(x), Dv - Dl(x)) of the
// current iterate; warm = true: the iterate becomes v = l(x) + d_v, Dv = Dl(x) + d_p with
// c = Gamma(Dv).  Row m of d holds the value part in column 0 and Dv in columns 1..n.
template <class G>
__global__ void delta_kernel(const float* __restrict__ x, int64_t ldx, int64_t M, GameParams g, double delta,
                             double eta, double c_min, double c_max, double* __restrict__ v,
                             float* __restrict__ p, int64_t ldp, float* __restrict__ c, float* __restrict__ d,
                             int64_t ldd, bool warm, const float* __restrict__ aux, int64_t ldaux) {
    constexpr int n = G::kN;
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double xd[n], gr[n];
    for (int j = 0; j < n; ++j) xd[j] = (double)x[m * ldx + j];
    const float* am = G::kAux > 0 ? aux + m * ldaux : nullptr;
    const double l = G::ell_d(xd, g, am);
    G::grad_ell_d(xd, gr, g, am);
    float* dm = d + m * ldd;
    if (!warm) {
        dm[0] = (float)(v[m] - l);
        for (int j = 0; j < n; ++j) dm[1 + j] = (float)((double)p[m * ldp + j] - gr[j]);
        return;
    }
    v[m] = l + (double)dm[0];
    double pp = 0.0;
    for (int j = 0; j < n; ++j) {
        const double pj = gr[j] + (double)dm[1 + j];
        p[m * ldp + j] = (float)pj;
        gr[j] = (double)(float)pj;   // Gamma of the stored FP32 Dv, as after any sweep
        pp += gr[j] * gr[j];
    }
    int clipped;
    c[m] = (float)coef_update(G::ham_d(xd, gr, g, am), pp, delta, eta, c_min, c_max, g.tube, &clipped);
}

template <class G>
cudaError_t launch_delta(const float* x, int64_t ldx, int64_t M, const GameParams& g, double delta, double eta,
                         double c_min, double c_max, double* v, float* p, int64_t ldp, float* c, float* d,
                         int64_t ldd, bool warm, const float* aux, int64_t ldaux, cudaStream_t st) {
    const int T = 128;
    delta_kernel<G><<<(unsigned)((M + T - 1) / T), T, 0, st>>>(x, ldx, M, g, delta, eta, c_min, c_max, v, p, ldp,
                                                               c, d, ldd, warm, aux, ldaux);
    return cudaGetLastError();
}

// Launch variants the autotuner chooses among: kind bit 0 = one warp per state (else one
// CTA per state), bit 1 = software-pipelined sampler, bit 2 = two sample groups per loop
// iteration, bits 3-4 = the Philox multiply form (philox4x32_10_rk); CTA size; minimum
// resident CTAs per SM (the register budget).  Every game's translation unit instantiates
// all of them.
#define HJG_SWEEP_VARIANTS(X) X(0, 4, 128, 8) X(1, 0, 128, 6) X(2, 2, 128, 6) X(3, 0, 128, 4) \
    X(4, 4, 128, 6) X(5, 1, 256, 3) X(6, 3, 256, 3) X(7, 5, 256, 3) X(8, 2, 256, 4)      \
    X(9, 2, 128, 8) X(10, 13, 256, 3) X(11, 10, 128, 8)
#define HJG_R45_VARIANTS(X) X(0, 0, 256, 1) X(1, 0, 256, 2) X(2, 0, 128, 3) X(3, 0, 128, 4) \
    X(4, 0, 512, 1) X(5, 2, 256, 1) X(6, 2, 128, 3) X(7, 2, 512, 1) X(8, 2, 256, 2)       \
    X(9, 4, 128, 3) X(10, 8, 128, 3) X(11, 6, 128, 3)
constexpr int kNumVariants = 12;
constexpr int kNumR45Variants = 12;   // below kCvVariant: the slots after the variants are taken

template <class G, int KIND, int THREADS, int MINB>
cudaError_t launch_sweep_generic(const SweepArgs& A, bool tilt, int grid, cudaStream_t st) {
    constexpr bool PIPE = (KIND & 2) != 0, U2 = (KIND & 4) != 0;
    constexpr int F = (KIND >> 3) & 3;
    if constexpr ((KIND & 1) != 0) {
        if (tilt) sweep_kernel_warp<G, THREADS, MINB, true, PIPE, U2, F><<<grid, THREADS, 0, st>>>(A);
        else sweep_kernel_warp<G, THREADS, MINB, false, PIPE, U2, F><<<grid, THREADS, 0, st>>>(A);
    } else {
        if (tilt) sweep_kernel<G, THREADS, MINB, true, PIPE, false, U2, F><<<grid, THREADS, 0, st>>>(A);
        else sweep_kernel<G, THREADS, MINB, false, PIPE, false, U2, F><<<grid, THREADS, 0, st>>>(A);
    }
    return cudaGetLastError();
}

// The control-variate kernel: one CTA per state, 256 threads, 4 CTAs per SM.  It is
// launched in the slot after the ordinary variants.
constexpr int kCvVariant = kNumVariants;
constexpr int kF64Variant = kNumVariants + 1;   // the FP64-throughout sweep (sweep_f64.cuh)
template <class G>
cudaError_t launch_sweep_cv(const SweepArgs& A, bool tilt, int grid, cudaStream_t st) {
    if (tilt) sweep_kernel<G, 256, 4, true, false, true><<<grid, 256, 0, st>>>(A);
    else sweep_kernel<G, 256, 4, false, false, true><<<grid, 256, 0, st>>>(A);
    return cudaGetLastError();
}
template <class G>
int occupancy_cv(bool tilt) {
    int nb = 0;
    if (tilt) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<G, 256, 4, true, false, true>, 256, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<G, 256, 4, false, false, true>, 256, 0);
    return nb;
}

template <class G, int KIND, int THREADS, int MINB>
int occupancy_generic(bool tilt) {
    int nb = 0;
    constexpr bool PIPE = (KIND & 2) != 0, U2 = (KIND & 4) != 0;
    constexpr int F = (KIND >> 3) & 3;
    if constexpr ((KIND & 1) != 0) {
        if (tilt) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel_warp<G, THREADS, MINB, true, PIPE, U2, F>, THREADS, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel_warp<G, THREADS, MINB, false, PIPE, U2, F>, THREADS, 0);
    } else {
        if (tilt) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<G, THREADS, MINB, true, PIPE, false, U2, F>, THREADS, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<G, THREADS, MINB, false, PIPE, false, U2, F>, THREADS, 0);
    }
    return nb;
}

template <class G>
cudaError_t launch_init(const float* x, int64_t ldx, int64_t M, const GameParams& g, double delta,
                        double eta, double c_min, double c_max, double* v, float* p, int64_t ldp,
                        float* c, float* ess, cudaStream_t st, const float* aux, int64_t ldaux) {
    const int T = 128;
    const int64_t blocks = (M + T - 1) / T;
    init_kernel<G><<<(unsigned)blocks, T, 0, st>>>(x, ldx, M, g, delta, eta, c_min, c_max, v, p,
                                                  ldp, c, ess, aux, ldaux);
    return cudaGetLastError();
}

}  // namespace hjg
