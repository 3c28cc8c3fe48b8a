// sweep_f64.cuh -- the Picard sweep in FP64 throughout (the "FP64 samples" precision of the
// 3-D workload, and a cross-check of the FP32 path): the same Philox stream and bit
// layout, but the normals (log, sqrt, sincospi), the samples, the target, the log-weights
// and every sum in double precision.  One CTA of 128 threads per state; the iterate is
// stored as on the FP32 path (v FP64; Dv and c FP32), so that one K-sweep launch equals K
// one-sweep launches.  Games with n <= 8.
#pragma once
#include "sweep_impl.cuh"

namespace hjg {

constexpr int kF64Threads = 128;

// The FP64 Box-Muller pair of one Philox word, with the uniforms of bm_normals_raw: radius
// uniform ((w & (2^20-1)) + 0.5) 2^-20, angle uniform ((w >> 20) + 0.5) 2^-12.
__device__ __forceinline__ void bm_pair_f64(uint32_t w, double* z) {
    const double ur = ((double)(w & 0xFFFFFu) + 0.5) * 0x1p-20;
    const double ua = ((double)(w >> 20) + 0.5) * 0x1p-12;
    const double rad = sqrt(-2.0 * log(ur));
    double s, c;
    sincospi(2.0 * ua, &s, &c);
    z[0] = rad * c;
    z[1] = rad * s;
}

__device__ __forceinline__ uint32_t block_word(const uint4& r, int j) {
    return j == 0 ? r.x : j == 1 ? r.y : j == 2 ? r.z : r.w;
}

template <class G, bool TILT>
__global__ void __launch_bounds__(kF64Threads) sweep_kernel_f64(const SweepArgs A) {
    constexpr int n = G::kN;
    static_assert(n <= 8, "the FP64 sweep keeps a state's sums in registers: n <= 8");
    constexpr int T = kF64Threads;
    constexpr int S = slot_stride(n);
    constexpr int KA = G::kAux > 0 ? G::kAux : 1;
    __shared__ double s_x[n], s_pd[n], s_th[n];
    __shared__ double s_m[T], s_s[T], s_q[T], s_S[T][n];
    __shared__ float s_aux[KA];
    __shared__ double s_c;
    const int tid = threadIdx.x;
    const uint32_t N32 = (uint32_t)A.N;

    for (int64_t pt = blockIdx.x; pt < A.M; pt += gridDim.x) {
        const Sig sig = item_sig(A, pt);
        const uint32_t point = A.pt0 + (uint32_t)pt;
        __syncthreads();   // the previous state's epilogue is done with the shared arrays
        if (tid < n) {
            s_x[tid] = (double)A.x[pt * A.ldx + tid];
            s_pd[tid] = (double)A.p[pt * A.ldp + tid];
        }
        if (G::kAux > 0 && tid < G::kAux) s_aux[tid] = A.aux[pt * A.ldaux + tid];
        if (tid == 0) {
            s_c = (double)A.c[pt];
            if (A.vhist) A.vhist[pt] = A.v[pt];
        }
        __syncthreads();
        for (int k = 0; k < A.K; ++k) {
            const bool last = (k + 1 == A.K);
            const uint32_t sweep = A.k0 + (uint32_t)k;
            const double c = s_c;
            double x[n], th[n], th2 = 0.0;
#pragma unroll
            for (int j = 0; j < n; ++j) {
                x[j] = s_x[j];
                th[j] = TILT ? -sig.sigma2_d * c * s_pd[j] : 0.0;   // Eq. tilt_shift
                th2 += th[j] * th[j];
            }
            double m = -INFINITY, s = 0.0, q = 0.0, Sz[n];
#pragma unroll
            for (int j = 0; j < n; ++j) Sz[j] = 0.0;
            for (uint32_t i = (uint32_t)tid; i < N32; i += T) {
                // only the pairs the sample reads: the FP64 transcendentals dominate this kernel
                double z[n], zp[2];
                const uint64_t q0 = (uint64_t)i * (uint64_t)S;
                uint64_t cur = ~0ull, curp = ~0ull;
                uint4 rb = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                for (int d = 0; d < n; ++d) {
                    const uint64_t qq = q0 + (uint64_t)d;
                    if (qq / kNormalsPerBlock != cur) {
                        cur = qq / kNormalsPerBlock;
                        rb = stream_block((uint32_t)cur, point, sweep, A.rk);
                    }
                    if (qq / 2 != curp) {
                        curp = qq / 2;
                        bm_pair_f64(block_word(rb, (int)((qq % kNormalsPerBlock) / 2)), zp);
                    }
                    z[d] = zp[qq % 2];
                }
                double y[n], dot = 0.0;
#pragma unroll
                for (int d = 0; d < n; ++d) {
                    const double dy = th[d] + sig.sigma_d * z[d];   // y - x
                    y[d] = x[d] + dy;
                    dot += dy * th[d];
                }
                // log-weight of Cor. B.4 / B.6: -c l(y) + (|theta|^2 - 2 <y - x, theta>) / (2 sigma^2)
                const double a = -c * G::ell_d(y, A.g, s_aux) + (th2 - 2.0 * dot) / (2.0 * sig.sigma2_d);
                if (a > m) {   // exact running maximum
                    const double f = (m == -INFINITY) ? 0.0 : exp(m - a);
                    s *= f;
                    q *= f * f;
#pragma unroll
                    for (int d = 0; d < n; ++d) Sz[d] *= f;
                    m = a;
                }
                const double w = exp(a - m);
                s += w;
                q = fma(w, w, q);
#pragma unroll
                for (int d = 0; d < n; ++d) Sz[d] = fma(w, z[d], Sz[d]);
            }
            s_m[tid] = m;
            s_s[tid] = s;
            s_q[tid] = q;
#pragma unroll
            for (int d = 0; d < n; ++d) s_S[tid][d] = Sz[d];
            __syncthreads();
            if (tid == 0) {
                double M = -INFINITY;
                for (int t = 0; t < T; ++t) M = fmax(M, s_m[t]);
                double st = 0.0, qt = 0.0, St[n];
                for (int d = 0; d < n; ++d) St[d] = 0.0;
                for (int t = 0; t < T; ++t) {
                    const double f = (s_m[t] == -INFINITY) ? 0.0 : exp(s_m[t] - M);
                    st = fma(f, s_s[t], st);
                    qt = fma(f * f, s_q[t], qt);
                    for (int d = 0; d < n; ++d) St[d] = fma(f, s_S[t][d], St[d]);
                }
                double v = -(M + log(st / (double)A.N)) / c;   // Cor. B.4
                double pd[n], pp = 0.0;
                bool finite = isfinite(v);
                for (int d = 0; d < n; ++d) {   // Cor. B.5 / B.6, centred form
                    pd[d] = -(th[d] + sig.sigma_d * St[d] / st) / (c * sig.sigma2_d);
                }
                if (G::kObstacle) obstacle_project(x, A.g, n, v, pd);   // reach-avoid: v >= o(x)
                for (int d = 0; d < n; ++d) {
                    pp += pd[d] * pd[d];
                    finite = finite && isfinite(pd[d]);
                }
                finite = finite && isfinite(v);
                int clipped = 0;
                const float c_new = (float)coef_update(G::ham_d(x, pd, A.g, s_aux), pp, A.delta, A.eta, A.c_min,
                                                       A.c_max, A.g.tube, &clipped);
                if (A.vhist) A.vhist[(int64_t)(k + 1) * A.M + pt] = v;
                A.v[pt] = v;
                s_c = (double)c_new;   // the next sweep starts from the stored (FP32) iterate
                for (int d = 0; d < n; ++d) s_pd[d] = (double)(float)pd[d];
                if (last) {
                    A.c[pt] = c_new;
                    A.ess[pt] = (float)(st * st / qt);
                    if (A.se) A.se[pt] = (float)(sqrt(fmax(0.0, qt / (st * st) - 1.0 / (double)A.N)) / fabs(c));
                    for (int d = 0; d < n; ++d) A.p[pt * A.ldp + d] = (float)pd[d];
                    if (!finite) atomicAdd(&A.counters[0], 1ull);
                    if (clipped) atomicAdd(&A.counters[1], 1ull);
                }
            }
            __syncthreads();
        }
    }
}

template <class G>
cudaError_t launch_sweep_f64(const SweepArgs& A, bool tilt, int grid, cudaStream_t st) {
    if (tilt) sweep_kernel_f64<G, true><<<grid, kF64Threads, 0, st>>>(A);
    else sweep_kernel_f64<G, false><<<grid, kF64Threads, 0, st>>>(A);
    return cudaGetLastError();
}
template <class G>
int occupancy_f64(bool tilt) {
    int nb = 0;
    if (tilt) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel_f64<G, true>, kF64Threads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel_f64<G, false>, kF64Threads, 0);
    return nb;
}

}  // namespace hjg
