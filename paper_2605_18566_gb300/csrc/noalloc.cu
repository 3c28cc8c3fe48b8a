// noalloc.cu -- hjg_value_grad_noalloc: a one-shot solve (initial iterate, K Picard
// sweeps, residuals) that allocates no device memory at all.
//
// Some callers cannot call cudaMalloc once they are running: control loops with a hard
// real-time budget, processes whose device memory is owned by another runtime's caching
// allocator, and services that reserve every byte at start-up and must not fail later
// for want of memory.  This entry point serves them.  The caller passes its inputs and
// outputs as device pointers; the working memory the sweep needs besides them (frozen
// coefficients, ESS, the value history behind the residual, counters) lives in one
// file-scope device array of fixed size that every GPU loading the library keeps until
// the process exits.  Calls share that array, so two calls that overlap on the GPU (on
// different streams, or from different host threads) race on it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/hjg.h"
#include "dispatch.h"

using namespace hjg;

namespace {

constexpr size_t kScratchBytes = 16u << 20;   // 16 MiB per device
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (host code only sees a stand-in
// symbol); looked up once per device, on the first call made with that device current.
hjg_status scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HJG_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return HJG_ECUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return HJG_OK;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Relative L2 and sup-norm change per sweep from the value history (fixed reduction
// order, so repeated calls give identical residuals).
__global__ void residual_noalloc_kernel(const double* __restrict__ vhist, int64_t M, double* out) {
    constexpr int T = 256;
    __shared__ double s_num[T], s_den[T], s_sup[T];
    const int k = blockIdx.x, tid = threadIdx.x;
    const double* a = vhist + (int64_t)k * M;
    const double* b = a + M;
    double num = 0.0, den = 0.0, sup = 0.0;
    for (int64_t m = tid; m < M; m += T) {
        const double d = b[m] - a[m];
        num = fma(d, d, num);
        den = fma(a[m], a[m], den);
        sup = fmax(sup, fabs(d));
    }
    s_num[tid] = num; s_den[tid] = den; s_sup[tid] = sup;
    __syncthreads();
    for (int w = T / 2; w > 0; w >>= 1) {
        if (tid < w) {
            s_num[tid] += s_num[tid + w];
            s_den[tid] += s_den[tid + w];
            s_sup[tid] = fmax(s_sup[tid], s_sup[tid + w]);
        }
        __syncthreads();
    }
    if (tid == 0) {
        out[2 * k] = sqrt(s_num[0]) / sqrt(s_den[0]);
        out[2 * k + 1] = s_sup[0];
    }
}

bool pick_kernels(const hjg_dynamics* dyn, GameKernels* k) {
    switch (dyn->game) {
    case HJG_DUBINS3: *k = kernels_dubins3(); break;
    case HJG_ROCKETS6: *k = kernels_rockets6(); break;
    case HJG_ROCKETS45: *k = kernels_rockets45(); break;
    case HJG_ROCKETS_REL3: *k = kernels_rockets_rel3(); break;
    case HJG_DOUBLE_INT2: *k = kernels_double_int2(); break;
    case HJG_TEST_QUADRATIC:
    case HJG_TEST_ZERO_H:
        if (!kernels_quadratic(dyn->n, dyn->game == HJG_TEST_ZERO_H, k)) return false;
        break;
    default: return false;
    }
    return k->n == dyn->n;
}

GameParams game_params(const hjg_dynamics* dyn, const hjg_target* t, int tube) {
    GameParams g;
    memset(&g, 0, sizeof g);
    g.game = dyn->game;
    g.n = dyn->n;
    g.tube = tube != 0;
    g.radius = (float)t->radius;
    g.radius_d = t->radius;
    g.h_sign = (float)dyn->h_sign;
    g.h_sign_d = dyn->h_sign;
    for (int i = 0; i < 16; ++i) {
        const double s = dyn->speed[i] == 0.0 ? 1.0 : dyn->speed[i];
        g.speed[i] = (float)s;
        g.speed_d[i] = s;
    }
    for (int i = 0; i < 64; ++i) { g.A[i] = (float)t->A[i]; g.A_d[i] = t->A[i]; }
    for (int i = 0; i < 8; ++i) { g.x0[i] = (float)t->x0[i]; g.x0_d[i] = t->x0[i]; }
    g.d = (float)t->d;
    g.d_d = t->d;
    if (t->obstacle_radius > 0.0) {
        g.obstacle = 1;
        for (int i = 0; i < 2; ++i) {
            g.obs_c[i] = (float)t->obstacle_center[i];
            g.obs_c_d[i] = t->obstacle_center[i];
        }
        g.obs_r_d = t->obstacle_radius;
        g.obs_off = (float)(t->radius + t->obstacle_radius);
    }
    return g;
}

}  // namespace

extern "C" hjg_status hjg_value_grad_noalloc(const hjg_dynamics* dyn, const hjg_target* target,
                                             double nu, double T, const hjg_options* opt,
                                             const float* pts, int64_t M, int64_t ld, double* v_out,
                                             float* grad_out, int64_t ldg, double* residual_out,
                                             void* stream) {
    if (!dyn || !target || !opt) return HJG_EINVAL;
    if (!(nu > 0) || !(T > 0) || !std::isfinite(nu) || !std::isfinite(T)) return HJG_EINVAL;
    if (opt->N < 1 || opt->N > 0xFFFFFFFFll || opt->K < 1 || M < 0 || M > 0xFFFFFFFFll) return HJG_EINVAL;
    if ((uint64_t)opt->point_offset + (uint64_t)M > 0x100000000ull) return HJG_EINVAL;   // 32-bit counter word
    if (!stream_blocks_fit(dyn->n, opt->N)) return HJG_EINVAL;
    GameKernels kern{};
    if (!pick_kernels(dyn, &kern)) return HJG_EINVAL;
    if (!obstacle_ok(dyn, target)) return HJG_EUNSUPPORTED;
    // every option is checked before any device work
    const double delta = 2.0 * nu;
    const double sigma2 = delta * T;
    const double eta = opt->eta < 0 ? 1e-6 : opt->eta;
    const double c_min = opt->c_min > 0 ? opt->c_min : 1e-2 / delta;
    const double c_max = opt->c_max > 0 ? opt->c_max : 1e2 / delta;
    if (!(c_min <= c_max)) return HJG_EINVAL;
    const bool tilt = opt->tilt != 0;
    int variant = opt->variant > 0 ? opt->variant - 1 : 0;
    if (variant >= kern.nvariants) return HJG_EINVAL;
    if (opt->variant <= 0 && opt->block_threads > 0) {   // the first variant of that CTA size
        variant = -1;
        for (int i = 0; i < kern.nvariants && variant < 0; ++i)
            if (kern.threads[i] == opt->block_threads) variant = i;
        if (variant < 0) return HJG_EINVAL;
    }
    if (opt->precision < 0 || opt->precision > 1) return HJG_EINVAL;
    if (opt->cv) {
        if (!kern.has_cv || (kern.cv_tilt_only && !tilt) || opt->precision) return HJG_EUNSUPPORTED;
        variant = kCvVariant;
    } else if (opt->precision == 1) {
        if (!kern.has_f64) return HJG_EUNSUPPORTED;
        variant = kF64Variant;
    }
    const int n = dyn->n;
    if (ld < n || ldg < n) return HJG_EINVAL;
    if (M > 0 && (!pts || !v_out || !grad_out)) return HJG_EINVAL;
    const int K = opt->K;
    // scratch layout: c [M] f32 | ess [M] f32 | value history [(K+1) M] f64 | counters | resid [2K]
    const size_t off_ess = align256((size_t)M * sizeof(float));
    const size_t off_hist = off_ess + align256((size_t)M * sizeof(float));
    const size_t off_cnt = off_hist + align256((size_t)(K + 1) * (size_t)M * sizeof(double));
    const size_t off_res = off_cnt + 256;
    const size_t need = off_res + align256((size_t)2 * K * sizeof(double));
    if (need > kScratchBytes) return HJG_EINVAL;   // beyond the fixed scratch: (8K + 16) M bytes + slack
    if (M == 0) return HJG_OK;

    void* base = nullptr;
    hjg_status st = scratch_address(&base);
    if (st != HJG_OK) return st;
    unsigned char* b = (unsigned char*)base;
    float* c = (float*)b;
    float* ess = (float*)(b + off_ess);
    double* vhist = (double*)(b + off_hist);
    unsigned long long* cnt = (unsigned long long*)(b + off_cnt);
    double* resid = (double*)(b + off_res);

    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return HJG_ECUDA;
    const int occ = kern.occupancy(tilt, variant);
    if (occ <= 0) return HJG_ECUDA;
    int64_t grid = opt->grid_blocks > 0 ? opt->grid_blocks : (int64_t)occ * sms;
    if (grid > M) grid = M;
    cudaStream_t s = (cudaStream_t)stream;
    const GameParams g = game_params(dyn, target, opt->tube);

    if (cudaMemsetAsync(cnt, 0, 256, s) != cudaSuccess) return HJG_ECUDA;
    if (kern.init(pts, ld, M, g, delta, eta, c_min, c_max, v_out, grad_out, ldg, c, ess, s, nullptr, 0) !=
        cudaSuccess)
        return HJG_ECUDA;
    SweepArgs A;
    memset(&A, 0, sizeof A);
    A.x = pts; A.p = grad_out; A.c = c; A.v = v_out; A.vhist = vhist; A.ess = ess; A.counters = cnt;
    A.ldx = ld; A.ldp = ldg; A.M = M; A.N = opt->N;
    A.rk = philox_round_keys((uint32_t)opt->seed, (uint32_t)(opt->seed >> 32) ^ opt->instance);
    A.k0 = 0; A.pt0 = opt->point_offset; A.K = K;
    A.sigma_d = std::sqrt(sigma2);
    A.sigma = (float)A.sigma_d;
    A.sk = (float)(A.sigma_d * (double)kBmScale);
    A.sigma2_d = sigma2; A.delta = delta; A.eta = eta; A.c_min = c_min; A.c_max = c_max;
    A.g = g;
    if (kern.sweep(A, tilt, variant, (int)grid, s) != cudaSuccess) return HJG_ECUDA;
    residual_noalloc_kernel<<<K, 256, 0, s>>>(vhist, M, resid);
    if (cudaGetLastError() != cudaSuccess) return HJG_ECUDA;
    if (residual_out &&
        cudaMemcpyAsync(residual_out, resid, (size_t)2 * K * sizeof(double), cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess)
        return HJG_ECUDA;
    return HJG_OK;
}
