// hjg_api.cu -- the C ABI of libhjg.so (declared in include/hjg.h): context management,
// argument checking, host<->device staging, and the launches of the sweep, init and
// residual kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/hjg.h"
#include "dispatch.h"
#include "frame45.cuh"

using namespace hjg;

struct hjg_ctx {
    hjg_dynamics dyn;
    hjg_target target;
    hjg_options opt;
    double nu = 0, T = 0, delta = 0, sigma2 = 0, eta = 0, c_min = 0, c_max = 0;
    int n = 0, ldx = 0;
    GameParams gp{};
    GameKernels kern{};
    int device = 0, num_sms = 0;
    cudaStream_t stream = nullptr;

    int64_t M = 0, cap = 0;
    float* d_x = nullptr;
    double* d_v = nullptr;
    float* d_p = nullptr;
    float* d_c = nullptr;
    float* d_ess = nullptr;
    float* d_se = nullptr;        // [M] Monte-Carlo standard error of v (last sweep)
    bool se_valid = false;        // a sweep has run since the iterate was last replaced
    int8_t* d_label = nullptr;    // [M] certificate labels
    float* d_band = nullptr;      // [M] certificate band half-widths
    unsigned long long* d_cert = nullptr;  // [3] label counts
    std::vector<double> horizons;  // several horizons t per solve (empty: the single T)
    Sig* d_tsig = nullptr;         // [horizons] kernel widths
    int64_t m_base = 0;            // states per horizon
    float* d_aux = nullptr;       // [M][22] flock: neighbour positions and their mean heading
    int32_t* d_idx = nullptr;     // [M][7] flock: neighbour indices
    unsigned long long* d_counters = nullptr;
    double* d_vhist = nullptr;
    int64_t vhist_rows = 0;   // allocated rows
    int last_sweeps = 0;      // rows used by the last call = last_sweeps + 1
    double* d_resid = nullptr;  // [K][2]
    double* d_parts = nullptr;  // [K][3] sums behind the residual
    int resid_cap = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // bracket the sweep kernel alone

    uint32_t next_sweep = 0;
    int64_t nonfinite = 0, clipped = 0;
    double last_ms = 0;
    int threads = 0, grid = 0;
    int variant = 0;          // launch variant of the sweep kernel (see hjg_autotune)
    std::string err;
};

namespace {

hjg_status fail(hjg_ctx* ctx, hjg_status st, const char* fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return st;
}

#define HJG_CUDA(ctx, call)                                                               \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail((ctx), e_ == cudaErrorMemoryAllocation ? HJG_ENOMEM : HJG_ECUDA,  \
                        "%s: %s", #call, cudaGetErrorString(e_));                         \
    } while (0)

cudaStream_t pick_stream(hjg_ctx* ctx, void* s) {
    return s ? (cudaStream_t)s : ctx->stream;
}

template <class T>
hjg_status grow(hjg_ctx* ctx, T** ptr, size_t count) {
    if (*ptr) cudaFree(*ptr);
    *ptr = nullptr;
    cudaError_t e = cudaMalloc((void**)ptr, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();   // reported here as ENOMEM: not left for a later launch check to find
        return fail(ctx, HJG_ENOMEM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T),
                    cudaGetErrorString(e));
    }
    return HJG_OK;
}

// Residual of Algorithm 1 from the value history: block k reduces rows k, k+1 over all
// states in a fixed order (deterministic) and writes (||v_{k+1}-v_k|| / ||v_k||, max |dv|).
__global__ void residual_kernel(const double* __restrict__ vhist, int64_t M, double* out, double* parts) {
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
        if (parts) {
            parts[3 * k] = s_num[0];
            parts[3 * k + 1] = s_den[0];
            parts[3 * k + 2] = s_sup[0];
        }
    }
}

__global__ void philox_blocks_kernel(const uint32_t* __restrict__ ctr, const uint32_t* __restrict__ key,
                                     uint32_t* __restrict__ out, int64_t count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const uint4 r = philox4x32_10(make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]),
                                  key[2 * i], key[2 * i + 1]);
    out[4 * i] = r.x; out[4 * i + 1] = r.y; out[4 * i + 2] = r.z; out[4 * i + 3] = r.w;
}

// The normals the sweep draws for samples 0..ns-1 of (point, sweep): sample i, dim d is
// slot i * slot_stride(n) + d of the stream, i.e. lane (slot % 8) of block slot / 8.
__global__ void normals_kernel(int n, uint32_t k0, uint32_t k1, uint32_t point, uint32_t sweep,
                               int64_t ns, float* __restrict__ out) {
    bm_table_fill();
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    const uint64_t q0 = (uint64_t)i * (uint64_t)slot_stride(n);
    uint64_t cached = ~0ull;
    float z[kNormalsPerBlock];
    for (int d = 0; d < n; ++d) {
        const uint64_t q = q0 + (uint64_t)d;
        if (q / kNormalsPerBlock != cached) {
            cached = q / kNormalsPerBlock;
            block_normals<kNormalsPerBlock>((uint32_t)cached, point, sweep, k0, k1, z);
        }
        out[i * n + d] = z[q % kNormalsPerBlock];
    }
}

void fill_game_params(hjg_ctx* ctx) {
    GameParams& g = ctx->gp;
    memset(&g, 0, sizeof g);
    g.game = ctx->dyn.game;
    g.n = ctx->n;
    g.tube = ctx->opt.tube != 0;
    g.radius = (float)ctx->target.radius;
    g.radius_d = ctx->target.radius;
    g.h_sign = (float)ctx->dyn.h_sign;
    g.h_sign_d = ctx->dyn.h_sign;
    for (int i = 0; i < 16; ++i) {
        const double s = ctx->dyn.speed[i] == 0.0 ? 1.0 : ctx->dyn.speed[i];
        g.speed[i] = (float)s;
        g.speed_d[i] = s;
    }
    for (int i = 0; i < 64; ++i) { g.A[i] = (float)ctx->target.A[i]; g.A_d[i] = ctx->target.A[i]; }
    for (int i = 0; i < 8; ++i) { g.x0[i] = (float)ctx->target.x0[i]; g.x0_d[i] = ctx->target.x0[i]; }
    g.d = (float)ctx->target.d;
    g.d_d = ctx->target.d;
    if (ctx->target.obstacle_radius > 0.0) {
        g.obstacle = 1;
        for (int i = 0; i < 2; ++i) {
            g.obs_c[i] = (float)ctx->target.obstacle_center[i];
            g.obs_c_d[i] = ctx->target.obstacle_center[i];
        }
        g.obs_r_d = ctx->target.obstacle_radius;
        g.obs_off = (float)(ctx->target.radius + ctx->target.obstacle_radius);
    }
}

hjg_status ensure_capacity(hjg_ctx* ctx, int64_t M) {
    if (M <= ctx->cap) return HJG_OK;
    // Drop the loaded states and the recorded sizes first: if an allocation below fails,
    // the context holds no states (every later call sees M = 0) and the next load grows
    // every buffer again, instead of trusting a capacity some buffers no longer have.
    ctx->M = 0;
    ctx->m_base = 0;
    ctx->last_sweeps = 0;
    ctx->se_valid = false;
    ctx->cap = 0;
    if (ctx->d_vhist) { cudaFree(ctx->d_vhist); ctx->d_vhist = nullptr; }
    ctx->vhist_rows = 0;
    hjg_status st;
    if ((st = grow(ctx, &ctx->d_x, (size_t)M * ctx->ldx))) return st;
    if ((st = grow(ctx, &ctx->d_v, (size_t)M))) return st;
    if ((st = grow(ctx, &ctx->d_p, (size_t)M * ctx->ldx))) return st;
    if ((st = grow(ctx, &ctx->d_c, (size_t)M))) return st;
    if ((st = grow(ctx, &ctx->d_ess, (size_t)M))) return st;
    if ((st = grow(ctx, &ctx->d_se, (size_t)M))) return st;
    if ((st = grow(ctx, &ctx->d_label, (size_t)M))) return st;
    if ((st = grow(ctx, &ctx->d_band, (size_t)M))) return st;
    if (ctx->dyn.game == HJG_FLOCK4) {
        if ((st = grow(ctx, &ctx->d_aux, (size_t)M * kFlockAux))) return st;
        if ((st = grow(ctx, &ctx->d_idx, (size_t)M * 7))) return st;
    }
    ctx->cap = M;
    return HJG_OK;
}

hjg_status ensure_history(hjg_ctx* ctx, int K) {
    hjg_status st;
    if (K + 1 > ctx->vhist_rows) {
        ctx->vhist_rows = 0;   // a failed growth leaves no rows to trust
        if ((st = grow(ctx, &ctx->d_vhist, (size_t)(K + 1) * ctx->cap))) return st;
        ctx->vhist_rows = K + 1;
    }
    if (K > ctx->resid_cap) {
        ctx->resid_cap = 0;
        if ((st = grow(ctx, &ctx->d_resid, (size_t)2 * K))) return st;
        if ((st = grow(ctx, &ctx->d_parts, (size_t)3 * K))) return st;
        ctx->resid_cap = K;
    }
    return HJG_OK;
}

// Copy states [M][ld] (host or device) into the context's padded [M][ldx] buffer.
hjg_status stage_points(hjg_ctx* ctx, const float* pts, int64_t M, int64_t ld, int on_device,
                        cudaStream_t st) {
    const size_t row = (size_t)ctx->n * sizeof(float);
    if (ld == ctx->ldx) {
        HJG_CUDA(ctx, cudaMemcpyAsync(ctx->d_x, pts, (size_t)M * ld * sizeof(float),
                                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    } else {
        HJG_CUDA(ctx, cudaMemcpy2DAsync(ctx->d_x, ctx->ldx * sizeof(float), pts, ld * sizeof(float), row,
                                        (size_t)M, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                        st));
    }
    return HJG_OK;
}

SweepArgs make_args(hjg_ctx* ctx, int K) {
    SweepArgs A;
    memset(&A, 0, sizeof A);
    A.x = ctx->d_x;
    A.p = ctx->d_p;
    A.c = ctx->d_c;
    A.v = ctx->d_v;
    A.vhist = ctx->d_vhist;
    A.ess = ctx->d_ess;
    A.se = ctx->d_se;
    A.counters = ctx->d_counters;
    A.ldx = ctx->ldx;
    A.ldp = ctx->ldx;
    A.M = ctx->M;
    A.N = ctx->opt.N;
    if (!ctx->horizons.empty()) {
        A.tsig = ctx->d_tsig;
        A.m_base = ctx->m_base;
    }
    A.rk = philox_round_keys((uint32_t)ctx->opt.seed,
                             (uint32_t)(ctx->opt.seed >> 32) ^ ctx->opt.instance);
    A.k0 = ctx->next_sweep;
    A.pt0 = ctx->opt.point_offset;
    A.K = K;
    A.sigma_d = std::sqrt(ctx->sigma2);
    A.sigma = (float)A.sigma_d;
    A.sk = (float)(A.sigma_d * (double)kBmScale);
    A.sigma2_d = ctx->sigma2;
    A.delta = ctx->delta;
    A.eta = ctx->eta;
    A.c_min = ctx->c_min;
    A.c_max = ctx->c_max;
    A.g = ctx->gp;
    A.aux = ctx->d_aux;
    A.ldaux = kFlockAux;
    return A;
}

hjg_status choose_launch(hjg_ctx* ctx) {
    const bool tilt = ctx->opt.tilt != 0;
    int v = ctx->variant;
    if (ctx->opt.cv) {   // the control variate has one kernel of its own
        if (!ctx->kern.has_cv) return fail(ctx, HJG_EUNSUPPORTED, "no control-variate kernel for this game");
        if (ctx->kern.cv_tilt_only && !tilt)
            return fail(ctx, HJG_EUNSUPPORTED, "this game's control variate runs with the tilt only");
        if (ctx->opt.precision != 0)
            return fail(ctx, HJG_EUNSUPPORTED, "the control variate runs on the FP32 path only");
        v = kCvVariant;
    } else if (ctx->opt.precision == 1) {   // FP64 throughout: one kernel of its own
        if (!ctx->kern.has_f64) return fail(ctx, HJG_EUNSUPPORTED, "no FP64 sweep for this game");
        v = kF64Variant;
    } else if (ctx->opt.variant > 0) {
        v = ctx->opt.variant - 1;
        if (v >= ctx->kern.nvariants) return fail(ctx, HJG_EINVAL, "variant %d out of range", v);
    } else if (ctx->opt.block_threads > 0) {
        v = -1;
        for (int i = 0; i < ctx->kern.nvariants && v < 0; ++i)
            if (ctx->kern.threads[i] == ctx->opt.block_threads) v = i;
        if (v < 0) return fail(ctx, HJG_EINVAL, "block_threads=%d is not available for this game",
                               ctx->opt.block_threads);
    }
    const int occ = ctx->kern.occupancy(tilt, v);
    if (occ <= 0) return fail(ctx, HJG_ECUDA, "sweep variant %d cannot launch", v);
    int64_t grid = ctx->opt.grid_blocks > 0 ? ctx->opt.grid_blocks : (int64_t)occ * ctx->num_sms;
    const int64_t per_cta = ctx->kern.per_warp[v] ? ctx->kern.threads[v] / 32 : 1;   // states per CTA pass
    grid = std::min<int64_t>(grid, std::max<int64_t>((ctx->M + per_cta - 1) / per_cta, 1));
    ctx->threads = ctx->kern.threads[v];
    ctx->grid = (int)grid;
    ctx->variant = v;
    return HJG_OK;
}

}  // namespace

namespace hjg {
// The reach-avoid obstacle is defined for the games whose state dims 0, 1 are a position.
bool obstacle_ok(const hjg_dynamics* dyn, const hjg_target* t) {
    if (!(t->obstacle_radius > 0.0)) return t->obstacle_radius == 0.0;   // NaN or negative: refused
    if (!std::isfinite(t->obstacle_radius) || !std::isfinite(t->obstacle_center[0]) ||
        !std::isfinite(t->obstacle_center[1]))
        return false;
    return dyn->game == HJG_DUBINS3 || dyn->game == HJG_ROCKETS_REL3 || dyn->game == HJG_DOUBLE_INT2;
}

}  // namespace hjg

// Conservative certificate of Cor. 2.9 per state: band E_m = e0 + q/(1-q) ||v^(K) - v^(K-1)||_inf
// + z se_m (the a-posteriori iteration bound of Theorem 2.8 from the last sweep's sup-norm
// change, and the Monte-Carlo term from the state's standard error); label +1 (SAFE) if
// v > E_m, -1 (UNSAFE) if v < -E_m, else 0 (UNDETERMINED); a state whose ESS is below
// ess_min is UNDETERMINED.
__global__ void certify_kernel(const double* __restrict__ v, const float* __restrict__ se,
                               const float* __restrict__ ess, int64_t M, double e0, double qf,
                               const double* __restrict__ sup_last, double z, double ess_min,
                               int8_t* __restrict__ label, float* __restrict__ band,
                               unsigned long long* __restrict__ counts) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const double b = e0 + (qf > 0.0 ? qf * sup_last[0] : 0.0) + z * (double)se[m];
    const double vm = v[m];
    int8_t l = vm > b ? 1 : (vm < -b ? -1 : 0);
    if ((double)ess[m] < ess_min) l = 0;   // collapsed weights: the error estimate is not trusted
    label[m] = l;
    band[m] = (float)b;
    atomicAdd(&counts[l + 1], 1ull);
}

extern "C" {

const char* hjg_status_string(hjg_status s) {
    switch (s) {
    case HJG_OK: return "ok";
    case HJG_EINVAL: return "invalid argument";
    case HJG_ENOMEM: return "out of memory";
    case HJG_ECUDA: return "CUDA error";
    case HJG_ENONFINITE: return "non-finite result";
    case HJG_ETIMEOUT: return "device wait timed out";
    case HJG_ENOTCONVERGED: return "not converged";
    case HJG_EUNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char* hjg_last_error(const hjg_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

hjg_status hjg_create(const hjg_dynamics* dyn, const hjg_target* target, double nu, double T,
                      const hjg_options* opt, hjg_ctx** out) {
    if (!out) return HJG_EINVAL;
    *out = nullptr;
    if (!dyn || !target || !opt) return HJG_EINVAL;
    if (!(nu > 0) || !(T > 0) || !std::isfinite(nu) || !std::isfinite(T)) return HJG_EINVAL;
    if (opt->N < 1 || opt->N > 0xFFFFFFFFll || opt->K < 0) return HJG_EINVAL;
    if (!stream_blocks_fit(dyn->n, opt->N)) return HJG_EINVAL;
    hjg_ctx* ctx = new (std::nothrow) hjg_ctx();
    if (!ctx) return HJG_ENOMEM;
    ctx->dyn = *dyn;
    ctx->target = *target;
    ctx->opt = *opt;
    ctx->nu = nu;
    ctx->T = T;
    ctx->delta = 2.0 * nu;
    ctx->sigma2 = ctx->delta * T;
    ctx->eta = opt->eta < 0 ? 1e-6 : opt->eta;
    ctx->c_min = opt->c_min > 0 ? opt->c_min : 1e-2 / ctx->delta;
    ctx->c_max = opt->c_max > 0 ? opt->c_max : 1e2 / ctx->delta;
    ctx->n = dyn->n;
    hjg_status st = HJG_OK;
    switch (dyn->game) {
    case HJG_DUBINS3: ctx->kern = kernels_dubins3(); break;
    case HJG_ROCKETS6: ctx->kern = kernels_rockets6(); break;
    case HJG_ROCKETS45: ctx->kern = kernels_rockets45(); break;
    case HJG_TEST_QUADRATIC:
    case HJG_TEST_ZERO_H:
        if (!kernels_quadratic(dyn->n, dyn->game == HJG_TEST_ZERO_H, &ctx->kern)) st = HJG_EUNSUPPORTED;
        break;
    case HJG_FLOCK4: ctx->kern = kernels_flock4(); break;
    case HJG_ROCKETS_REL3: ctx->kern = kernels_rockets_rel3(); break;
    case HJG_DOUBLE_INT2: ctx->kern = kernels_double_int2(); break;
    default: st = HJG_EINVAL;
    }
    if (st == HJG_OK && ctx->kern.n != dyn->n) st = HJG_EINVAL;
    if (st == HJG_OK && !obstacle_ok(dyn, target)) st = HJG_EUNSUPPORTED;
    if (st == HJG_OK && (opt->precision < 0 || opt->precision > 1)) st = HJG_EINVAL;
    if (st == HJG_OK && opt->precision == 1 && !ctx->kern.has_f64) st = HJG_EUNSUPPORTED;
    if (st == HJG_OK && !(ctx->c_min <= ctx->c_max)) st = HJG_EINVAL;
    if (st != HJG_OK) { delete ctx; return st; }
    ctx->ldx = (ctx->n + 3) / 4 * 4;
    fill_game_params(ctx);
    if (cudaGetDevice(&ctx->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess) {
        delete ctx;
        return HJG_ECUDA;
    }
    if (cudaMalloc((void**)&ctx->d_counters, 4 * sizeof(unsigned long long)) != cudaSuccess) {
        delete ctx;
        return HJG_ENOMEM;
    }
    if (cudaEventCreate(&ctx->ev0) != cudaSuccess || cudaEventCreate(&ctx->ev1) != cudaSuccess) {
        hjg_destroy(ctx);
        return HJG_ECUDA;
    }
    *out = ctx;
    return HJG_OK;
}

void hjg_destroy(hjg_ctx* ctx) {
    if (!ctx) return;
    cudaFree(ctx->d_x); cudaFree(ctx->d_v); cudaFree(ctx->d_p); cudaFree(ctx->d_c);
    cudaFree(ctx->d_ess); cudaFree(ctx->d_se); cudaFree(ctx->d_label); cudaFree(ctx->d_band);
    cudaFree(ctx->d_cert); cudaFree(ctx->d_tsig); cudaFree(ctx->d_counters); cudaFree(ctx->d_vhist); cudaFree(ctx->d_resid);
    cudaFree(ctx->d_aux); cudaFree(ctx->d_idx); cudaFree(ctx->d_parts);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    delete ctx;
}

hjg_status hjg_set_stream(hjg_ctx* ctx, void* stream) {
    if (!ctx) return HJG_EINVAL;
    ctx->stream = (cudaStream_t)stream;
    return HJG_OK;
}

hjg_status hjg_set_points(hjg_ctx* ctx, const float* pts, int64_t M, int64_t ld, int on_device,
                          void* stream) {
    if (!ctx) return HJG_EINVAL;
    if (ctx->dyn.game == HJG_FLOCK4 && M > 0 && M < 8)
        return fail(ctx, HJG_EINVAL, "a flock needs at least 8 agents (7 neighbours each)");
    const int64_t H = ctx->horizons.empty() ? 1 : (int64_t)ctx->horizons.size();
    if (M < 0 || M * H > 0xFFFFFFFFll || (M > 0 && !pts) || ld < ctx->n)
        return fail(ctx, HJG_EINVAL, "set_points: bad M=%lld or ld=%lld (n=%d)", (long long)M,
                    (long long)ld, ctx->n);
    if ((uint64_t)ctx->opt.point_offset + (uint64_t)(M * H) > 0x100000000ull)   // 32-bit counter word
        return fail(ctx, HJG_EINVAL, "set_points: point_offset + items exceeds 2^32");
    cudaStream_t st = pick_stream(ctx, stream);
    hjg_status s;
    const int64_t items = M * H;   // item j M + m: state m at horizon j
    if ((s = ensure_capacity(ctx, items))) return s;
    ctx->M = items;
    ctx->m_base = M;
    ctx->next_sweep = 0;
    ctx->last_sweeps = 0;
    ctx->se_valid = false;
    if (M == 0) return HJG_OK;
    if ((s = stage_points(ctx, pts, M, ld, on_device, st))) return s;
    if (ctx->ldx > ctx->n) {
        // zero the padding columns of x and p so every row is a clean float4 multiple
        HJG_CUDA(ctx, cudaMemset2DAsync(ctx->d_x + ctx->n, ctx->ldx * sizeof(float), 0,
                                        (ctx->ldx - ctx->n) * sizeof(float), (size_t)items, st));
        HJG_CUDA(ctx, cudaMemset2DAsync(ctx->d_p + ctx->n, ctx->ldx * sizeof(float), 0,
                                        (ctx->ldx - ctx->n) * sizeof(float), (size_t)items, st));
    }
    if (ctx->dyn.game == HJG_FLOCK4)   // neighbours among the loaded agents, frozen for the solve
        HJG_CUDA(ctx, flock_neighbours(ctx->d_x, ctx->ldx, M, ctx->d_idx, nullptr, ctx->d_aux, kFlockAux, st));
    for (int64_t h = 1; h < H; ++h) {   // the same states (and neighbour data) at every horizon
        HJG_CUDA(ctx, cudaMemcpyAsync(ctx->d_x + h * M * ctx->ldx, ctx->d_x, (size_t)M * ctx->ldx * sizeof(float),
                                      cudaMemcpyDeviceToDevice, st));
        if (ctx->dyn.game == HJG_FLOCK4)
            HJG_CUDA(ctx, cudaMemcpyAsync(ctx->d_aux + h * M * kFlockAux, ctx->d_aux,
                                          (size_t)M * kFlockAux * sizeof(float), cudaMemcpyDeviceToDevice, st));
    }
    HJG_CUDA(ctx, ctx->kern.init(ctx->d_x, ctx->ldx, items, ctx->gp, ctx->delta, ctx->eta, ctx->c_min,
                                 ctx->c_max, ctx->d_v, ctx->d_p, ctx->ldx, ctx->d_c, ctx->d_ess, st,
                                 ctx->d_aux, kFlockAux));
    return HJG_OK;
}

hjg_status hjg_set_horizons(hjg_ctx* ctx, const double* t, int n_horizons) {
    if (!ctx || n_horizons < 0 || (n_horizons > 0 && !t)) return HJG_EINVAL;
    for (int h = 0; h < n_horizons; ++h)
        if (!(t[h] > 0.0) || !std::isfinite(t[h])) return fail(ctx, HJG_EINVAL, "horizon %d is not > 0", h);
    ctx->M = 0;   // the loaded states are dropped: load them again for the new horizons
    ctx->m_base = 0;
    ctx->last_sweeps = 0;
    ctx->se_valid = false;
    ctx->horizons.assign(t, t + n_horizons);
    if (ctx->d_tsig) { cudaFree(ctx->d_tsig); ctx->d_tsig = nullptr; }
    if (n_horizons == 0) return HJG_OK;
    std::vector<Sig> tab((size_t)n_horizons);
    for (int h = 0; h < n_horizons; ++h) {
        tab[h].sigma2_d = ctx->delta * t[h];
        tab[h].sigma_d = std::sqrt(tab[h].sigma2_d);
        tab[h].sigma = (float)tab[h].sigma_d;
        tab[h].sk = (float)(tab[h].sigma_d * (double)kBmScale);
    }
    if (cudaMalloc((void**)&ctx->d_tsig, tab.size() * sizeof(Sig)) != cudaSuccess) {
        ctx->d_tsig = nullptr;
        ctx->horizons.clear();
        return fail(ctx, HJG_ENOMEM, "horizon table");
    }
    HJG_CUDA(ctx, cudaMemcpy(ctx->d_tsig, tab.data(), tab.size() * sizeof(Sig), cudaMemcpyHostToDevice));
    return HJG_OK;
}

hjg_status hjg_picard_sweep(hjg_ctx* ctx, int n_sweeps, double* residual_out, double* supnorm_out) {
    if (!ctx) return HJG_EINVAL;
    if (n_sweeps < 0) return fail(ctx, HJG_EINVAL, "n_sweeps < 0");
    if ((uint64_t)ctx->next_sweep + (uint64_t)n_sweeps > 0xFFFFFFFFull)
        return fail(ctx, HJG_EINVAL, "sweep counter would overflow");
    ctx->last_sweeps = 0;   // until this call's sweeps have been launched
    if (n_sweeps == 0 || ctx->M == 0) return HJG_OK;
    hjg_status s;
    if ((s = ensure_history(ctx, n_sweeps))) return s;
    if ((s = choose_launch(ctx))) return s;
    cudaStream_t st = ctx->stream;
    HJG_CUDA(ctx, cudaMemsetAsync(ctx->d_counters, 0, 4 * sizeof(unsigned long long), st));
    SweepArgs A = make_args(ctx, n_sweeps);
    HJG_CUDA(ctx, cudaEventRecord(ctx->ev0, st));
    HJG_CUDA(ctx, ctx->kern.sweep(A, ctx->opt.tilt != 0, ctx->variant, ctx->grid, st));
    HJG_CUDA(ctx, cudaEventRecord(ctx->ev1, st));
    residual_kernel<<<n_sweeps, 256, 0, st>>>(ctx->d_vhist, ctx->M, ctx->d_resid, ctx->d_parts);
    HJG_CUDA(ctx, cudaGetLastError());
    ctx->next_sweep += (uint32_t)n_sweeps;
    ctx->last_sweeps = n_sweeps;
    ctx->se_valid = true;
    if (residual_out || supnorm_out) {
        std::vector<double> r(2 * (size_t)n_sweeps);
        unsigned long long cnt[4];
        HJG_CUDA(ctx, cudaMemcpyAsync(r.data(), ctx->d_resid, r.size() * sizeof(double),
                                      cudaMemcpyDeviceToHost, st));
        HJG_CUDA(ctx, cudaMemcpyAsync(cnt, ctx->d_counters, sizeof cnt, cudaMemcpyDeviceToHost, st));
        HJG_CUDA(ctx, cudaStreamSynchronize(st));
        float ms = 0;
        cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
        ctx->last_ms = ms;
        for (int k = 0; k < n_sweeps; ++k) {
            if (residual_out) residual_out[k] = r[2 * k];
            if (supnorm_out) supnorm_out[k] = r[2 * k + 1];
        }
        ctx->nonfinite = (int64_t)cnt[0];
        ctx->clipped = (int64_t)cnt[1];
        if (cnt[0]) return fail(ctx, HJG_ENONFINITE, "%llu states gave a non-finite v or Dv", cnt[0]);
    }
    return HJG_OK;
}

hjg_status hjg_get_state(hjg_ctx* ctx, double* v, float* p, int64_t ldp, float* c, float* ess,
                         int on_device) {
    if (!ctx) return HJG_EINVAL;
    if (p && ldp < ctx->n) return fail(ctx, HJG_EINVAL, "ldp < n");
    cudaStream_t st = ctx->stream;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const int64_t M = ctx->M;
    if (M == 0) return HJG_OK;
    if (v) HJG_CUDA(ctx, cudaMemcpyAsync(v, ctx->d_v, M * sizeof(double), kind, st));
    if (c) HJG_CUDA(ctx, cudaMemcpyAsync(c, ctx->d_c, M * sizeof(float), kind, st));
    if (ess) HJG_CUDA(ctx, cudaMemcpyAsync(ess, ctx->d_ess, M * sizeof(float), kind, st));
    if (p) HJG_CUDA(ctx, cudaMemcpy2DAsync(p, ldp * sizeof(float), ctx->d_p, ctx->ldx * sizeof(float),
                                           ctx->n * sizeof(float), (size_t)M, kind, st));
    HJG_CUDA(ctx, cudaStreamSynchronize(st));
    return HJG_OK;
}

hjg_status hjg_set_state(hjg_ctx* ctx, const double* v, const float* p, int64_t ldp, const float* c,
                         uint32_t next_sweep, int on_device) {
    if (!ctx) return HJG_EINVAL;
    if (p && ldp < ctx->n) return fail(ctx, HJG_EINVAL, "ldp < n");
    cudaStream_t st = ctx->stream;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const int64_t M = ctx->M;
    if (M > 0) {
        if (v) HJG_CUDA(ctx, cudaMemcpyAsync(ctx->d_v, v, M * sizeof(double), kind, st));
        if (c) HJG_CUDA(ctx, cudaMemcpyAsync(ctx->d_c, c, M * sizeof(float), kind, st));
        if (p) HJG_CUDA(ctx, cudaMemcpy2DAsync(ctx->d_p, ctx->ldx * sizeof(float), p, ldp * sizeof(float),
                                               ctx->n * sizeof(float), (size_t)M, kind, st));
        HJG_CUDA(ctx, cudaStreamSynchronize(st));
    }
    ctx->next_sweep = next_sweep;
    ctx->se_valid = false;
    return HJG_OK;
}

hjg_status hjg_warm_start(hjg_ctx* ctx, const double* v0, const float* p0, int64_t ldp, int on_device) {
    if (!ctx || !p0) return HJG_EINVAL;
    if (ldp < ctx->n) return fail(ctx, HJG_EINVAL, "ldp < n");
    const int64_t M = ctx->M;
    if (M == 0) return HJG_OK;
    cudaStream_t st = ctx->stream;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    ctx->se_valid = false;
    if (v0) HJG_CUDA(ctx, cudaMemcpyAsync(ctx->d_v, v0, M * sizeof(double), kind, st));
    HJG_CUDA(ctx, cudaMemcpy2DAsync(ctx->d_p, ctx->ldx * sizeof(float), p0, ldp * sizeof(float),
                                    ctx->n * sizeof(float), (size_t)M, kind, st));
    HJG_CUDA(ctx, ctx->kern.coef(ctx->d_x, ctx->ldx, M, ctx->d_p, ctx->ldx, ctx->gp, ctx->delta, ctx->eta,
                                 ctx->c_min, ctx->c_max, ctx->d_c, ctx->d_aux, kFlockAux, st));
    HJG_CUDA(ctx, cudaStreamSynchronize(st));
    return HJG_OK;
}

hjg_status hjg_warm_start_delta(hjg_ctx* ctx, const float* d, int64_t ldd) {
    if (!ctx || !d) return HJG_EINVAL;
    if (ldd < ctx->n + 1) return fail(ctx, HJG_EINVAL, "ldd < n + 1");
    const int64_t M = ctx->M;
    if (M == 0) return HJG_OK;
    cudaStream_t st = ctx->stream;
    ctx->se_valid = false;
    HJG_CUDA(ctx, ctx->kern.delta(ctx->d_x, ctx->ldx, M, ctx->gp, ctx->delta, ctx->eta, ctx->c_min, ctx->c_max,
                                  ctx->d_v, ctx->d_p, ctx->ldx, ctx->d_c, const_cast<float*>(d), ldd, true,
                                  ctx->d_aux, kFlockAux, st));
    HJG_CUDA(ctx, cudaStreamSynchronize(st));
    return HJG_OK;
}

hjg_status hjg_get_state_delta(hjg_ctx* ctx, float* out, int64_t ldo) {
    if (!ctx || !out) return HJG_EINVAL;
    if (ldo < ctx->n + 1) return fail(ctx, HJG_EINVAL, "ldo < n + 1");
    const int64_t M = ctx->M;
    if (M == 0) return HJG_OK;
    cudaStream_t st = ctx->stream;
    HJG_CUDA(ctx, ctx->kern.delta(ctx->d_x, ctx->ldx, M, ctx->gp, ctx->delta, ctx->eta, ctx->c_min, ctx->c_max,
                                  ctx->d_v, ctx->d_p, ctx->ldx, ctx->d_c, out, ldo, false, ctx->d_aux, kFlockAux,
                                  st));
    HJG_CUDA(ctx, cudaStreamSynchronize(st));
    return HJG_OK;
}

namespace {
// The invariant frame needs the 45-D game with one speed shared by the pursuers.
hjg_status frame45_ok(hjg_ctx* ctx) {
    if (ctx->dyn.game != HJG_ROCKETS45)
        return fail(ctx, HJG_EUNSUPPORTED, "the invariant surrogate frame is defined for the 45-D game only");
    for (int i = 1; i < kF45P; ++i)
        if (ctx->gp.speed_d[i] != ctx->gp.speed_d[0])
            return fail(ctx, HJG_EUNSUPPORTED, "the invariant surrogate frame needs equal pursuer speeds");
    if (!ctx->horizons.empty()) return fail(ctx, HJG_EUNSUPPORTED, "the invariant frame takes one horizon");
    return HJG_OK;
}
}  // namespace

hjg_status hjg_frame_features(hjg_ctx* ctx, float* out, int64_t ldo) {
    if (!ctx || !out) return HJG_EINVAL;
    hjg_status s;
    if ((s = frame45_ok(ctx))) return s;
    if (ldo < kF45In) return fail(ctx, HJG_EINVAL, "ldo < 56");
    const int64_t M = ctx->M;
    if (M == 0) return HJG_OK;
    const int T = 128;
    frame45_out_kernel<<<(unsigned)((M + T - 1) / T), T, 0, ctx->stream>>>(ctx->d_x, ctx->ldx, M, ctx->gp, ctx->d_v,
                                                                          ctx->d_p, ctx->ldx, out, ldo, 0);
    HJG_CUDA(ctx, cudaGetLastError());
    HJG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return HJG_OK;
}

hjg_status hjg_frame_targets(hjg_ctx* ctx, float* out, int64_t ldo) {
    if (!ctx || !out) return HJG_EINVAL;
    hjg_status s;
    if ((s = frame45_ok(ctx))) return s;
    if (ldo < kF45Out) return fail(ctx, HJG_EINVAL, "ldo < 43");
    const int64_t M = ctx->M;
    if (M == 0) return HJG_OK;
    const int T = 128;
    frame45_out_kernel<<<(unsigned)((M + T - 1) / T), T, 0, ctx->stream>>>(ctx->d_x, ctx->ldx, M, ctx->gp, ctx->d_v,
                                                                          ctx->d_p, ctx->ldx, out, ldo, 1);
    HJG_CUDA(ctx, cudaGetLastError());
    HJG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return HJG_OK;
}

hjg_status hjg_warm_start_frame(hjg_ctx* ctx, const float* pred, int64_t ldp, int positions_only) {
    if (!ctx || !pred) return HJG_EINVAL;
    hjg_status s;
    if ((s = frame45_ok(ctx))) return s;
    if (ldp < kF45Out) return fail(ctx, HJG_EINVAL, "ldp < 43");
    const int64_t M = ctx->M;
    if (M == 0) return HJG_OK;
    ctx->se_valid = false;
    const int T = 128;
    frame45_warm_kernel<<<(unsigned)((M + T - 1) / T), T, 0, ctx->stream>>>(
        ctx->d_x, ctx->ldx, M, ctx->gp, ctx->delta, ctx->eta, ctx->c_min, ctx->c_max, pred, ldp, positions_only != 0,
        ctx->d_v, ctx->d_p, ctx->ldx, ctx->d_c);
    HJG_CUDA(ctx, cudaGetLastError());
    HJG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return HJG_OK;
}

hjg_status hjg_get_residual_parts(hjg_ctx* ctx, double* out) {
    if (!ctx || !out) return HJG_EINVAL;
    if (ctx->last_sweeps == 0 || ctx->M == 0) return HJG_OK;
    HJG_CUDA(ctx, cudaMemcpyAsync(out, ctx->d_parts, (size_t)3 * ctx->last_sweeps * sizeof(double),
                                  cudaMemcpyDeviceToHost, ctx->stream));
    HJG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return HJG_OK;
}

hjg_status hjg_certify(hjg_ctx* ctx, double e0, double q, double delta_p, double ess_min, int8_t* label_out,
                       float* band_out, float* se_out, int64_t* counts_out, int on_device) {
    if (!ctx) return HJG_EINVAL;
    if (!(e0 >= 0.0) || !(q >= 0.0 && q < 1.0) || !(delta_p > 0.0 && delta_p < 1.0) || !(ess_min >= 0.0))
        return fail(ctx, HJG_EINVAL, "certify: need e0 >= 0, 0 <= q < 1, 0 < delta_p < 1, ess_min >= 0");
    const int64_t M = ctx->M;
    if (M == 0) {
        if (counts_out) counts_out[0] = counts_out[1] = counts_out[2] = 0;
        return HJG_OK;
    }
    if (!ctx->se_valid || ctx->last_sweeps == 0)
        return fail(ctx, HJG_EINVAL, "certify: run at least one sweep on the current iterate first");
    cudaStream_t st = ctx->stream;
    if (!ctx->d_cert && cudaMalloc((void**)&ctx->d_cert, 3 * sizeof(unsigned long long)) != cudaSuccess)
        return fail(ctx, HJG_ENOMEM, "certify: counters");
    HJG_CUDA(ctx, cudaMemsetAsync(ctx->d_cert, 0, 3 * sizeof(unsigned long long), st));
    const double z = std::sqrt(2.0 * std::log(2.0 / delta_p));
    const double qf = q / (1.0 - q);
    const double* sup_last = ctx->d_resid + 2 * (ctx->last_sweeps - 1) + 1;
    certify_kernel<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(ctx->d_v, ctx->d_se, ctx->d_ess, M, e0, qf,
                                                                 sup_last, z, ess_min, ctx->d_label, ctx->d_band,
                                                                 ctx->d_cert);
    HJG_CUDA(ctx, cudaGetLastError());
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (label_out) HJG_CUDA(ctx, cudaMemcpyAsync(label_out, ctx->d_label, M * sizeof(int8_t), kind, st));
    if (band_out) HJG_CUDA(ctx, cudaMemcpyAsync(band_out, ctx->d_band, M * sizeof(float), kind, st));
    if (se_out) HJG_CUDA(ctx, cudaMemcpyAsync(se_out, ctx->d_se, M * sizeof(float), kind, st));
    unsigned long long cnt[3] = {0, 0, 0};
    HJG_CUDA(ctx, cudaMemcpyAsync(cnt, ctx->d_cert, sizeof cnt, cudaMemcpyDeviceToHost, st));
    HJG_CUDA(ctx, cudaStreamSynchronize(st));
    if (counts_out) {   // SAFE, UNSAFE, UNDETERMINED
        counts_out[0] = (int64_t)cnt[2];
        counts_out[1] = (int64_t)cnt[0];
        counts_out[2] = (int64_t)cnt[1];
    }
    return HJG_OK;
}

hjg_status hjg_get_history(hjg_ctx* ctx, double* out, int on_device) {
    if (!ctx || !out) return HJG_EINVAL;
    if (ctx->last_sweeps == 0 || ctx->M == 0) return HJG_OK;
    cudaStream_t st = ctx->stream;
    HJG_CUDA(ctx, cudaMemcpyAsync(out, ctx->d_vhist, (size_t)(ctx->last_sweeps + 1) * ctx->M * sizeof(double),
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    HJG_CUDA(ctx, cudaStreamSynchronize(st));
    return HJG_OK;
}

hjg_status hjg_value_grad(hjg_ctx* ctx, const float* pts, int64_t M, int64_t ld, int on_device,
                          double* v_out, float* grad_out, int64_t ldg, double* residual_out,
                          void* stream) {
    if (!ctx) return HJG_EINVAL;
    if (grad_out && ldg < ctx->n) return fail(ctx, HJG_EINVAL, "ldg < n");
    cudaStream_t saved = ctx->stream;
    if (stream) ctx->stream = (cudaStream_t)stream;
    hjg_status s = hjg_set_points(ctx, pts, M, ld, on_device, nullptr);
    const int K = ctx->opt.K;
    std::vector<double> r(std::max(K, 1), NAN);
    hjg_status sweep_status = HJG_OK;
    if (s == HJG_OK && K > 0) {
        if (ctx->opt.eps > 0) {
            // Algorithm 1's stopping rule: stop after the sweep whose relative change < eps
            for (int k = 0; k < K; ++k) {
                s = hjg_picard_sweep(ctx, 1, &r[k], nullptr);
                if (s != HJG_OK && s != HJG_ENONFINITE) break;
                if (s == HJG_ENONFINITE) sweep_status = s;
                if (r[k] < ctx->opt.eps) break;
            }
        } else {
            s = hjg_picard_sweep(ctx, K, r.data(), nullptr);
            if (s == HJG_ENONFINITE) { sweep_status = s; s = HJG_OK; }
        }
        if (s == HJG_ENONFINITE) s = HJG_OK;
    }
    if (s == HJG_OK) s = hjg_get_state(ctx, v_out, grad_out, ldg, nullptr, nullptr, on_device);
    if (s == HJG_OK && residual_out)
        for (int k = 0; k < K; ++k) residual_out[k] = r[k];
    ctx->stream = saved;
    return s != HJG_OK ? s : sweep_status;
}

hjg_status hjg_get_diagnostics(hjg_ctx* ctx, hjg_diag* out) {
    if (!ctx || !out) return HJG_EINVAL;
    memset(out, 0, sizeof *out);
    out->M = ctx->M;
    out->next_sweep = ctx->next_sweep;
    out->nonfinite = ctx->nonfinite;
    out->clipped = ctx->clipped;
    out->last_ms = ctx->last_ms;
    out->block_threads = ctx->threads;
    out->grid_blocks = ctx->grid;
    out->variant = ctx->variant;
    if (ctx->M > 0) {
        std::vector<float> e((size_t)ctx->M);
        HJG_CUDA(ctx, cudaMemcpyAsync(e.data(), ctx->d_ess, e.size() * sizeof(float), cudaMemcpyDeviceToHost,
                                      ctx->stream));
        HJG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        std::vector<float> sorted = e;
        std::nth_element(sorted.begin(), sorted.begin() + sorted.size() / 2, sorted.end());
        out->ess_median = sorted[sorted.size() / 2];
        out->ess_min = *std::min_element(e.begin(), e.end());
    }
    return HJG_OK;
}

hjg_status hjg_autotune(hjg_ctx* ctx, int64_t max_states, int32_t* variant_out, int32_t* threads_out,
                        double* best_ms_out) {
    if (!ctx) return HJG_EINVAL;
    if (ctx->M == 0) return fail(ctx, HJG_EINVAL, "autotune needs loaded states");
    if (ctx->opt.cv || ctx->opt.precision) {   // these run one kernel of their own: nothing to tune
        const int fixed = ctx->opt.cv ? kCvVariant : kF64Variant;
        if (variant_out) *variant_out = fixed;
        if (threads_out) *threads_out = ctx->kern.threads[fixed];
        if (best_ms_out) *best_ms_out = 0.0;
        return HJG_OK;
    }
    const bool tilt = ctx->opt.tilt != 0;
    const int64_t Mt = std::min<int64_t>(ctx->M, max_states > 0 ? max_states : ctx->M);
    cudaStream_t st = ctx->stream;
    float *p = nullptr, *c = nullptr, *ess = nullptr;
    double* v = nullptr;
    unsigned long long* cnt = nullptr;
    hjg_status s = HJG_OK;
    if ((s = grow(ctx, &p, (size_t)Mt * ctx->ldx)) || (s = grow(ctx, &c, (size_t)Mt)) ||
        (s = grow(ctx, &ess, (size_t)Mt)) || (s = grow(ctx, &v, (size_t)Mt)) ||
        (s = grow(ctx, &cnt, (size_t)4))) {
        cudaFree(p); cudaFree(c); cudaFree(ess); cudaFree(v); cudaFree(cnt);
        return s;
    }
    int best = -1;
    float best_ms = 0.0f;
    for (int var = 0; var < ctx->kern.nvariants && s == HJG_OK; ++var) {
        const int occ = ctx->kern.occupancy(tilt, var);
        if (occ <= 0) continue;
        const int64_t per_cta = ctx->kern.per_warp[var] ? ctx->kern.threads[var] / 32 : 1;
        const int grid = (int)std::min<int64_t>((int64_t)occ * ctx->num_sms, (Mt + per_cta - 1) / per_cta);
        SweepArgs A = make_args(ctx, 1);
        A.M = Mt; A.p = p; A.c = c; A.v = v; A.ess = ess; A.se = nullptr; A.vhist = nullptr; A.counters = cnt;
        float ms = 0.0f, best_rep = 0.0f;
        for (int rep = 0; rep < 3 && s == HJG_OK; ++rep) {   // warm-up, then the faster of two timed runs
            cudaError_t e = cudaMemcpyAsync(p, ctx->d_p, (size_t)Mt * ctx->ldx * sizeof(float),
                                            cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(c, ctx->d_c, (size_t)Mt * sizeof(float),
                                                      cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) e = cudaEventRecord(ctx->ev0, st);
            if (e == cudaSuccess) e = ctx->kern.sweep(A, tilt, var, grid, st);
            if (e == cudaSuccess) e = cudaEventRecord(ctx->ev1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(ctx->ev1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
            if (e != cudaSuccess) s = fail(ctx, HJG_ECUDA, "autotune variant %d: %s", var, cudaGetErrorString(e));
            if (rep == 1 || (rep > 1 && ms < best_rep)) best_rep = ms;
        }
        ms = best_rep;
        if (s == HJG_OK && (best < 0 || ms < best_ms)) { best = var; best_ms = ms; }
    }
    cudaFree(p); cudaFree(c); cudaFree(ess); cudaFree(v); cudaFree(cnt);
    if (s != HJG_OK) return s;
    if (best < 0) return fail(ctx, HJG_ECUDA, "no sweep variant can launch");
    ctx->variant = best;
    ctx->opt.block_threads = 0;
    ctx->opt.variant = 0;
    if (variant_out) *variant_out = best;
    if (threads_out) *threads_out = ctx->kern.threads[best];
    if (best_ms_out) *best_ms_out = best_ms;
    return HJG_OK;
}

hjg_status hjg_philox_blocks(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t count,
                             void* stream) {
    if (count < 0 || (count > 0 && (!ctr || !key || !out))) return HJG_EINVAL;
    if (count == 0) return HJG_OK;
    const int T = 256;
    philox_blocks_kernel<<<(unsigned)((count + T - 1) / T), T, 0, (cudaStream_t)stream>>>(ctr, key, out, count);
    return cudaGetLastError() == cudaSuccess ? HJG_OK : HJG_ECUDA;
}

hjg_status hjg_sample_normals(int n, uint64_t seed, uint32_t instance, uint32_t point, uint32_t sweep,
                              int64_t n_samples, float* out, void* stream) {
    if (n < 1 || n > 64 || n_samples < 0 || n_samples > 0x3FFFFFFll || (n_samples > 0 && !out))
        return HJG_EINVAL;
    if (n_samples == 0) return HJG_OK;
    const int T = 256;
    normals_kernel<<<(unsigned)((n_samples + T - 1) / T), T, 0, (cudaStream_t)stream>>>(
        n, (uint32_t)seed, (uint32_t)(seed >> 32) ^ instance, point, sweep, n_samples, out);
    return cudaGetLastError() == cudaSuccess ? HJG_OK : HJG_ECUDA;
}


// ---------------------------------------------------------------------------------------
// Batches: several game instances (contexts) advanced together by one CUDA-graph launch.
// Each instance's sweep and residual kernels sit on their own branch of the graph, so
// instances of different games and sizes run concurrently on the SMs.

struct hjg_batch {
    std::vector<hjg_ctx*> ctxs;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr, t0 = nullptr, t1 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double last_ms = 0;
    std::string err;
};

hjg_status hjg_batch_create(hjg_batch** out) {
    if (!out) return HJG_EINVAL;
    hjg_batch* b = new (std::nothrow) hjg_batch();
    if (!b) return HJG_ENOMEM;
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&b->t0) != cudaSuccess || cudaEventCreate(&b->t1) != cudaSuccess) {
        hjg_batch_destroy(b);   // releases whichever events were created
        return HJG_ECUDA;
    }
    *out = b;
    return HJG_OK;
}

hjg_status hjg_batch_add(hjg_batch* b, hjg_ctx* ctx) {
    if (!b || !ctx) return HJG_EINVAL;
    for (hjg_ctx* c : b->ctxs)
        if (c == ctx) return HJG_EINVAL;
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return HJG_ECUDA;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
        cudaStreamDestroy(s);
        return HJG_ECUDA;
    }
    b->ctxs.push_back(ctx);
    b->side.push_back(s);
    b->join.push_back(e);
    return HJG_OK;
}

void hjg_batch_destroy(hjg_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (cudaStream_t s : b->side) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->join) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->t0) cudaEventDestroy(b->t0);
    if (b->t1) cudaEventDestroy(b->t1);
    delete b;
}

const char* hjg_batch_last_error(const hjg_batch* b) { return b ? b->err.c_str() : "null batch"; }

hjg_status hjg_batch_run(hjg_batch* b, int n_sweeps, double* residual_out, void* stream, double* device_ms) {
    if (!b) return HJG_EINVAL;
    if (n_sweeps < 1) return HJG_EINVAL;
    const size_t I = b->ctxs.size();
    for (hjg_ctx* c : b->ctxs) {
        if (c->M == 0) { b->err = "a batch instance has no states loaded"; return HJG_EINVAL; }
        if ((uint64_t)c->next_sweep + (uint64_t)n_sweeps > 0xFFFFFFFFull) return HJG_EINVAL;
        hjg_status s;
        c->last_sweeps = 0;   // until this call's sweeps have been launched
        if ((s = ensure_history(c, n_sweeps)) || (s = choose_launch(c))) {
            b->err = c->err;
            return s;
        }
    }
    cudaStream_t origin = (cudaStream_t)stream;
    bool own_origin = false;
    if (!origin) {   // capture needs a stream other than the legacy default stream
        if (cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking) != cudaSuccess) return HJG_ECUDA;
        own_origin = true;
    }
    auto bail = [&](const char* what, cudaError_t e) {
        cudaGraph_t g = nullptr;
        cudaStreamCaptureStatus cs;
        if (cudaStreamIsCapturing(origin, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
            cudaStreamEndCapture(origin, &g);
        if (g) cudaGraphDestroy(g);
        if (own_origin) cudaStreamDestroy(origin);
        b->err = std::string(what) + ": " + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? HJG_ENOMEM : HJG_ECUDA;
    };
    cudaError_t e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bail("begin capture", e);
    if ((e = cudaEventRecord(b->fork, origin)) != cudaSuccess) return bail("fork", e);
    for (size_t i = 0; i < I; ++i) {
        hjg_ctx* c = b->ctxs[i];
        cudaStream_t s = b->side[i];
        if ((e = cudaStreamWaitEvent(s, b->fork, 0)) != cudaSuccess) return bail("wait fork", e);
        if ((e = cudaMemsetAsync(c->d_counters, 0, 4 * sizeof(unsigned long long), s)) != cudaSuccess)
            return bail("counters", e);
        SweepArgs A = make_args(c, n_sweeps);
        if ((e = c->kern.sweep(A, c->opt.tilt != 0, c->variant, c->grid, s)) != cudaSuccess)
            return bail("sweep", e);
        residual_kernel<<<n_sweeps, 256, 0, s>>>(c->d_vhist, c->M, c->d_resid, c->d_parts);
        if ((e = cudaGetLastError()) != cudaSuccess) return bail("residual", e);
        if ((e = cudaEventRecord(b->join[i], s)) != cudaSuccess) return bail("join", e);
        if ((e = cudaStreamWaitEvent(origin, b->join[i], 0)) != cudaSuccess) return bail("wait join", e);
    }
    cudaGraph_t g = nullptr;
    if ((e = cudaStreamEndCapture(origin, &g)) != cudaSuccess) return bail("end capture", e);
    bool updated = false;
    if (b->exec) {
        cudaGraphExecUpdateResultInfo info;
        updated = cudaGraphExecUpdate(b->exec, g, &info) == cudaSuccess;
        if (!updated) {
            cudaGetLastError();
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
    }
    if (!updated && (e = cudaGraphInstantiate(&b->exec, g, 0)) != cudaSuccess) {
        cudaGraphDestroy(g);
        return bail("instantiate", e);
    }
    if (b->graph) cudaGraphDestroy(b->graph);
    b->graph = g;
    if ((e = cudaEventRecord(b->t0, origin)) != cudaSuccess) return bail("timing", e);
    if ((e = cudaGraphLaunch(b->exec, origin)) != cudaSuccess) return bail("graph launch", e);
    if ((e = cudaEventRecord(b->t1, origin)) != cudaSuccess) return bail("timing", e);
    for (hjg_ctx* c : b->ctxs) {
        c->next_sweep += (uint32_t)n_sweeps;
        c->last_sweeps = n_sweeps;
        c->se_valid = true;
    }
    hjg_status result = HJG_OK;
    if (residual_out || device_ms || own_origin) {
        if ((e = cudaStreamSynchronize(origin)) != cudaSuccess) return bail("synchronize", e);
        float ms = 0;
        cudaEventElapsedTime(&ms, b->t0, b->t1);
        b->last_ms = ms;
        if (device_ms) *device_ms = ms;
        for (size_t i = 0; i < I && residual_out; ++i) {
            hjg_ctx* c = b->ctxs[i];
            std::vector<double> r(2 * (size_t)n_sweeps);
            unsigned long long cnt[4];
            if ((e = cudaMemcpy(r.data(), c->d_resid, r.size() * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess ||
                (e = cudaMemcpy(cnt, c->d_counters, sizeof cnt, cudaMemcpyDeviceToHost)) != cudaSuccess)
                return bail("copy residuals", e);
            for (int k = 0; k < n_sweeps; ++k) residual_out[i * n_sweeps + k] = r[2 * k];
            c->nonfinite = (int64_t)cnt[0];
            c->clipped = (int64_t)cnt[1];
            if (cnt[0]) result = HJG_ENONFINITE;
        }
    }
    if (own_origin) cudaStreamDestroy(origin);
    return result;
}

}  // extern "C"
