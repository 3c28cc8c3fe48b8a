// games.cuh -- targets l, their gradients and closed-form Hamiltonians
// H(x, p) = max_u min_d <p, f(x, u, d)> (Eq. sign_convention) for the games the
// sweep supports.  Sample-level targets run in FP32 on registers; the per-state
// quantities of the coefficient update (Eq. coeff_frozen) run in FP64.
#pragma once
#include <cmath>
#include <cstdint>

namespace hjg {

struct GameParams {
    int32_t game;
    int32_t n;
    int32_t tube;     // 1: the tube form, Gamma built from min{0, H} (Eq. HJ-RCBRT-Visc)
    float radius;
    float h_sign;
    float speed[16];
    float A[64];      // quadratic test target (row-major n x n)
    float x0[8];
    float d;
    double radius_d;
    double h_sign_d;
    double speed_d[16];
    double A_d[64];
    double x0_d[8];
    double d_d;
    int32_t obstacle;   // 1: reach-avoid avoid disc in the plane of state dims 0, 1
    float obs_c[2];     // its centre
    float obs_off;      // radius + obstacle radius: the sample datum max{l, o} in "dist" units
    double obs_c_d[2];
    double obs_r_d;     // obstacle radius
};

// ------------------------------------------------------------- reach-avoid obstacle
// Reading of Eq. HJI-RCBRAT-Visc: an avoid disc with constraint function o(y) = r_O -
// |y_{0,1} - c_O| (> 0 inside).  The sweep's datum is max{l, o}; after every sweep the value
// is held above o: v <- max{v, o(x)}, Dv <- Do(x) where the obstacle binds.
// Sample level (FP32): the games' "dist" returns d with l = d - radius, so max{l, o} is
// max{d, radius + r_O - |y - c_O|}.
__device__ __forceinline__ float obstacle_dist(float d, float y0, float y1, const GameParams& g) {
    const float ox = y0 - g.obs_c[0], oy = y1 - g.obs_c[1];
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(fmaf(ox, ox, oy * oy)));
    return fmaxf(d, g.obs_off - r);
}
__device__ inline double obstacle_d(const double* x, const GameParams& g) {
    const double dx = x[0] - g.obs_c_d[0], dy = x[1] - g.obs_c_d[1];
    return g.obs_r_d - sqrt(dx * dx + dy * dy);
}
__device__ inline void obstacle_grad_d(const double* x, const GameParams& g, int n, double* gr) {
    const double dx = x[0] - g.obs_c_d[0], dy = x[1] - g.obs_c_d[1];
    const double rho = sqrt(dx * dx + dy * dy);
    for (int j = 0; j < n; ++j) gr[j] = 0.0;
    if (rho > 0) { gr[0] = -dx / rho; gr[1] = -dy / rho; }
}
// The projection after a sweep: true (and v, Dv replaced) where the obstacle binds.
__device__ inline bool obstacle_project(const double* x, const GameParams& g, int n, double& v, double* pd) {
    if (!g.obstacle) return false;
    const double o = obstacle_d(x, g);
    if (!(o > v)) return false;
    v = o;
    obstacle_grad_d(x, g, n, pd);
    return true;
}

enum GameId : int32_t {
    kDubins3 = 1, kRockets6 = 2, kRockets45 = 3, kFlock4 = 4, kRocketsRel3 = 5, kDoubleInt2 = 6,
    kTestQuadratic = 100, kTestZeroH = 101
};

// ---------------------------------------------------------------- Dubins (App. D.2)
// x1' = -1 + cos x3 + u x2,  x2' = sin x3 - u x1,  x3' = d - u;  u evader (max), d pursuer (min)
// Per-sample target in the sweep: l(y) = dist(...) - radius (radius 0 for the quadratic
// tests), with y = yoff + sk z for the sample mean yoff and the scaled raw normals z.
__device__ __forceinline__ float sqrtf_fast(float a) {
    float r; asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a)); return r;
}

struct Dubins3 {
    static constexpr int kN = 3;
    static constexpr bool kRadius = true;
    static constexpr int kAux = 0;
    static constexpr bool kObstacle = true;   // supports the reach-avoid obstacle (dims 0, 1 a position)
    __device__ static __forceinline__ float dist(const float* z, const float* yoff, float sk,
                                                 const GameParams& g, const float* = nullptr) {
        const float y0 = fmaf(sk, z[0], yoff[0]), y1 = fmaf(sk, z[1], yoff[1]);
        const float d = sqrtf_fast(fmaf(y0, y0, y1 * y1));
        return g.obstacle ? obstacle_dist(d, y0, y1, g) : d;
    }
    __device__ static double ell_d(const double* x, const GameParams& g, const float* = nullptr) {
        const double l = sqrt(x[0] * x[0] + x[1] * x[1]) - g.radius_d;
        return g.obstacle ? fmax(l, obstacle_d(x, g)) : l;
    }
    __device__ static void grad_ell_d(const double* x, double* gr, const GameParams& g, const float* = nullptr) {
        const double rho = sqrt(x[0] * x[0] + x[1] * x[1]);
        if (g.obstacle && obstacle_d(x, g) > rho - g.radius_d) { obstacle_grad_d(x, g, kN, gr); return; }
        gr[0] = rho > 0 ? x[0] / rho : 0.0;
        gr[1] = rho > 0 ? x[1] / rho : 0.0;
        gr[2] = 0.0;
    }
    __device__ static double ham_d(const double* x, const double* p, const GameParams&, const float* = nullptr) {
        double s, c;
        sincos(x[2], &s, &c);
        return p[0] * (c - 1.0) + p[1] * s + fabs(p[0] * x[1] - p[1] * x[0] - p[2]) - fabs(p[2]);
    }
    // Per-state trigonometric cache of H (computed once per state, one value per thread).
    static constexpr int kCache = 2;
    __device__ static double cache(const double* x, int j, const float* = nullptr) { return j == 0 ? cos(x[2]) : sin(x[2]); }
    __device__ static double ham_c(const double* x, const double* hc, const double* p, const GameParams&) {
        return p[0] * (hc[0] - 1.0) + p[1] * hc[1] + fabs(p[0] * x[1] - p[1] * x[0] - p[2]) - fabs(p[2]);
    }
};

// ------------------------------------------------ relative rockets (App. D, Eq. ham_def)
// (x, z, th): f = (a cos th + u_e x, a sin th + a - g + u_p x, u_p - u_e), H = -max min <p, f>
// with a = speed[0], g = speed[1]; target: capture disc in the (x, z) plane.
struct RocketsRel3 {
    static constexpr int kN = 3;
    static constexpr bool kRadius = true;
    static constexpr int kAux = 0;
    static constexpr bool kObstacle = true;   // supports the reach-avoid obstacle (dims 0, 1 a position)
    __device__ static __forceinline__ float dist(const float* z, const float* yoff, float sk,
                                                 const GameParams& g, const float* = nullptr) {
        const float y0 = fmaf(sk, z[0], yoff[0]), y1 = fmaf(sk, z[1], yoff[1]);
        const float d = sqrtf_fast(fmaf(y0, y0, y1 * y1));
        return g.obstacle ? obstacle_dist(d, y0, y1, g) : d;
    }
    __device__ static double ell_d(const double* x, const GameParams& g, const float* = nullptr) {
        const double l = sqrt(x[0] * x[0] + x[1] * x[1]) - g.radius_d;
        return g.obstacle ? fmax(l, obstacle_d(x, g)) : l;
    }
    __device__ static void grad_ell_d(const double* x, double* gr, const GameParams& g, const float* = nullptr) {
        const double rho = sqrt(x[0] * x[0] + x[1] * x[1]);
        if (g.obstacle && obstacle_d(x, g) > rho - g.radius_d) { obstacle_grad_d(x, g, kN, gr); return; }
        gr[0] = rho > 0 ? x[0] / rho : 0.0;
        gr[1] = rho > 0 ? x[1] / rho : 0.0;
        gr[2] = 0.0;
    }
    __device__ static double ham_h(const double* x, double c, double s, const double* p, const GameParams& g) {
        const double a = g.speed_d[0], gr = g.speed_d[1];
        return -(a * p[0] * c + p[1] * (a * s + a - gr) + fabs(p[0] * x[0] - p[2]) - fabs(p[1] * x[0] + p[2]));
    }
    __device__ static double ham_d(const double* x, const double* p, const GameParams& g, const float* = nullptr) {
        double s, c;
        sincos(x[2], &s, &c);
        return ham_h(x, c, s, p, g);
    }
    static constexpr int kCache = 2;
    __device__ static double cache(const double* x, int j, const float* = nullptr) { return j == 0 ? cos(x[2]) : sin(x[2]); }
    __device__ static double ham_c(const double* x, const double* hc, const double* p, const GameParams& g) {
        return ham_h(x, hc[0], hc[1], p, g);
    }
};

// ------------------------------------------------ double integrator (App. D, Eq. dint_ham)
// x1' = x2, x2' = u, |u| <= 1, u minimises: H = p1 x2 - |p2|; target: disc about the origin.
struct DoubleInt2 {
    static constexpr int kN = 2;
    static constexpr bool kRadius = true;
    static constexpr int kAux = 0;
    static constexpr bool kObstacle = true;   // supports the reach-avoid obstacle (dims 0, 1 a position)
    __device__ static __forceinline__ float dist(const float* z, const float* yoff, float sk,
                                                 const GameParams& g, const float* = nullptr) {
        const float y0 = fmaf(sk, z[0], yoff[0]), y1 = fmaf(sk, z[1], yoff[1]);
        const float d = sqrtf_fast(fmaf(y0, y0, y1 * y1));
        return g.obstacle ? obstacle_dist(d, y0, y1, g) : d;
    }
    __device__ static double ell_d(const double* x, const GameParams& g, const float* = nullptr) {
        const double l = sqrt(x[0] * x[0] + x[1] * x[1]) - g.radius_d;
        return g.obstacle ? fmax(l, obstacle_d(x, g)) : l;
    }
    __device__ static void grad_ell_d(const double* x, double* gr, const GameParams& g, const float* = nullptr) {
        const double rho = sqrt(x[0] * x[0] + x[1] * x[1]);
        if (g.obstacle && obstacle_d(x, g) > rho - g.radius_d) { obstacle_grad_d(x, g, kN, gr); return; }
        gr[0] = rho > 0 ? x[0] / rho : 0.0;
        gr[1] = rho > 0 ? x[1] / rho : 0.0;
    }
    __device__ static double ham_d(const double* x, const double* p, const GameParams&, const float* = nullptr) {
        return p[0] * x[1] - fabs(p[1]);
    }
    static constexpr int kCache = 0;
    __device__ static double cache(const double*, int, const float* = nullptr) { return 0.0; }
    __device__ static double ham_c(const double* x, const double*, const double* p, const GameParams&) {
        return p[0] * x[1] - fabs(p[1]);
    }
};

// ---------------------------------------------------------------- two rockets
// state (xA, zA, xB, zB, thA, thB); A: x' = a cos th, z' = a sin th, th' = u (max);
// B likewise with turn rate d (min).
struct Rockets6 {
    static constexpr int kN = 6;
    static constexpr bool kRadius = true;
    static constexpr int kAux = 0;
    static constexpr bool kObstacle = false;   // supports the reach-avoid obstacle (dims 0, 1 a position)
    __device__ static __forceinline__ float dist(const float* z, const float* yoff, float sk,
                                                 const GameParams&, const float* = nullptr) {
        const float dx = fmaf(sk, z[0] - z[2], yoff[0] - yoff[2]);
        const float dz = fmaf(sk, z[1] - z[3], yoff[1] - yoff[3]);
        return sqrtf_fast(fmaf(dx, dx, dz * dz));
    }
    __device__ static double ell_d(const double* x, const GameParams& g, const float* = nullptr) {
        const double dx = x[0] - x[2], dz = x[1] - x[3];
        return sqrt(dx * dx + dz * dz) - g.radius_d;
    }
    __device__ static void grad_ell_d(const double* x, double* gr, const GameParams&, const float* = nullptr) {
        const double dx = x[0] - x[2], dz = x[1] - x[3];
        const double rho = sqrt(dx * dx + dz * dz);
        const double a = rho > 0 ? dx / rho : 0.0, b = rho > 0 ? dz / rho : 0.0;
        gr[0] = a; gr[1] = b; gr[2] = -a; gr[3] = -b; gr[4] = 0.0; gr[5] = 0.0;
    }
    __device__ static double ham_d(const double* x, const double* p, const GameParams& g, const float* = nullptr) {
        double sA, cA, sB, cB;
        sincos(x[4], &sA, &cA);
        sincos(x[5], &sB, &cB);
        return g.speed_d[0] * (p[0] * cA + p[1] * sA) + g.speed_d[1] * (p[2] * cB + p[3] * sB)
             + fabs(p[4]) - fabs(p[5]);
    }
    static constexpr int kCache = 4;   // cos thA, sin thA, cos thB, sin thB
    __device__ static double cache(const double* x, int j, const float* = nullptr) {
        const double a = x[4 + (j >> 1)];
        return (j & 1) ? sin(a) : cos(a);
    }
    __device__ static double ham_c(const double*, const double* hc, const double* p, const GameParams& g) {
        return g.speed_d[0] * (p[0] * hc[0] + p[1] * hc[1]) + g.speed_d[1] * (p[2] * hc[2] + p[3] * hc[3])
             + fabs(p[4]) - fabs(p[5]);
    }
};

// ---------------------------------------------------------------- 15 rockets (Sec. 3.2)
// agents i = 0..14 with (x_i, z_i, th_i) at dims 3i..3i+2; agent 14 evades.
// l = min_{i < 14} |pos_i - pos_14| - r.  The per-sample target is evaluated cooperatively
// by the two lanes of a sample (sweep_kernel_r45); only the per-state FP64 parts live here.
struct Rockets45 {
    static constexpr int kN = 45;
    static constexpr bool kRadius = true;
    static constexpr int kAux = 0;
    static constexpr bool kObstacle = false;   // supports the reach-avoid obstacle (dims 0, 1 a position)
    __device__ static double ell_d(const double* x, const GameParams& g, const float* = nullptr) {
        double best = INFINITY;
        for (int i = 0; i < 14; ++i) {
            const double dx = x[3 * i] - x[42], dz = x[3 * i + 1] - x[43];
            best = fmin(best, sqrt(dx * dx + dz * dz));
        }
        return best - g.radius_d;
    }
    __device__ static void grad_ell_d(const double* x, double* gr, const GameParams&, const float* = nullptr) {
        int arg = -1;
        double best = INFINITY;
        for (int i = 0; i < 14; ++i) {
            const double dx = x[3 * i] - x[42], dz = x[3 * i + 1] - x[43];
            const double dd = sqrt(dx * dx + dz * dz);
            if (dd < best) { best = dd; arg = i; }
        }
        for (int a = 0; a < 45; ++a) gr[a] = 0.0;
        if (arg >= 0 && best > 0) {
            const double dx = x[3 * arg] - x[42], dz = x[3 * arg + 1] - x[43];
            gr[3 * arg] = dx / best; gr[3 * arg + 1] = dz / best;
            gr[42] = -dx / best; gr[43] = -dz / best;
        }
    }
    __device__ static double ham_d(const double* x, const double* p, const GameParams& g, const float* = nullptr) {
        double h = 0.0;
        for (int i = 0; i < 15; ++i) {
            double s, c;
            sincos(x[3 * i + 2], &s, &c);
            h += g.speed_d[i] * (p[3 * i] * c + p[3 * i + 1] * s);
        }
        h += fabs(p[44]);
        for (int i = 0; i < 14; ++i) h -= fabs(p[3 * i + 2]);
        return h;
    }
    static constexpr int kCache = 30;  // cos th_i, sin th_i for the 15 agents
    __device__ static double cache(const double* x, int j, const float* = nullptr) {
        const double a = x[3 * (j >> 1) + 2];
        return (j & 1) ? sin(a) : cos(a);
    }
    __device__ static double ham_c(const double*, const double* hc, const double* p, const GameParams& g) {
        double h = fabs(p[44]);
        for (int i = 0; i < 15; ++i) h += g.speed_d[i] * (p[3 * i] * hc[2 * i] + p[3 * i + 1] * hc[2 * i + 1]);
        for (int i = 0; i < 14; ++i) h -= fabs(p[3 * i + 2]);
        return h;
    }
};

// ---------------------------------------------------------------- murmuration agent
// One starling of the flock game (Appendix D.5, in the per-agent reading): state
// (p_x, p_y, p_z, psi).  The agent flies at speed a in its heading, sets its climb rate
// u_z (|u_z| <= 1, maximises), and its heading relaxes toward the circular mean heading
// psibar of its 7 nearest neighbours under a bounded attack disturbance d (|d| <= 1,
// minimises): p' = (a cos psi, a sin psi, u_z), psi' = wrap(psibar - psi) + d.  Target:
// distance to the nearest of those (frozen) neighbours minus the radius (union of the
// per-neighbour signed distances, Eq. sdf_union).  Per-state data aux = the 7 neighbour
// positions (21 floats) followed by psibar.
__device__ __forceinline__ double wrap_angle_d(double a) {
    const double two_pi = 6.283185307179586476925286766559;
    double r = fmod(a + 3.14159265358979323846, two_pi);
    if (r <= 0.0) r += two_pi;
    return r - 3.14159265358979323846;
}

struct Flock4 {
    static constexpr int kN = 4;
    static constexpr bool kRadius = true;
    static constexpr int kAux = 22;
    static constexpr bool kObstacle = false;   // supports the reach-avoid obstacle (dims 0, 1 a position)
    static constexpr int kNbr = 7;
    __device__ static __forceinline__ float dist(const float* z, const float* yoff, float sk,
                                                 const GameParams&, const float* aux) {
        const float y0 = fmaf(sk, z[0], yoff[0]), y1 = fmaf(sk, z[1], yoff[1]), y2 = fmaf(sk, z[2], yoff[2]);
        float best = INFINITY;
#pragma unroll
        for (int j = 0; j < kNbr; ++j) {
            const float dx = y0 - aux[3 * j], dy = y1 - aux[3 * j + 1], dz = y2 - aux[3 * j + 2];
            best = fminf(best, fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        }
        return sqrtf_fast(best);
    }
    __device__ static double ell_d(const double* x, const GameParams& g, const float* aux) {
        double best = INFINITY;
        for (int j = 0; j < kNbr; ++j) {
            const double dx = x[0] - aux[3 * j], dy = x[1] - aux[3 * j + 1], dz = x[2] - aux[3 * j + 2];
            best = fmin(best, sqrt(dx * dx + dy * dy + dz * dz));
        }
        return best - g.radius_d;
    }
    __device__ static void grad_ell_d(const double* x, double* gr, const GameParams&, const float* aux) {
        int arg = -1;
        double best = INFINITY;
        for (int j = 0; j < kNbr; ++j) {
            const double dx = x[0] - aux[3 * j], dy = x[1] - aux[3 * j + 1], dz = x[2] - aux[3 * j + 2];
            const double dd = sqrt(dx * dx + dy * dy + dz * dz);
            if (dd < best) { best = dd; arg = j; }
        }
        for (int a = 0; a < 4; ++a) gr[a] = 0.0;
        if (arg >= 0 && best > 0)
            for (int a = 0; a < 3; ++a) gr[a] = (x[a] - aux[3 * arg + a]) / best;
    }
    __device__ static double ham_d(const double* x, const double* p, const GameParams& g, const float* aux) {
        double s, c;
        sincos(x[3], &s, &c);
        return g.speed_d[0] * (p[0] * c + p[1] * s) + fabs(p[2]) + p[3] * wrap_angle_d((double)aux[21] - x[3])
             - fabs(p[3]);
    }
    static constexpr int kCache = 3;   // cos psi, sin psi, wrap(psibar - psi)
    __device__ static double cache(const double* x, int j, const float* aux) {
        return j == 0 ? cos(x[3]) : (j == 1 ? sin(x[3]) : wrap_angle_d((double)aux[21] - x[3]));
    }
    __device__ static double ham_c(const double*, const double* hc, const double* p, const GameParams& g) {
        return g.speed_d[0] * (p[0] * hc[0] + p[1] * hc[1]) + fabs(p[2]) + p[3] * hc[2] - fabs(p[3]);
    }
};

// ---------------------------------------------------------------- quadratic tests
// H = h_sign |p|^2 / 2 (ZERO_H: H = 0), l = (y - x0)^T A (y - x0) / 2 + d.  NDIM <= 8.
template <int NDIM, bool kZeroH>
struct Quadratic {
    static constexpr int kN = NDIM;
    static constexpr bool kRadius = false;
    static constexpr int kAux = 0;
    static constexpr bool kObstacle = false;
    __device__ static __forceinline__ float dist(const float* z, const float* yoff, float sk,
                                                 const GameParams& g, const float* = nullptr) {
        float e[NDIM];
#pragma unroll
        for (int a = 0; a < NDIM; ++a) e[a] = fmaf(sk, z[a], yoff[a]) - g.x0[a];
        float r = 0.0f;
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            float row = 0.0f;
#pragma unroll
            for (int b = 0; b < NDIM; ++b) row = fmaf(g.A[a * NDIM + b], e[b], row);
            r = fmaf(e[a], row, r);
        }
        return fmaf(0.5f, r, g.d);
    }
    __device__ static double ell_d(const double* x, const GameParams& g, const float* = nullptr) {
        double r = 0.0;
        for (int a = 0; a < NDIM; ++a)
            for (int b = 0; b < NDIM; ++b)
                r += (x[a] - g.x0_d[a]) * g.A_d[a * NDIM + b] * (x[b] - g.x0_d[b]);
        return 0.5 * r + g.d_d;
    }
    __device__ static void grad_ell_d(const double* x, double* gr, const GameParams& g, const float* = nullptr) {
        for (int a = 0; a < NDIM; ++a) {
            double s = 0.0;
            for (int b = 0; b < NDIM; ++b) s += g.A_d[a * NDIM + b] * (x[b] - g.x0_d[b]);
            gr[a] = s;
        }
    }
    __device__ static double ham_d(const double*, const double* p, const GameParams& g, const float* = nullptr) {
        if (kZeroH) return 0.0;
        double s = 0.0;
        for (int a = 0; a < NDIM; ++a) s += p[a] * p[a];
        return g.h_sign_d * 0.5 * s;
    }
    static constexpr int kCache = 0;
    __device__ static double cache(const double*, int, const float* = nullptr) { return 0.0; }
    __device__ static double ham_c(const double* x, const double*, const double* p, const GameParams& g) {
        return ham_d(x, p, g);
    }
};

// Coefficient-update map Gamma (Eq. coeff_frozen with the regulariser of Lemma 2.7 and
// the sign-keeping clip of Remark 2.8; sign(0) = +, NaN -> c_min).
__device__ __forceinline__ double coef_update(double h, double pp, double delta, double eta,
                                              double c_min, double c_max, int tube, int* clipped) {
    if (tube) h = fmin(h, 0.0);   // the freezing operator min{0, H} of the tube form
    const double c = (2.0 / delta) * h / (pp + eta);
    double mag = fabs(c);
    int cl = 0;
    if (!(mag >= c_min)) { mag = c_min; cl = 1; }
    if (mag > c_max) { mag = c_max; cl = 1; }
    *clipped = cl;
    return (c < 0.0) ? -mag : mag;
}

}  // namespace hjg
