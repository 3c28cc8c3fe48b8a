// frame45.cuh -- the invariant frame of the 45-D multi-rocket game for the surrogate network.
//
// The game of Section 3.2 (14 pursuers and one evader, planar unicycles of Eq.
// multiagent_dynamics, target = distance from the evader to its nearest pursuer) is
// invariant under a common translation of all positions, under a common rotation of all
// positions together with the same turn of all headings, and -- when the pursuers share
// one speed -- under any permutation of the pursuers.  Its value function, and the
// correction v - l that the Picard iteration makes to its initial iterate, inherit these
// symmetries.  The frame removes them before the network sees a state: the evader sits at
// the origin with its heading along the first axis, and the pursuers, ordered by distance
// to the evader (ties by index), are given by their rotated relative positions
// r_k = R(-theta_e)(p_i - p_e) and the cosine and sine of their relative headings
// phi_k = theta_i - theta_e: 4 x 14 = 56 inputs.
//
// The network's 43 outputs are the correction in that frame: (dv, then per ordered pursuer
// u_k = d(v - l)/d r_k and w_k = d(v - l)/d phi_k).  By the chain rule the correction of Dv
// in state coordinates is, for pursuer i = order[k], d/dp_i = R(-theta_e)^T u_k and
// d/dtheta_i = w_k; translation invariance gives d/dp_e = -sum_i d/dp_i, and
// d/dtheta_e = sum_k (u_k,x r_k,z - u_k,z r_k,x) - sum_k w_k (the derivative of R(-theta_e)
// and of the relative headings).  The same maps turn a sweep's iterate into training
// targets.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "games.cuh"

namespace hjg {

constexpr int kF45P = 14;              // pursuers
constexpr int kF45In = 4 * kF45P;      // frame inputs
constexpr int kF45Out = 1 + 3 * kF45P; // frame outputs

// Pursuers of state x ordered by squared distance to the evader (stable: ties keep the
// index order): ord[k] is the index of the k-th nearest.
__device__ __forceinline__ void frame45_order(const double* x, int* ord) {
    double d2[kF45P];
    for (int i = 0; i < kF45P; ++i) {
        const double dx = x[3 * i] - x[42], dz = x[3 * i + 1] - x[43];
        const double d = dx * dx + dz * dz;
        int k = i;
        while (k > 0 && d2[k - 1] > d) { d2[k] = d2[k - 1]; ord[k] = ord[k - 1]; --k; }
        d2[k] = d;
        ord[k] = i;
    }
}

// mode 0: features [M][ldo] (56 used); mode 1: training targets [M][ldo] (43 used) from the
// iterate (v, p) minus the initial iterate (l, Dl).
__global__ void frame45_out_kernel(const float* __restrict__ x, int64_t ldx, int64_t M, GameParams g,
                                   const double* __restrict__ v, const float* __restrict__ p, int64_t ldp,
                                   float* __restrict__ out, int64_t ldo, int mode) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double xd[45];
    for (int j = 0; j < 45; ++j) xd[j] = (double)x[m * ldx + j];
    int ord[kF45P];
    frame45_order(xd, ord);
    double se, ce;
    sincos(xd[44], &se, &ce);
    float* o = out + m * ldo;
    if (mode == 0) {
        for (int k = 0; k < kF45P; ++k) {
            const int i = ord[k];
            const double dx = xd[3 * i] - xd[42], dz = xd[3 * i + 1] - xd[43];
            double sp, cp;
            sincos(xd[3 * i + 2] - xd[44], &sp, &cp);
            o[4 * k] = (float)(dx * ce + dz * se);
            o[4 * k + 1] = (float)(-dx * se + dz * ce);
            o[4 * k + 2] = (float)cp;
            o[4 * k + 3] = (float)sp;
        }
        return;
    }
    double gr[45];
    Rockets45::grad_ell_d(xd, gr, g);
    o[0] = (float)(v[m] - Rockets45::ell_d(xd, g));
    for (int k = 0; k < kF45P; ++k) {
        const int i = ord[k];
        const double ax = (double)p[m * ldp + 3 * i] - gr[3 * i];
        const double az = (double)p[m * ldp + 3 * i + 1] - gr[3 * i + 1];
        o[1 + 3 * k] = (float)(ax * ce + az * se);     // u = R(-theta_e) d/dp_i
        o[1 + 3 * k + 1] = (float)(-ax * se + az * ce);
        o[1 + 3 * k + 2] = (float)((double)p[m * ldp + 3 * i + 2] - gr[3 * i + 2]);
    }
}

// Warm start from the network's frame outputs pred [M][ldpr]: v = l + dv, Dv = Dl + the
// correction mapped back to state coordinates, c = Gamma(Dv) on the stored FP32 Dv.  With
// positions_only the heading rows of Dv keep Dl's (zero: l does not depend on the headings)
// and only the position rows take the correction.
__global__ void frame45_warm_kernel(const float* __restrict__ x, int64_t ldx, int64_t M, GameParams g,
                                    double delta, double eta, double c_min, double c_max,
                                    const float* __restrict__ pred, int64_t ldpr, bool positions_only,
                                    double* __restrict__ v, float* __restrict__ p, int64_t ldp,
                                    float* __restrict__ c) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double xd[45], gr[45];
    for (int j = 0; j < 45; ++j) xd[j] = (double)x[m * ldx + j];
    int ord[kF45P];
    frame45_order(xd, ord);
    double se, ce;
    sincos(xd[44], &se, &ce);
    Rockets45::grad_ell_d(xd, gr, g);
    const float* q = pred + m * ldpr;
    double ex = 0.0, ez = 0.0, th = 0.0;
    for (int k = 0; k < kF45P; ++k) {
        const int i = ord[k];
        const double ux = (double)q[1 + 3 * k], uz = (double)q[1 + 3 * k + 1], w = (double)q[1 + 3 * k + 2];
        const double dx = xd[3 * i] - xd[42], dz = xd[3 * i + 1] - xd[43];
        const double rx = dx * ce + dz * se, rz = -dx * se + dz * ce;
        const double gx = ux * ce - uz * se, gz = ux * se + uz * ce;   // R(-theta_e)^T u
        gr[3 * i] += gx;
        gr[3 * i + 1] += gz;
        if (!positions_only) gr[3 * i + 2] += w;
        ex -= gx;
        ez -= gz;
        th += ux * rz - uz * rx - w;
    }
    gr[42] += ex;
    gr[43] += ez;
    if (!positions_only) gr[44] += th;
    v[m] = Rockets45::ell_d(xd, g) + (double)q[0];
    double pp = 0.0;
    for (int j = 0; j < 45; ++j) {
        const float pj = (float)gr[j];
        p[m * ldp + j] = pj;
        pp += (double)pj * (double)pj;
        gr[j] = (double)pj;   // Gamma of the stored FP32 Dv, as after any sweep
    }
    int clipped;
    c[m] = (float)coef_update(Rockets45::ham_d(xd, gr, g), pp, delta, eta, c_min, c_max, g.tube, &clipped);
}

}  // namespace hjg
