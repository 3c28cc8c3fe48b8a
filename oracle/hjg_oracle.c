/*
 * hjg_oracle.c -- plain, slow FP64 CPU oracle for the HJ-Gauss frozen-coefficient
 * Picard sweep (arXiv 2605.18566).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link or call
 * this file; it exists so that the tests, the smoke check and the CPU baseline of the
 * benchmark can compare the CUDA path against an independent restatement of the paper.
 * It shares no source with the CUDA library.
 *
 * What it computes, and where the paper defines it:
 *   - Algorithm 1 (quasi-linearisation Picard loop): v^(0)=g, c^(0)=Gamma(Dg); per
 *     sweep freeze c, solve the heat equation through its Gaussian expectation,
 *     recover v = -(1/c) log phi, update Dv and c, report the relative change.
 *   - Eq. (coeff_frozen) / Lemma 2.7 (coeff_regularized): c = (2/delta) H / (|p|^2+eta),
 *     Remark 2.8 (coeff_sign): sign kept, |c| clipped to [c_min, c_max].
 *   - Proposition 2.1 / Lemma 2.2 (heat-kernel expectation, sample covariance delta*t*I),
 *     Corollary B.4 (log-sum-exp value estimator), Corollary B.5 (MC gradient estimator
 *     (x - sum s_i w_i / sum w_i) / (t delta c)), Corollary B.6 (tilted proposal with
 *     density-ratio weight w_theta), Section 2.4 (ESS).
 *   - Games: Appendix D.2 Dubins relative game (Hamiltonian of Eq. dubins_ham_unit
 *     with the sign of the p2 term taken from the dynamics of Eq. dubins_dyna),
 *     Section 3.2 multi-rocket game (Eq. multiagent_dynamics), a two-rocket planar game
 *     built from the same per-agent dynamics, the relative two-rocket game (Eq. ham_def),
 *     the double integrator (Eq. dint_ham), the flock of Appendix D.5 (aerial Dubins
 *     agents steered toward the circular mean heading of their 7 nearest neighbours,
 *     target = nearness to those neighbours), and quadratic test problems
 *     (H = +-|p|^2/2, the exact Cole-Hopf case of Corollary B.2).
 *   - Reach-avoid tube (reading of Eq. HJI-RCBRAT-Visc): an avoid disc whose constraint
 *     function o enters the datum as max{l, o} and bounds the value from below after every
 *     sweep (see obstacle_fn).
 *   - Counter-based sampler: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11); each
 *     32-bit word of a block gives one Box-Muller pair (radius uniform ((x & (2^20-1)) + 0.5)
 *     2^-20 from its low 20 bits, angle uniform ((x >> 20) + 0.5) 2^-12 from its high 12),
 *     eight normals per block; packed per-sample slots.
 *
 * Everything is double precision except the Philox integer stream itself.
 * Pinned by tests/test_oracle_*.py (closed forms, quadrature, brute force, an
 * independent Philox implementation); see each function for its pin.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXN 64

enum {
    ORC_DUBINS3 = 1,
    ORC_ROCKETS6 = 2,
    ORC_ROCKETS45 = 3,
    ORC_FLOCK4 = 4,
    ORC_ROCKETS_REL3 = 5,
    ORC_DOUBLE_INT2 = 6,
    ORC_TEST_QUADRATIC = 100,
    ORC_TEST_ZERO_H = 101
};

/* Problem description.  Field order is mirrored by the ctypes Structure in
 * oracle/__init__.py. */
typedef struct {
    int32_t game;
    int32_t n;          /* state dimension */
    double delta;       /* viscosity delta (= 2 nu) */
    double T;           /* horizon t at which v(t;x) is evaluated */
    double eta;         /* denominator regulariser of Lemma 2.7 */
    double c_min;       /* |c| clip bounds of Remark 2.8 */
    double c_max;
    double radius;      /* capture radius of the signed-distance target */
    double speed[16];   /* per-agent forward speeds */
    double h_sign;      /* quadratic test: H = h_sign * |p|^2 / 2 */
    double A[64];       /* quadratic test target l(y) = (y-x0)^T A (y-x0)/2 + d, A row-major n x n */
    double x0[8];
    double d;
    uint64_t seed;
    uint32_t instance;
    int32_t tilt;       /* 1: tilted proposal theta = -sigma^2 c p (Eq. tilt_shift) */
    int32_t flock_k;    /* flock: neighbours per agent */
    int32_t tube;       /* 1: tube form, Gamma built from min{0, H} (Eq. HJ-RCBRT-Visc) */
    int32_t cv;         /* 1: Stein control variate around the current iterate (see solve_point) */
    int32_t obstacle;   /* 1: reach-avoid obstacle, a disc in the plane of state dims 0, 1 */
    double obs_c[2];    /* obstacle centre */
    double obs_r;       /* obstacle radius */
} orc_problem;

/* ------------------------------------------------------------------------- */
/* Philox4x32-10.  Each round multiplies two counter words by fixed odd
 * constants (full 64-bit products), swaps and mixes the halves with the key,
 * and the key is advanced by the Weyl increments between rounds. */

static const uint32_t PHILOX_MUL0 = 0xD2511F53u;
static const uint32_t PHILOX_MUL1 = 0xCD9E8D57u;
static const uint32_t PHILOX_WEYL0 = 0x9E3779B9u;
static const uint32_t PHILOX_WEYL1 = 0xBB67AE85u;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)PHILOX_MUL0 * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)PHILOX_MUL1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += PHILOX_WEYL0;
        k1 += PHILOX_WEYL1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

void orc_philox_batch(int64_t count, const uint32_t *ctr, const uint32_t *key, uint32_t *out)
{
    for (int64_t i = 0; i < count; ++i)
        orc_philox4x32_10(ctr + 4 * i, key + 2 * i, out + 4 * i);
}

/* Radius uniform of one Philox word, strictly inside (0,1): the low 20 bits k give
 * u = (k + 0.5) 2^-20; every value is exact in FP32 and FP64. */
double orc_u01(uint32_t x)
{
    return ((double)(x & 0xFFFFFu) + 0.5) * (1.0 / 1048576.0);
}

/* Angle uniform of one Philox word: the high 12 bits k give (k + 0.5) 2^-12, also exact in
 * both precisions. */
static double angle_u(uint32_t x)
{
    return ((double)(x >> 20) + 0.5) / 4096.0;
}

/* Normals per Philox block: one Box-Muller pair per 32-bit word. */
#define ORC_NPB 8

/* Slots per sample in the normal stream of one (state, sweep): n for n <= 8 (the normals
 * of consecutive samples are packed back to back), n rounded up to a multiple of 8 above
 * (each sample starts on a fresh Philox block). */
int orc_slot_stride(int n)
{
    return n <= 8 ? n : (n + 7) / 8 * 8;
}

/* The eight normals of one Philox output block (X, Y, Z, W); block b of the stream of
 * (point, sweep) has counter (point, b_lo, sweep, b_hi) and key (seed_lo, seed_hi ^
 * instance).  Word j = 0..3 makes pair j (slots 8b+2j, 8b+2j+1) and every one of its 32
 * bits feeds exactly one uniform: the radius uniform u_r from its low 20 bits, the angle
 * uniform u_a from its high 12 bits;
 *   (z_2j, z_2j+1) = sqrt(-2 ln u_r) (cos 2 pi u_a, sin 2 pi u_a)  (Box-Muller). */
void orc_block_words_normals(const uint32_t r[4], double zz[ORC_NPB])
{
    const double two_pi = 6.283185307179586476925286766559;
    for (int j = 0; j < 4; ++j) {
        double rad = sqrt(-2.0 * log(orc_u01(r[j])));
        double ua = angle_u(r[j]);
        zz[2 * j] = rad * cos(two_pi * ua);
        zz[2 * j + 1] = rad * sin(two_pi * ua);
    }
}

static void block_normals(uint64_t seed, uint32_t instance, uint64_t b, uint32_t point,
                          uint32_t sweep, double zz[ORC_NPB])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ instance};
    uint32_t ctr[4] = {point, (uint32_t)b, sweep, (uint32_t)(b >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    orc_block_words_normals(r, zz);
}

/* Standard normals z[0..n) of sample `sample` of state `point` in sweep `sweep`: slot
 * q = sample * orc_slot_stride(n) + d of the stream, i.e. lane q % 8 of block q / 8. */
void orc_normals(int n, uint64_t seed, uint32_t instance, uint32_t sample,
                 uint32_t point, uint32_t sweep, double *z)
{
    uint64_t q0 = (uint64_t)sample * (uint64_t)orc_slot_stride(n);
    uint64_t cached = UINT64_MAX;
    double zz[ORC_NPB] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int d = 0; d < n; ++d) {
        uint64_t q = q0 + (uint64_t)d;
        if (q / ORC_NPB != cached) {
            cached = q / ORC_NPB;
            block_normals(seed, instance, cached, point, sweep, zz);
        }
        z[d] = zz[q % ORC_NPB];
    }
}

/* ------------------------------------------------------------------------- */
/* Games: target l (signed distance), its gradient, and the closed-form
 * Hamiltonian H(x,p) = max_u min_d <p, f(x,u,d)>. */

/* Flock auxiliary data: per agent, k neighbour positions (3 each) followed by
 * the neighbours' circular-mean heading.  Unused by the other games. */
typedef struct {
    const double *nbr;  /* [M][k*3] */
    const double *psibar; /* [M] */
} orc_aux;

static double quad_form(const orc_problem *P, const double *y)
{
    int n = P->n;
    double r = P->d;
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b)
            r += 0.5 * (y[a] - P->x0[a]) * P->A[a * n + b] * (y[b] - P->x0[b]);
    return r;
}

static double ell_base(const orc_problem *P, const double *y, const double *nbr)
{
    switch (P->game) {
    case ORC_DUBINS3:
    case ORC_ROCKETS_REL3:   /* capture disc in the relative (x, z) plane */
    case ORC_DOUBLE_INT2:    /* disc about the origin of the (position, velocity) plane */
        return sqrt(y[0] * y[0] + y[1] * y[1]) - P->radius;
    case ORC_ROCKETS6: {
        double dx = y[0] - y[2], dz = y[1] - y[3];
        return sqrt(dx * dx + dz * dz) - P->radius;
    }
    case ORC_ROCKETS45: {
        /* agents i = 0..14 with state (x_i, z_i, theta_i); agent 14 evades */
        double best = INFINITY;
        for (int i = 0; i < 14; ++i) {
            double dx = y[3 * i] - y[42], dz = y[3 * i + 1] - y[43];
            double dist = sqrt(dx * dx + dz * dz);
            if (dist < best) best = dist;
        }
        return best - P->radius;
    }
    case ORC_FLOCK4: {
        double best = INFINITY;
        for (int j = 0; j < P->flock_k; ++j) {
            double dx = y[0] - nbr[3 * j], dy = y[1] - nbr[3 * j + 1], dz = y[2] - nbr[3 * j + 2];
            double dist = sqrt(dx * dx + dy * dy + dz * dz);
            if (dist < best) best = dist;
        }
        return best - P->radius;
    }
    case ORC_TEST_QUADRATIC:
    case ORC_TEST_ZERO_H:
        return quad_form(P, y);
    }
    return NAN;
}

/* Reach-avoid obstacle (reading of Eq. HJI-RCBRAT-Visc): the avoid set is a disc of radius
 * obs_r about obs_c in the plane of state dims 0 and 1 (the position, or relative position,
 * of the games that support it), with constraint function o(y) = obs_r - |y_{0,1} - obs_c|,
 * positive inside the obstacle.  The value is held above o: the datum of every sweep is
 * max{l, o} (a sample inside the obstacle counts as outside the target), and after every
 * sweep v <- max{v, o(x)} with Dv <- Do(x) where the obstacle binds -- the projection form of
 * the reach-avoid variational inequality max{min{v_t + H - (delta/2) Lap v, l - v}, o - v} = 0. */
static double obstacle_fn(const orc_problem *P, const double *y)
{
    double dx = y[0] - P->obs_c[0], dy = y[1] - P->obs_c[1];
    return P->obs_r - sqrt(dx * dx + dy * dy);
}

static void obstacle_grad(const orc_problem *P, const double *x, double *g)
{
    double dx = x[0] - P->obs_c[0], dy = x[1] - P->obs_c[1];
    double rho = sqrt(dx * dx + dy * dy);
    for (int a = 0; a < P->n; ++a) g[a] = 0.0;
    if (rho > 0) { g[0] = -dx / rho; g[1] = -dy / rho; }
}

/* The datum l of the sweep: the target's signed distance, or max{l, o} with an obstacle. */
double orc_ell(const orc_problem *P, const double *y, const double *nbr)
{
    double l = ell_base(P, y, nbr);
    if (P->obstacle) {
        double o = obstacle_fn(P, y);
        if (o > l) l = o;
    }
    return l;
}

static void grad_ell_base(const orc_problem *P, const double *x, const double *nbr, double *g);

/* Analytic gradient of the datum, 0 where it is undefined (the ridge of a distance); with
 * an obstacle, the gradient of whichever of l and o is larger. */
void orc_grad_ell(const orc_problem *P, const double *x, const double *nbr, double *g)
{
    if (P->obstacle && obstacle_fn(P, x) > ell_base(P, x, nbr)) {
        obstacle_grad(P, x, g);
        return;
    }
    grad_ell_base(P, x, nbr, g);
}

static void grad_ell_base(const orc_problem *P, const double *x, const double *nbr, double *g)
{
    int n = P->n;
    for (int a = 0; a < n; ++a) g[a] = 0.0;
    switch (P->game) {
    case ORC_DUBINS3:
    case ORC_ROCKETS_REL3:
    case ORC_DOUBLE_INT2: {
        double rho = sqrt(x[0] * x[0] + x[1] * x[1]);
        if (rho > 0) { g[0] = x[0] / rho; g[1] = x[1] / rho; }
        break;
    }
    case ORC_ROCKETS6: {
        double dx = x[0] - x[2], dz = x[1] - x[3];
        double rho = sqrt(dx * dx + dz * dz);
        if (rho > 0) { g[0] = dx / rho; g[1] = dz / rho; g[2] = -dx / rho; g[3] = -dz / rho; }
        break;
    }
    case ORC_ROCKETS45: {
        int arg = -1; double best = INFINITY;
        for (int i = 0; i < 14; ++i) {
            double dx = x[3 * i] - x[42], dz = x[3 * i + 1] - x[43];
            double dist = sqrt(dx * dx + dz * dz);
            if (dist < best) { best = dist; arg = i; }
        }
        if (arg >= 0 && best > 0) {
            double dx = x[3 * arg] - x[42], dz = x[3 * arg + 1] - x[43];
            g[3 * arg] = dx / best; g[3 * arg + 1] = dz / best;
            g[42] = -dx / best; g[43] = -dz / best;
        }
        break;
    }
    case ORC_FLOCK4: {
        int arg = -1; double best = INFINITY;
        for (int j = 0; j < P->flock_k; ++j) {
            double dx = x[0] - nbr[3 * j], dy = x[1] - nbr[3 * j + 1], dz = x[2] - nbr[3 * j + 2];
            double dist = sqrt(dx * dx + dy * dy + dz * dz);
            if (dist < best) { best = dist; arg = j; }
        }
        if (arg >= 0 && best > 0)
            for (int a = 0; a < 3; ++a) g[a] = (x[a] - nbr[3 * arg + a]) / best;
        break;
    }
    case ORC_TEST_QUADRATIC:
    case ORC_TEST_ZERO_H:
        for (int a = 0; a < n; ++a) {
            double s = 0.0;
            for (int b = 0; b < n; ++b) s += P->A[a * n + b] * (x[b] - P->x0[b]);
            g[a] = s;
        }
        break;
    }
}

/* wrap an angle difference into (-pi, pi] */
static double wrap_angle(double a)
{
    const double pi = 3.14159265358979323846;
    double r = fmod(a + pi, 2.0 * pi);
    if (r <= 0) r += 2.0 * pi;
    return r - pi;
}

double orc_hamiltonian(const orc_problem *P, const double *x, const double *p, double psibar)
{
    switch (P->game) {
    case ORC_DUBINS3:
        /* x1' = -1 + cos x3 + u x2, x2' = sin x3 - u x1, x3' = d - u; u evader (max), d pursuer (min) */
        return p[0] * (cos(x[2]) - 1.0) + p[1] * sin(x[2])
             + fabs(p[0] * x[1] - p[1] * x[0] - p[2]) - fabs(p[2]);
    case ORC_ROCKETS6:
        /* (xA,zA,xB,zB,thA,thB); A evader turn rate u (max), B pursuer turn rate d (min) */
        return P->speed[0] * (p[0] * cos(x[4]) + p[1] * sin(x[4]))
             + P->speed[1] * (p[2] * cos(x[5]) + p[3] * sin(x[5]))
             + fabs(p[4]) - fabs(p[5]);
    case ORC_ROCKETS45: {
        double h = 0.0;
        for (int i = 0; i < 15; ++i)
            h += P->speed[i] * (p[3 * i] * cos(x[3 * i + 2]) + p[3 * i + 1] * sin(x[3 * i + 2]));
        h += fabs(p[44]);
        for (int i = 0; i < 14; ++i) h -= fabs(p[3 * i + 2]);
        return h;
    }
    case ORC_FLOCK4:
        /* (px,py,pz,psi): p' = (v cos psi, v sin psi, u_z), psi' = wrap(psibar - psi) + d;
           the bird controls u_z (max), the attack disturbance d (min) */
        return P->speed[0] * (p[0] * cos(x[3]) + p[1] * sin(x[3])) + fabs(p[2])
             + p[3] * wrap_angle(psibar - x[3]) - fabs(p[3]);
    case ORC_ROCKETS_REL3: {
        /* relative rockets (x, z, theta), Eq. ham_def: f = (a cos th + u_e x,
           a sin th + a - g + u_p x, u_p - u_e), H = -max_{u_e} min_{u_p} <p, f> with
           a = speed[0], g = speed[1], |u_e|, |u_p| <= 1 */
        double a = P->speed[0], g = P->speed[1];
        return -(a * p[0] * cos(x[2]) + p[1] * (a * sin(x[2]) + a - g)
                 + fabs(p[0] * x[0] - p[2]) - fabs(p[1] * x[0] + p[2]));
    }
    case ORC_DOUBLE_INT2:
        /* x1' = x2, x2' = u, |u| <= 1, the control minimises (Eq. dint_ham) */
        return p[0] * x[1] - fabs(p[1]);
    case ORC_TEST_QUADRATIC: {
        double s = 0.0;
        for (int a = 0; a < P->n; ++a) s += p[a] * p[a];
        return P->h_sign * 0.5 * s;
    }
    case ORC_TEST_ZERO_H:
        return 0.0;
    }
    return NAN;
}

/* Coefficient-update map Gamma of Theorem 2.8 with the regularised denominator
 * of Lemma 2.7 and the sign-keeping clip of Remark 2.8 (sign(0) taken as +).  The
 * tube form (Eq. HJ-RCBRT-Visc) replaces H by min{0, H}. */
double orc_coef(const orc_problem *P, const double *x, const double *p, double psibar)
{
    double h = orc_hamiltonian(P, x, p, psibar);
    if (P->tube && !(h <= 0.0)) h = 0.0;   /* min{0, H}; a NaN H counts as 0 */
    double pp = 0.0;
    for (int a = 0; a < P->n; ++a) pp += p[a] * p[a];
    double c = (2.0 / P->delta) * h / (pp + P->eta);
    double mag = fabs(c);
    if (!(mag >= P->c_min)) mag = P->c_min; /* also maps NaN to c_min */
    if (mag > P->c_max) mag = P->c_max;
    return (c < 0.0) ? -mag : mag;
}

/* ------------------------------------------------------------------------- */
/* One frozen-coefficient heat-kernel solve at one evaluation state.
 *   samples  y_i = x + theta + sqrt(delta t) z_i,  z_i ~ N(0,I)  (theta = 0 untilted)
 *   log-weights  lw_i = -c l(y_i) + (|theta|^2 - 2<y_i - x, theta>)/(2 sigma^2)
 *   v  = -(1/c) log( (1/N) sum_i exp(lw_i) )              (Cor. B.4 / B.6)
 *   Dv = (x - sum_i y_i w_i / sum_i w_i) / (t delta c)     (Cor. B.5 / B.6)
 *   ESS = (sum w)^2 / sum w^2                              (Section 2.4)
 * Two passes: the first finds max lw (log-sum-exp shift), the second regenerates
 * the same samples and accumulates.
 *
 * Control variate (cv_g != NULL): zero-mean Stein polynomials of the normals with
 * coefficients from a guess (v_hat, g_hat) of the value and gradient at x (the current
 * iterate, or a surrogate's prediction after a warm start).  To first order the weight is
 * w ~ mu (1 + b.z) with mu = exp(-c v_hat) and b = -c sigma g_hat - theta / sigma; b is 0
 * in the tilted frame (theta = -sigma^2 c g_hat removes the linear term), so there b = 0.
 * The sums become
 *   sum w        -> sum w - mu b.(sum z)
 *   sum w z      -> sum w z - mu (sum z + sum z (z.b) - N b)
 * (E z = 0, E (z z^T - I) = 0: both corrections have mean zero for any fixed mu, b).  The
 * uncorrected sums are kept when the guess is poor -- mu more than a factor 4 away from the
 * sample mean weight (sum w)/N -- or the corrected weight sum is not positive.  ESS stays
 * that of the raw weights. */
static void solve_point(const orc_problem *P, const double *x, double c, const double *theta,
                        const double *nbr, int64_t N, uint32_t point, uint32_t sweep,
                        const double *cv_g, double cv_v,
                        double *lw, double *v_out, double *p_out, double *ess_out)
{
    int n = P->n;
    double sigma2 = P->delta * P->T;
    double sigma = sqrt(sigma2);
    double z[ORC_MAXN], y[ORC_MAXN];
    double th2 = 0.0;
    for (int a = 0; a < n; ++a) th2 += theta[a] * theta[a];

    double mx = -INFINITY;
    for (int64_t i = 0; i < N; ++i) {
        orc_normals(n, P->seed, P->instance, (uint32_t)i, point, sweep, z);
        double dot = 0.0;
        for (int a = 0; a < n; ++a) {
            y[a] = x[a] + theta[a] + sigma * z[a];
            dot += (y[a] - x[a]) * theta[a];
        }
        lw[i] = -c * orc_ell(P, y, nbr) + (th2 - 2.0 * dot) / (2.0 * sigma2);
        if (lw[i] > mx) mx = lw[i];
    }
    double b[ORC_MAXN];
    for (int a = 0; a < n; ++a) b[a] = (cv_g && !P->tilt) ? -c * sigma * cv_g[a] : 0.0;
    double sw = 0.0, sw2 = 0.0, swz[ORC_MAXN], z1[ORC_MAXN], z2[ORC_MAXN];
    for (int a = 0; a < n; ++a) { swz[a] = 0.0; z1[a] = 0.0; z2[a] = 0.0; }
    for (int64_t i = 0; i < N; ++i) {
        orc_normals(n, P->seed, P->instance, (uint32_t)i, point, sweep, z);
        double w = exp(lw[i] - mx);
        sw += w;
        sw2 += w * w;
        double zb = 0.0;
        for (int a = 0; a < n; ++a) zb += z[a] * b[a];
        for (int a = 0; a < n; ++a) {
            swz[a] += w * z[a];
            z1[a] += z[a];
            z2[a] += z[a] * zb;
        }
    }
    double s = sw, S[ORC_MAXN];
    for (int a = 0; a < n; ++a) S[a] = swz[a];
    if (cv_g) {
        double lmu = -c * cv_v - mx;       /* log mu in the units of the shifted weights */
        double mu = exp(lmu);
        double bz = 0.0;
        for (int a = 0; a < n; ++a) bz += b[a] * z1[a];
        double s_cv = sw - mu * bz;
        if (fabs(lmu - log(sw / (double)N)) <= log(4.0) && s_cv > 0.0 && isfinite(s_cv)) {
            s = s_cv;
            for (int a = 0; a < n; ++a) S[a] = swz[a] - mu * (z1[a] + z2[a] - (double)N * b[a]);
        }
    }
    *v_out = -(mx + log(s / (double)N)) / c;
    for (int a = 0; a < n; ++a) {
        double ysum = (x[a] + theta[a]) * s + sigma * S[a];   /* sum_i y_i w_i */
        p_out[a] = (x[a] - ysum / s) / (P->T * P->delta * c);
    }
    *ess_out = sw * sw / sw2;
    if (P->obstacle) {   /* the value is held above the obstacle's constraint function */
        double o = obstacle_fn(P, x);
        if (o > *v_out) {
            *v_out = o;
            obstacle_grad(P, x, p_out);
        }
    }
}

int orc_sweep(const orc_problem *P, int64_t M, const double *x, const double *c,
              const double *theta, const double *nbr, const int64_t *idx, int64_t N,
              uint32_t sweep, const double *cv_v, const double *cv_p, double *v, double *p,
              double *ess)
{
    int n = P->n;
    if (n < 1 || n > ORC_MAXN || N < 1) return 1;
    int failed = 0;
#pragma omp parallel
    {
        double *lw = (double *)malloc(sizeof(double) * (size_t)N);
        double zero[ORC_MAXN];
        for (int a = 0; a < ORC_MAXN; ++a) zero[a] = 0.0;
        if (!lw) {
#pragma omp atomic write
            failed = 1;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int64_t m = 0; m < M; ++m) {
                const double *th = theta ? theta + m * n : zero;
                const double *nb = nbr ? nbr + m * 3 * P->flock_k : NULL;
                uint32_t point = (uint32_t)(idx ? idx[m] : m);
                const int use_cv = P->cv && cv_v && cv_p;
                solve_point(P, x + m * n, c[m], th, nb, N, point, sweep,
                            use_cv ? cv_p + m * n : NULL, use_cv ? cv_v[m] : 0.0, lw,
                            v + m, p + m * n, ess + m);
            }
        }
        free(lw);
    }
    return failed ? 2 : 0;
}

/* Initial iterate (Algorithm 1, "Fix"): v0 = g(x), p0 = Dg(x), c0 = Gamma(p0). */
void orc_init(const orc_problem *P, int64_t M, const double *x, const double *nbr,
              const double *psibar, double *v0, double *p0, double *c0)
{
    int n = P->n;
    for (int64_t m = 0; m < M; ++m) {
        const double *nb = nbr ? nbr + m * 3 * P->flock_k : NULL;
        double pb = psibar ? psibar[m] : 0.0;
        v0[m] = orc_ell(P, x + m * n, nb);
        orc_grad_ell(P, x + m * n, nb, p0 + m * n);
        c0[m] = orc_coef(P, x + m * n, p0 + m * n, pb);
    }
}

/* Gamma applied to M states (p rows of n), for checking a coefficient update. */
void orc_coef_batch(const orc_problem *P, int64_t M, const double *x, const double *p,
                    const double *psibar, double *c)
{
    for (int64_t m = 0; m < M; ++m)
        c[m] = orc_coef(P, x + m * P->n, p + m * P->n, psibar ? psibar[m] : 0.0);
}

/* Relative L2 change ||v1 - v0|| / ||v0|| and sup-norm change (Algorithm 1, last step). */
void orc_residual(int64_t M, const double *v_old, const double *v_new, double *rel, double *sup)
{
    double num = 0.0, den = 0.0, mx = 0.0;
    for (int64_t m = 0; m < M; ++m) {
        double dv = v_new[m] - v_old[m];
        num += dv * dv;
        den += v_old[m] * v_old[m];
        if (fabs(dv) > mx) mx = fabs(dv);
    }
    *rel = sqrt(num) / sqrt(den);
    *sup = mx;
}

/* Algorithm 1 for K sweeps starting at sweep index k0 from the state (v, p, c).
 * With tilt, sweep k uses theta = -sigma^2 c^(k) p^(k) (Eq. tilt_shift).
 * v_hist is [K+1][M] (row 0 = incoming v); p and c are updated in place;
 * resid/sup get K entries; ess gets the last sweep's ESS. */
int orc_picard(const orc_problem *P, int64_t M, const double *x, const double *nbr,
               const double *psibar, const int64_t *idx, int64_t N, int K, uint32_t k0,
               double *v_hist, double *p, double *c, double *resid, double *sup, double *ess)
{
    int n = P->n;
    double sigma2 = P->delta * P->T;
    double *theta = NULL, *p_old = NULL;
    if (P->tilt) {
        theta = (double *)malloc(sizeof(double) * (size_t)(M * n));
        if (!theta) return 2;
    }
    if (P->cv) {   /* the control variate's gradient guess is the iterate entering the sweep */
        p_old = (double *)malloc(sizeof(double) * (size_t)(M * n));
        if (!p_old) { free(theta); return 2; }
    }
    for (int k = 0; k < K; ++k) {
        double *v_old = v_hist + (int64_t)k * M;
        double *v_new = v_hist + (int64_t)(k + 1) * M;
        if (theta)
            for (int64_t m = 0; m < M; ++m)
                for (int a = 0; a < n; ++a) theta[m * n + a] = -sigma2 * c[m] * p[m * n + a];
        if (p_old) memcpy(p_old, p, sizeof(double) * (size_t)(M * n));
        int rc = orc_sweep(P, M, x, c, theta, nbr, idx, N, k0 + (uint32_t)k, v_old, p_old, v_new, p, ess);
        if (rc) { free(theta); free(p_old); return rc; }
        for (int64_t m = 0; m < M; ++m)
            c[m] = orc_coef(P, x + m * n, p + m * n, psibar ? psibar[m] : 0.0);
        orc_residual(M, v_old, v_new, resid + k, sup + k);
    }
    free(theta);
    free(p_old);
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
