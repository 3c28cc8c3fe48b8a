/*
 * hjg.h -- C ABI of libhjg.so, a GB300 (sm_103a) implementation of the HJ-Gauss
 * frozen-coefficient Picard sweep (arXiv 2605.18566).
 *
 * The library solves the viscous Hamilton-Jacobi initial-value problem
 *     v_t + H(x, Dv) = (delta/2) Lap v,   v(0, x) = l(x)            (Eq. HJ-Visc)
 * at M independent evaluation states x_m by Algorithm 1 of the paper:
 *     v^(0) = l,  c^(0) = Gamma(Dl);  for k = 0, 1, ...:
 *         freeze c^(k); phi = E_{y ~ N(x, delta t I)}[exp(-c^(k) l(y))]       (Prop. 2.1)
 *         v^(k+1) = -(1/c^(k)) log phi                                        (Lemma 2.2)
 *         Dv^(k+1) = (x - E[y e^{-c l}] / E[e^{-c l}]) / (t delta c^(k))       (Cor. 2.3)
 *         c^(k+1) = (2/delta) H(x, Dv^(k+1)) / (|Dv^(k+1)|^2 + eta)          (Eq. coeff_frozen,
 *                   |c| clipped to [c_min, c_max], sign kept                   Lemma 2.7, Rem. 2.8)
 *         residual_k = ||v^(k+1) - v^(k)||_2 / ||v^(k)||_2                     (Algorithm 1)
 * with N Monte-Carlo samples per state and sweep, estimated by the log-sum-exp form
 * (Cor. B.4), optionally under the tilted proposal theta = -delta t c^(k) Dv^(k)
 * (Eq. tilt_shift, Cor. B.6).  Viscosity is given as nu with delta = 2 nu, so samples
 * are y = x + sqrt(2 nu t) z.
 *
 * Samples are never stored.  The normals of state m in sweep k form one stream: slot q
 * is lane q % 8 of Philox4x32-10 block b = q / 8, counter (m, b_lo, k, b_hi), key
 * (seed_lo, seed_hi ^ instance).  Each word w of a block (X, Y, Z, W) gives one Box-Muller
 * pair, every bit used once: radius uniform ((w & (2^20-1)) + 0.5) 2^-20 from its low 20
 * bits, angle uniform ((w >> 20) + 0.5) 2^-12 from its high 12 bits.  Sample i, dim d is
 * slot i S + d, S = n for n <= 8 and n rounded up to a multiple of 8 above.
 *
 * Conventions for every entry point:
 *   - Return an hjg_status; no call aborts or exits.  hjg_last_error() gives a message.
 *   - "on_device" = 1: the pointer is CUDA device memory of the current device;
 *     0: ordinary (pageable or pinned) host memory.  The caller owns all buffers it
 *     passes; the context owns its internal state.
 *   - "stream" is a cudaStream_t (NULL = the context's stream, default the legacy
 *     stream).  Calls that return host results synchronise that stream.
 *   - Arrays of states are row-major [M][ld] FP32 with ld >= n.
 *   - One context must not be used from two host threads at once.
 */
#ifndef HJG_H
#define HJG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HJG_OK = 0,
    HJG_EINVAL = 1,        /* bad argument (size, pointer, option) */
    HJG_ENOMEM = 2,        /* device or host allocation failed */
    HJG_ECUDA = 3,         /* a CUDA call or kernel launch failed */
    HJG_ENONFINITE = 4,    /* results contain non-finite values (results still written) */
    HJG_ETIMEOUT = 5,      /* a bounded device wait gave up */
    HJG_ENOTCONVERGED = 6, /* tolerance not reached within the sweep budget (results written) */
    HJG_EUNSUPPORTED = 7   /* game / dimension / option not available */
} hjg_status;

/* Games (dynamics f, closed-form Hamiltonian H(x,p) = max_u min_d <p, f>, target l). */
typedef enum {
    HJG_DUBINS3 = 1,    /* Appendix D.2 relative Dubins game, unit speeds and turn rates:
                           x1' = -1 + cos x3 + u x2, x2' = sin x3 - u x1, x3' = d - u;
                           l = |(x1,x2)| - radius.  n = 3. */
    HJG_ROCKETS6 = 2,   /* two planar rockets (xA,zA,xB,zB,thA,thB), per-agent dynamics of
                           Eq. multiagent_dynamics, A evades (turn rate u), B pursues (d);
                           l = |(xA,zA) - (xB,zB)| - radius.  n = 6. */
    HJG_ROCKETS45 = 3,  /* Section 3.2: 15 agents (x_i, z_i, th_i), agent 15 evades;
                           l = min_{i<=14} |pos_i - pos_15| - radius.  n = 45. */
    HJG_FLOCK4 = 4,     /* one agent of a murmuration (Appendix D.5, per-agent reading): state
                           (p_x, p_y, p_z, psi); p' = (a cos psi, a sin psi, u_z), psi' =
                           wrap(psibar - psi) + d, |u_z|, |d| <= 1, u_z maximises, d minimises;
                           l = distance to the nearest of the agent's 7 nearest neighbours minus
                           radius.  The loaded states are the agents themselves: hjg_set_points
                           finds each one's neighbours and their circular mean heading psibar
                           and holds them frozen for the solve.  n = 4, M >= 8. */
    HJG_ROCKETS_REL3 = 5, /* Appendix D: two rockets in relative coordinates (x, z, theta),
                           Eq. ham_def: f = (a cos th + u_e x, a sin th + a - g + u_p x,
                           u_p - u_e), H = -max_{u_e} min_{u_p} <p, f>, a = speed[0], g =
                           speed[1]; l = |(x, z)| - radius.  n = 3. */
    HJG_DOUBLE_INT2 = 6,  /* Appendix D: double integrator x1' = x2, x2' = u, |u| <= 1, the
                           control minimises (Eq. dint_ham): H = p1 x2 - |p2|;
                           l = |(x1, x2)| - radius.  n = 2. */
    HJG_TEST_QUADRATIC = 100, /* H = h_sign |p|^2 / 2, l = (y-x0)^T A (y-x0)/2 + d; n <= 8 */
    HJG_TEST_ZERO_H = 101     /* H = 0 (pure heat equation), same quadratic l; n <= 8 */
} hjg_game;

typedef struct {
    int32_t game;        /* hjg_game */
    int32_t n;           /* state dimension; must equal the game's (3, 6, 45) or 1..8 for tests */
    double speed[16];    /* forward speeds per agent (ROCKETS6: [0]=A, [1]=B; ROCKETS45: a_1..a_15);
                            0 entries are read as 1 */
    double h_sign;       /* TEST_QUADRATIC only: +1 or -1 */
} hjg_dynamics;

typedef struct {
    double radius;       /* capture radius of the signed-distance target */
    double A[64];        /* quadratic test target, row-major n x n, symmetric */
    double x0[8];
    double d;
    double obstacle_radius;     /* > 0: reach-avoid tube (reading of Eq. HJI-RCBRAT-Visc) with an
                                   avoid disc of this radius about obstacle_center in the plane of
                                   state dims 0 and 1, o(y) = radius - |y_{0,1} - center| (> 0
                                   inside); the datum of every sweep is max{l, o} and after every
                                   sweep v <- max{v, o(x)}, Dv <- Do(x) where the obstacle binds.
                                   HJG_DUBINS3, HJG_ROCKETS_REL3 and HJG_DOUBLE_INT2 only
                                   (HJG_EUNSUPPORTED otherwise); 0: no obstacle */
    double obstacle_center[2];
} hjg_target;

typedef struct {
    int64_t N;           /* samples per state and sweep (1 .. 2^32 - 1, and at most
                            8 * 2^32 / S, S = n for n <= 8 and n rounded up to a multiple of
                            8 above, so that one state's stream needs at most 2^32 Philox
                            blocks; HJG_EINVAL otherwise) */
    int32_t K;           /* sweeps run by hjg_value_grad */
    int32_t tilt;        /* 1: tilted proposal theta = -delta t c Dv (Eq. tilt_shift) */
    double eps;          /* hjg_value_grad stops after the sweep whose residual < eps (0: never) */
    double eta;          /* Lemma 2.7 regulariser; < 0 selects 1e-6 */
    double c_min, c_max; /* |c| clip; <= 0 selects 1e-2/delta and 1e2/delta */
    uint64_t seed;       /* Philox key (low word, high word ^ instance) */
    uint32_t instance;
    int32_t block_threads; /* 0: tuned default; else the CTA size of one of the game's launch
                              variants (128 or 256; also 512 for the 45-D game) */
    int32_t grid_blocks;   /* 0: tuned default (persistent grid over the SMs) */
    int32_t variant;       /* 0: default / autotuned; v > 0 forces sweep launch variant v - 1 */
    uint32_t point_offset; /* global index of the first loaded state (Philox counter word 0):
                              a shard of a larger state set draws the samples it would draw
                              in the whole set; point_offset + loaded items must not exceed
                              2^32 (HJG_EINVAL) */
    int32_t tube;          /* 1: tube form v_t + min{0, H} = (delta/2) Lap v (Eq. HJ-RCBRT-Visc):
                              Gamma is built from min{0, H}, so a state that has entered the
                              target keeps a non-positive value */
    int32_t cv;            /* 1: Stein control variate in every sweep (surrogate-assisted sweep):
                              zero-mean polynomials of the normals with coefficients from the
                              iterate entering the sweep (a surrogate's prediction after
                              hjg_warm_start): mu = exp(-c v), b = -c sigma Dv (b = 0 with
                              tilt); sum w -= mu b.(sum z), sum w z -= mu (sum z + sum z (z.b)
                              - N b), kept only if mu is within a factor 4 of the sample
                              mean weight and the weight sum stays positive.  Runs its
                              own launch configuration (256-thread CTA per state); the 45-D
                              game supports it with tilt only (EUNSUPPORTED otherwise) */
    int32_t precision;     /* 0: FP32 per-sample path with FP64 combine, log, coefficient and
                              residual (default); 1: FP64 throughout -- normals, samples, target,
                              log-weights and sums in double precision (one 128-thread CTA per
                              state; games with n <= 8; not with cv: EUNSUPPORTED).  The
                              iterate is stored alike in both (v FP64, Dv and c FP32) */
    int32_t reserved[2];
} hjg_options;

typedef struct {
    int64_t M;                /* states currently loaded */
    uint32_t next_sweep;      /* global index of the next sweep (Philox counter word 3) */
    int64_t nonfinite;        /* states with non-finite v or Dv in the last call */
    int64_t clipped;          /* states whose |c| hit a clip bound in the last sweep */
    double ess_min, ess_median; /* effective sample size of the last sweep (Section 2.4) */
    double last_ms;           /* device time of the sweep kernel of the last hjg_picard_sweep that
                                 returned residuals */
    int32_t block_threads, grid_blocks; /* launch shape of that sweep */
    int32_t variant;          /* launch variant of the sweep kernel (hjg_autotune) */
} hjg_diag;

typedef struct hjg_ctx hjg_ctx;

/* Create a solver for one game instance (Eq. HJ-Visc with delta = 2 nu, evaluated at
 * t = T).  Allocates nothing on the device until points are set.  *out receives the
 * context; free it with hjg_destroy.  EINVAL on inconsistent game/n/options,
 * EUNSUPPORTED for a reserved game. */
hjg_status hjg_create(const hjg_dynamics *dyn, const hjg_target *target, double nu, double T,
                      const hjg_options *opt, hjg_ctx **out);

/* Load M evaluation states (row-major [M][ld] FP32, host or device) and form the initial
 * iterate of Algorithm 1: v^(0) = l(x), p^(0) = Dl(x) (0 where undefined), c^(0) =
 * Gamma(p^(0)).  Resets the sweep counter to 0.  Device buffers grow as needed.  With H
 * horizons set (hjg_set_horizons) the context holds M H items, item h M + m being state m
 * at horizon t_h, and every per-state array of the other calls has M H rows in that order. */
hjg_status hjg_set_points(hjg_ctx *ctx, const float *pts, int64_t M, int64_t ld, int on_device,
                          void *stream);

/* Run n_sweeps Picard sweeps (Algorithm 1 loop body) on the loaded states, continuing the
 * global sweep counter.  residual_out / supnorm_out: host arrays of n_sweeps doubles
 * (relative L2 change and sup-norm change per sweep) or NULL (then the call does not
 * synchronise); the relative change divides by ||v^(k)||_2 as IEEE arithmetic does (+inf,
 * or NaN when v^(k+1) = v^(k) = 0, if every loaded value is 0).  ENONFINITE if any state
 * produced a non-finite v or Dv. */
hjg_status hjg_picard_sweep(hjg_ctx *ctx, int n_sweeps, double *residual_out, double *supnorm_out);

/* Copy the current iterate out: v [M] FP64, p = Dv [M][ldp] FP32, c [M] FP32 (the frozen
 * coefficient for the next sweep), ess [M] FP32 (last sweep).  Any pointer may be NULL. */
hjg_status hjg_get_state(hjg_ctx *ctx, double *v, float *p, int64_t ldp, float *c, float *ess,
                         int on_device);

/* Overwrite the iterate (checkpoint resume, or a warm start): any of v, p, c may be NULL
 * (kept); next_sweep sets the global sweep counter.  Resuming with the state and counter
 * of an earlier run reproduces it bit for bit. */
hjg_status hjg_set_state(hjg_ctx *ctx, const double *v, const float *p, int64_t ldp,
                         const float *c, uint32_t next_sweep, int on_device);

/* Several horizons in one solve: the value v(t_h; x) at each of the n_horizons times
 * t_h > 0 (host array, copied) is computed for every loaded state in the same launches,
 * item h M + m using the heat kernel of width sqrt(delta t_h) (Lemma 2.2 at t = t_h) and
 * its own Philox stream (counter word 0 = point_offset + h M + m).  The items are
 * independent solves; the residual runs over all of them.  Drops the loaded states (load
 * them again); n_horizons = 0 returns to the single horizon T of hjg_create.  EINVAL for a
 * non-positive or non-finite time. */
hjg_status hjg_set_horizons(hjg_ctx *ctx, const double *t, int n_horizons);

/* Warm start (a surrogate's prediction in place of Algorithm 1's initial iterate): set
 * p^(0) = p0 [M][ldp] FP32 and, if v0 is not NULL, v^(0) = v0 [M] FP64, then recompute the
 * frozen coefficient c^(0) = Gamma(p0) (Eq. coeff_frozen with Lemma 2.7 and Remark 2.8) on
 * the device.  With opt.tilt the first sweep is then drawn from the tilted proposal around
 * theta = -delta t c^(0) p0 (Eq. tilt_shift).  Synchronises the context's stream. */
hjg_status hjg_warm_start(hjg_ctx *ctx, const double *v0, const float *p0, int64_t ldp, int on_device);

/* Warm start from a learned correction to Algorithm 1's initial iterate ("Fix" step:
 * v^(0) = l, p^(0) = Dl): v = l(x_m) + d[m][0], Dv_j = D_j l(x_m) + d[m][1 + j], then
 * c = Gamma(Dv) (Eq. coeff_frozen, Lemma 2.7, Remark 2.8), l and Dl evaluated in FP64 per
 * state.  d is a DEVICE array [M][ldd] FP32 (ldd >= n + 1; the layout of a surrogate's
 * output rows (v, Dv) trained on hjg_get_state_delta targets).  Synchronises the context's
 * stream.  EINVAL for ldd < n + 1 or a NULL d. */
hjg_status hjg_warm_start_delta(hjg_ctx *ctx, const float *d, int64_t ldd);

/* The current iterate minus the initial one, per loaded state: out[m][0] = v - l(x_m),
 * out[m][1 + j] = Dv_j - D_j l(x_m) (FP64 difference rounded to FP32), out a DEVICE array
 * [M][ldo], ldo >= n + 1: the targets of a surrogate that learns the correction the Picard
 * iteration makes to its initial iterate.  Synchronises the context's stream. */
hjg_status hjg_get_state_delta(hjg_ctx *ctx, float *out, int64_t ldo);

/* The invariant frame of the 45-D game for a surrogate network (Section 3.2's game is
 * invariant under a common translation, under a common rotation of positions and headings,
 * and -- with equal pursuer speeds -- under permutations of the pursuers; the paper has no
 * network).  Per loaded state the pursuers are ordered by distance to the evader (ties by
 * index) and described in the evader's frame: r_k = R(-theta_e)(p_i - p_e), phi_k =
 * theta_i - theta_e.
 *   hjg_frame_features: out [M][ldo] (ldo >= 56) = (r_k, cos phi_k, sin phi_k) for k = 0..13.
 *   hjg_frame_targets:  out [M][ldo] (ldo >= 43) = (v - l, then per ordered pursuer
 *                       R(-theta_e) (Dv - Dl)_{p_i} and (Dv - Dl)_{theta_i}) of the current
 *                       iterate: the training targets.
 *   hjg_warm_start_frame: from a prediction pred [M][ldp] (ldp >= 43) in that layout, the
 *                       iterate v = l + dv, Dv = Dl + the correction mapped back by the chain
 *                       rule (the evader's position part from translation invariance, its
 *                       heading part from the frame's rotation), c = Gamma(Dv) (Eq.
 *                       coeff_frozen).  With positions_only != 0 only the position rows of
 *                       Dv take the correction and the 15 heading rows keep Dl's (zero:
 *                       l does not depend on the headings).  The sweep sees the iterate only
 *                       through c, and the game's Hamiltonian subtracts |p_theta| for every
 *                       pursuer heading, so small errors of a network in those rows lower H
 *                       and can flip the sign of c where Dl gets it right; measured on the
 *                       paper's wide 45-D domain, positions_only is the form that helps.
 * All arrays are DEVICE memory; each call synchronises the context's stream.
 * EUNSUPPORTED for another game, unequal pursuer speeds or several horizons. */
hjg_status hjg_frame_features(hjg_ctx *ctx, float *out, int64_t ldo);
hjg_status hjg_frame_targets(hjg_ctx *ctx, float *out, int64_t ldo);
hjg_status hjg_warm_start_frame(hjg_ctx *ctx, const float *pred, int64_t ldp, int positions_only);

/* Per-sweep parts of the residual of the last hjg_picard_sweep call over the loaded
 * states: out [n_sweeps][3] = (sum (v^(k+1)-v^(k))^2, sum (v^(k))^2, max |v^(k+1)-v^(k)|),
 * FP64, host.  Shards of one state set combine these (sum, sum, max) to the global
 * relative residual sqrt(sum0)/sqrt(sum1) of Algorithm 1. */
hjg_status hjg_get_residual_parts(hjg_ctx *ctx, double *out);

/* Conservative safety certificate (Cor. 2.9) of the current iterate, after at least one
 * sweep: per state the band half-width
 *     E_m = e0 + q/(1-q) ||v^(K) - v^(K-1)||_inf + sqrt(2 log(2/delta_p)) se_m
 * (e0 >= 0: the caller's bound on the quasi-linearisation defect and the viscosity error;
 * the second term is the a-posteriori iteration bound of Theorem 2.8 with contraction factor
 * 0 <= q < 1 and the last sweep's sup-norm change; se_m = sqrt(1/ESS_m - 1/N) / |c_m| is the
 * delta-method Monte-Carlo standard error of v_m in the last sweep, c_m the coefficient that
 * sweep used, and the factor a sub-Gaussian two-sided quantile for failure probability
 * 0 < delta_p < 1).  label_out [M] int8: +1 SAFE (v > E_m), -1 UNSAFE (v < -E_m), 0
 * UNDETERMINED, also wherever the last sweep's ESS is below ess_min >= 0 (collapsed
 * weights, Section 2.4: the standard error is then not trustworthy); band_out [M] FP32 = E_m; se_out [M] FP32 = se_m; counts_out [3] (host) =
 * (SAFE, UNSAFE, UNDETERMINED) counts.  Every output may be NULL; on_device selects
 * device or host pointers for the arrays.  EINVAL for parameters outside their ranges or
 * when no sweep has run since the iterate was loaded or replaced.  Synchronises the
 * context's stream. */
hjg_status hjg_certify(hjg_ctx *ctx, double e0, double q, double delta_p, double ess_min, int8_t *label_out,
                       float *band_out, float *se_out, int64_t *counts_out, int on_device);

/* v^(k) history of the last hjg_picard_sweep call: rows 0..n_sweeps, row 0 = the
 * incoming v.  out is [(n_sweeps+1)][M] FP64. */
hjg_status hjg_get_history(hjg_ctx *ctx, double *out, int on_device);

/* hjg_set_points + up to opt.K sweeps (stopping early once residual < opt.eps > 0) +
 * copy-out: v_out [M] FP64, grad_out [M][ldg] FP32, residual_out [K] FP64 (host; entries
 * after an early stop are set to NaN).  Host or device buffers per on_device. */
hjg_status hjg_value_grad(hjg_ctx *ctx, const float *pts, int64_t M, int64_t ld, int on_device,
                          double *v_out, float *grad_out, int64_t ldg, double *residual_out,
                          void *stream);

hjg_status hjg_get_diagnostics(hjg_ctx *ctx, hjg_diag *out);

/* Autotuner: time one sweep of every launch variant of the sweep kernel (kernel kind, CTA
 * size x register budget, sampler pipelining, with the persistent grid that fills the SMs;
 * one warm-up launch, then the faster of two timed launches) on the first
 * min(M, max_states) loaded states (max_states <= 0: all), keep the fastest for this
 * context and report its index, CTA size and time.  Works on scratch copies: the iterate
 * and the sweep counter are unchanged.  Allocates and frees device scratch; synchronises
 * the context's stream.  EINVAL when no states are loaded.  An explicit
 * opt.block_threads is cleared by tuning. */
hjg_status hjg_autotune(hjg_ctx *ctx, int64_t max_states, int32_t *variant_out, int32_t *threads_out,
                        double *best_ms_out);
hjg_status hjg_set_stream(hjg_ctx *ctx, void *stream);
void hjg_destroy(hjg_ctx *ctx);
const char *hjg_last_error(const hjg_ctx *ctx);
const char *hjg_status_string(hjg_status s);

/* One-shot solve that allocates no device memory (the paper has no counterpart; this
 * is a deployment variant of hjg_value_grad).  For callers that must not allocate once
 * running: hard real-time control loops, processes whose device memory belongs to
 * another runtime's allocator, services that reserve everything at start-up.  Runs the
 * initial iterate, opt->K sweeps (no early stop) and the residuals for the M states at
 * pts ([M][ld] FP32, device) and writes v_out [M] FP64, grad_out [M][ldg] FP32 (also used
 * as the Dv iterate) and, if not NULL, residual_out [2*K] FP64 (relative L2 and sup-norm
 * change of each sweep, interleaved) -- all device pointers, all owned by the caller.
 * Its other working memory is one fixed 16 MiB device array inside the library, which
 * every GPU that loads the library holds until the process exits; the call needs
 * (8*K + 16)*M bytes of it plus a little alignment slack and returns EINVAL beyond that
 * (e.g. M <= 95,000 states at K = 20).  No cudaMalloc, no cudaFree, no allocating library
 * routine.  The first call on each device looks up that array's device address (with
 * the device current), so make it before any stream capture.  Asynchronous on `stream`;
 * calls share the array, so calls that overlap on the GPU race and must be serialised by
 * the caller.  Default launch variant 0 (opt->variant > 0 selects another; otherwise
 * opt->block_threads > 0 selects the first variant of that CTA size, as in hjg_create, and
 * EINVAL if the game has none).  The call never synchronises, so it cannot see the
 * sweep's non-finite counter and never returns HJG_ENONFINITE: a state whose v or Dv is
 * not finite shows up as NaN or inf in v_out / grad_out, which the caller checks.  Every game
 * but the flock (HJG_FLOCK4 returns EINVAL: its neighbour data is per-agent storage), with
 * the options of hjg_create (tilt, tube, obstacle, cv, precision, point_offset); every
 * argument is checked, and a refusal returned, before any device work. */
hjg_status hjg_value_grad_noalloc(const hjg_dynamics *dyn, const hjg_target *target, double nu,
                                  double T, const hjg_options *opt, const float *pts, int64_t M,
                                  int64_t ld, double *v_out, float *grad_out, int64_t ldg,
                                  double *residual_out, void *stream);

/* ---- building blocks, exposed for bit-level tests ------------------------------ */

/* Philox4x32-10 blocks on the device: ctr [count][4], key [count][2], out [count][4]
 * uint32, all device pointers. */
hjg_status hjg_philox_blocks(const uint32_t *ctr, const uint32_t *key, uint32_t *out,
                             int64_t count, void *stream);

/* The FP32 standard normals the sweep consumes for state `point`, sweep `sweep`, samples
 * 0..n_samples-1 (the stream layout at the top of this header): out is device
 * [n_samples][n] FP32. */
hjg_status hjg_sample_normals(int n, uint64_t seed, uint32_t instance, uint32_t point,
                              uint32_t sweep, int64_t n_samples, float *out, void *stream);

/* Neighbour structure of a flock (the HJG_FLOCK4 game): for agent states [M][ld] FP32
 * (ld >= 4; components 0..2 position, 3 heading), idx_out [M][k] int32 receives the k
 * nearest other agents (exact, squared FP32 distance, ties by index) and psibar_out [M]
 * FP32 (or NULL) the circular mean atan2(sum sin psi_j, sum cos psi_j) of their headings.
 * A NaN distance (a non-finite position) never qualifies: where fewer than k other agents
 * remain, the empty slots hold -1 and psibar is NaN (a solve then reports that agent as
 * non-finite).  k must be 7; device pointers; asynchronous on stream. */
hjg_status hjg_flock_neighbours(const float *states, int64_t M, int64_t ld, int k, int32_t *idx_out,
                                float *psibar_out, void *stream);

/* Event flags of hjg_topology (the threshold rules of the murmuration study's phase-
 * transition markers, recorded at the later of two consecutive slices). */
enum {
    HJG_EVENT_VACUOLE = 1,        /* chi dropped: chi_h - chi_{h-1} < -0.5 */
    HJG_EVENT_CORDON = 2,         /* beta_1 >= 1 and beta_1 was 0 at the previous slice */
    HJG_EVENT_FRAGMENTATION = 4   /* n_comp grew */
};

/* Topology of the zero sublevel set {v <= 0} on H 2-D value slices (Appendix D, phase-
 * transition markers): v [H][m][m] FP64 on the device (e.g. a grid of states solved at H
 * horizons).  Each slice is first smoothed by a separable Gaussian of smooth_cells grid
 * cells (weights exp(-k^2/(2 s^2)), |k| <= int(4 s + 0.5), normalised, half-sample-symmetric
 * reflection at the border; 0 skips it; the radius must stay below m), then its set cells
 * (4-connected) and complement cells (8-connected) are labelled.  markers_out [H][3] int32
 * (host) = (n_comp, beta_1 = complement components not touching the border, chi = n_comp -
 * beta_1); events_out [H] int32 (host, or NULL) = HJG_EVENT_* flags against the previous
 * slice (0 for the first); smoothed_out [H][m][m] FP64 and labels_out [H][m][m] int32 (root
 * cell index of each cell's component; host or device, or NULL).  Temporaries are stream-
 * ordered allocations; synchronises the stream.  EINVAL for bad sizes, ETIMEOUT if a
 * union-find walk hit its iteration bound. */
hjg_status hjg_topology(const double *v, int H, int m, double smooth_cells, double *smoothed_out,
                        int32_t *markers_out, int32_t *events_out, int32_t *labels_out, void *stream);

/* ---- surrogate network (BF16 tensor cores, trained on the sweep's own tuples) ---- */

/* An MLP n_in -> width -> width -> width -> n_out with SiLU activations (the surrogate of
 * the learned warm start; the paper has no counterpart): BF16 weights and activations,
 * FP32 accumulation on the tensor cores, FP32 master weights, Adam.  For the value
 * surrogate n_out = n + 1: output 0 predicts v, outputs 1..n predict Dv.  Training loss:
 * (o_0 - v)^2 + mean_j (o_j - Dv_j)^2, averaged over the batch.  Weights start uniform in
 * +-sqrt(6/(fan_in + fan_out)) from a hash of `seed`, biases at zero.  width must be a
 * multiple of 16 and at least n_in and n_out rounded up to 16.  SiLU is evaluated as
 * z (1 + tanh(z / 2)) / 2 with the hardware tanh approximation (relative error about
 * 2^-11, below the BF16 rounding of the activations).  With width 256 and n_in, n_out at
 * most 64 the training calls run the fused three-kernel step, whose kernels are launched as
 * programmatic dependents of the work before them in the stream (each waits for that work
 * before its first global read).  Device pointers throughout; the context's stream
 * (hjg_mlp_set_stream) orders every call. */
typedef struct hjg_mlp hjg_mlp;

hjg_status hjg_mlp_create(int n_in, int n_out, int width, uint64_t seed, hjg_mlp **out);
void hjg_mlp_destroy(hjg_mlp *m);
hjg_status hjg_mlp_set_stream(hjg_mlp *m, void *stream);
/* Number of FP32 parameters: [W1 b1 W2 b2 W3 b3 W4 b4], W_l [out_pad][in_pad] row-major
 * (inputs and outputs padded to multiples of 16 with zero weights). */
int64_t hjg_mlp_num_params(const hjg_mlp *m);
hjg_status hjg_mlp_get_params(hjg_mlp *m, float *out, int on_device);
/* Load parameters (resets Adam's moments and step count). */
hjg_status hjg_mlp_set_params(hjg_mlp *m, const float *in, int on_device);
/* out [B][ldout] (n_out used) = MLP(x [B][ldx] (n_in used)). */
hjg_status hjg_mlp_forward(hjg_mlp *m, const float *x, int64_t ldx, int64_t B, float *out, int64_t ldout);
/* Loss (host, FP64, may be NULL) and gradients w.r.t. all parameters (host grad_out of
 * hjg_mlp_num_params floats, may be NULL) on one batch; parameters unchanged. */
hjg_status hjg_mlp_gradients(hjg_mlp *m, const float *x, int64_t ldx, const float *y, int64_t ldy,
                             int64_t B, double *loss_out, float *grad_out);
/* Gradient of output j with respect to the inputs (chain rule through the network, BF16
 * operands, FP32 accumulation): gx [B][ldg] (n_in used).  For the value surrogate, j = 0
 * gives the derivative of the predicted value, a gradient field consistent with it. */
hjg_status hjg_mlp_input_grad(hjg_mlp *m, const float *x, int64_t ldx, int64_t B, int j, float *gx,
                              int64_t ldg);
/* Feature standardisation of the network (a training convenience; the paper's network is
 * not specified to this level): inputs enter as (x_i - shift_i) mul_i and the network's
 * outputs o_j are reported as o_j mul_j + shift_j, so that features and targets of very
 * different sizes (positions of +-100 next to headings) train alike.  The default is the
 * identity.  hjg_mlp_fit_scaling sets shift = mean and mul = 1/std for the inputs x [B][ldx]
 * and shift = mean, mul = std for the targets y [B][ldy] (device, FP64 sums; a constant
 * column gets std 1); the loss of hjg_mlp_gradients / hjg_mlp_train_step is then measured on
 * standardised targets.  get/set exchange the four arrays as one host buffer
 * [in_shift n_in | in_mul n_in | out_shift n_out | out_mul n_out] (set: EINVAL unless every
 * mul > 0 and every shift finite). */
hjg_status hjg_mlp_fit_scaling(hjg_mlp *m, const float *x, int64_t ldx, const float *y, int64_t ldy, int64_t B);
hjg_status hjg_mlp_get_scaling(hjg_mlp *m, float *out);
hjg_status hjg_mlp_set_scaling(hjg_mlp *m, const float *in);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on one batch;
 * loss_out (host) may be NULL (then the call does not synchronise). */
hjg_status hjg_mlp_train_step(hjg_mlp *m, const float *x, int64_t ldx, const float *y, int64_t ldy,
                              int64_t B, float lr, double *loss_out);

/* Training loop in the library: Adam steps over the contiguous minibatches [b0, b0 + batch)
 * of the n rows of x [n][ldx] and y [n][ldy] (device; shuffle the rows beforehand), b0 =
 * 0, batch, 2 batch, ... while b0 + batch <= n (one minibatch of all n rows when n <
 * batch), for `epochs` passes, the learning rate decaying geometrically from lr at the first
 * step to lr_final at the last.  With standardize != 0 the feature standardisation is first
 * fitted to (x, y) (hjg_mlp_fit_scaling).  hist (host, `epochs` doubles, may be NULL)
 * receives each epoch's loss on its last minibatch; the call synchronises once per epoch
 * when hist is given, else not at all.  EINVAL for epochs < 1, batch < 1, lr <= 0 or
 * lr_final <= 0. */
hjg_status hjg_mlp_fit(hjg_mlp *m, const float *x, int64_t ldx, const float *y, int64_t ldy, int64_t n,
                       int epochs, int64_t batch, float lr, float lr_final, int standardize, double *hist);

/* The surrogate's GEMM on its own (the tensor-core kernel behind hjg_mlp_*):
 * C(m, n) = sum_k A(m, k) B(k, n) with A(m, k) = A[m*sam + k*sak] and B(k, n) =
 * B[k*sbk + n*sbn] in BF16, C [M][ldc] FP32, device pointers.  timed_out (host, may be
 * NULL) receives 1 if a bounded wait of the kernel gave up (then ETIMEOUT); passing it
 * synchronises the stream. */
hjg_status hjg_gemm_bf16(const void *A, int64_t sam, int64_t sak, const void *B, int64_t sbk, int64_t sbn,
                         int M, int N, int K, float *C, int64_t ldc, int *timed_out, void *stream);

/* ---- batches: many instances, one CUDA-graph launch ------------------------------- */

/* A batch advances several instances (contexts, possibly of different games, dimensions
 * and state counts) by the same number of Picard sweeps in one CUDA-graph launch: each
 * instance's fused sweep kernel and residual kernel run on their own branch of the graph,
 * concurrently on the SMs.  This is Algorithm 1 applied to each instance independently
 * (instances share nothing).  The contexts stay owned by the caller and must outlive the
 * batch; their points must be loaded (hjg_set_points) before each run. */
typedef struct hjg_batch hjg_batch;

hjg_status hjg_batch_create(hjg_batch **out);
/* Add an instance; EINVAL if it is already in the batch. */
hjg_status hjg_batch_add(hjg_batch *b, hjg_ctx *ctx);
/* Run n_sweeps sweeps of every instance in one graph launch on `stream` (NULL: a private
 * stream, and the call synchronises).  The graph is captured on each call and the
 * instantiated graph updated in place (the sweep counters advance between calls).
 * residual_out: host [instances][n_sweeps] relative L2 residuals, or NULL (then, with a
 * caller stream, the call is asynchronous).  device_ms: device time of the graph launch,
 * or NULL.  ENONFINITE if an instance produced non-finite values. */
hjg_status hjg_batch_run(hjg_batch *b, int n_sweeps, double *residual_out, void *stream,
                         double *device_ms);
void hjg_batch_destroy(hjg_batch *b);
const char *hjg_batch_last_error(const hjg_batch *b);

/* Self-test of the bounded device waits (no counterpart in the paper): a one-thread kernel
 * waits on an mbarrier with the same wait loop the tensor-core GEMM uses, limited to
 * `limit` polls; with arrive = 0 nothing arrives, the wait gives up and the call returns
 * HJG_ETIMEOUT with the device still usable; with arrive = 1 it returns HJG_OK.
 * Synchronises the stream. */
hjg_status hjg_selftest_bounded_wait(int arrive, int64_t limit, void *stream);

/* ---- pipe micro-benchmarks (roofline denominators) ------------------------------ */

/* Instruction classes timed by hjg_microbench: FP32 FMA, the MUFU transcendental
 * approximations (ex2, lg2, sin, cos, sqrt), whole Philox4x32-10 blocks, whole
 * Box-Muller normals as the sweep draws them, 32x32->64-bit integer multiplies, their low
 * and high halves alone, and Philox blocks whose products are formed as separate high and
 * low multiplies. */
enum {
    HJG_MB_FFMA = 1, HJG_MB_EX2 = 2, HJG_MB_LG2 = 3, HJG_MB_SIN = 4, HJG_MB_COS = 5,
    HJG_MB_SQRT = 6, HJG_MB_PHILOX = 7, HJG_MB_NORMALS = 8, HJG_MB_IMAD_WIDE = 9,
    HJG_MB_IMUL_LO = 10, HJG_MB_IMUL_HI = 11, HJG_MB_PHILOX_SPLIT = 12, HJG_MB_PHILOX_MIXED = 13
};

/* Run one saturating launch (8 CTAs of 256 threads per SM, 8 independent chains per
 * thread, `iters` steps per chain) of instruction class `op` on the current device and
 * return its throughput in operations (or blocks, or normals) per second, and the launch
 * time in ms.  Allocates (and frees) a 1 KB sink; synchronises the device; EINVAL for an
 * unknown op. */
hjg_status hjg_microbench(int op, int64_t iters, double *ops_per_s, double *ms);

#ifdef __cplusplus
}
#endif
#endif /* HJG_H */
