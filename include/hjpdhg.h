/*
 * hjpdhg.h -- C ABI of the batched Lax / PDHG Hamilton-Jacobi solver (sm_103a).
 *
 * The library computes, for every query point (x, t), the value
 *     phi(x, t) ~ max_{p_1..p_N} min_{x_0..x_{N-1}}
 *         g(x_0) + sum_{j=1}^N <p_j, x_j - x_{j-1}> - delta sum_{j=1}^N H(x_j, p_j)
 * (Lin, Chow, Osher 2018, Eq. (disclaxBE): the Lax formula with a backward Euler
 * discretisation of the dynamics, x_N = x, delta = t / N), by running Algorithm 1
 * (PDHG / Chambolle-Pock with the updates of Section 5.3 and the loop of Appendix
 * Algorithm A.1) independently on every point, and returns the trajectory
 * x_0..x_N and costate p_1..p_N it converged to (Section 5.4).
 *
 * Conventions for every entry point:
 *  - Plain C types only.  "device" pointers are CUDA device (or managed) memory
 *    owned by the caller; "host" pointers are ordinary host memory read during
 *    the call.  The library never takes ownership of caller memory.
 *  - Calls are asynchronous on `stream` (a cudaStream_t passed as void*, NULL =
 *    the legacy default stream).  The return value reports argument errors and
 *    launch errors only; the per-point outcome is written to `status[]`.
 *  - Arrays are row-major and densely packed.  Floating-point inputs and the
 *    value output are double; the iterate arrays (trajectories, warm starts)
 *    use the precision selected in the options (float for HJ_PREC_FP32,
 *    double for HJ_PREC_FP64).
 *  - No entry point synchronises the device.
 */
#ifndef HJPDHG_H
#define HJPDHG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
typedef enum {
  HJ_OK = 0,
  HJ_ERR_INVALID_ARG = 1, /* null pointer, size out of range, non-finite parameter */
  HJ_ERR_UNSUPPORTED = 2, /* valid request this build has no kernel for (d, N too large) */
  HJ_ERR_STEP_SIZE = 3,   /* sigma*tau*||D||^2 >= 1 with ||D||^2 < 4 (Section 3.2 step rule) */
  HJ_ERR_CUDA = 4,        /* a CUDA runtime call or kernel launch failed */
  HJ_ERR_OOM = 5          /* device allocation inside hj_problem_create failed */
} hj_status;

/* Hamiltonian families, all with L = |u|^2/2 and H = max_u {<f,p> - L}
 * (Section 2, backward-in-time control convention).                       */
enum {
  /* H = |p|^2/2.  dyn: none (n_dyn = 0).                                       */
  HJ_FAMILY_QUADRATIC = 0,
  /* 12-D quadcopter of Section 6.4 with thrust measured from hover and an
   * additive disturbance input: H = <p, f0(x)> + |B(x)^T p|^2/2 + eps |p|^2/2.
   * dyn (host, 4 doubles): m, a_h (hover thrust per unit mass), g_z, eps.  d = 12. */
  HJ_FAMILY_QUADCOPTER = 1,
  /* H = <p, tanh(A x)> + |p|^2/2.  dyn (host): A, d*d doubles, row-major.       */
  HJ_FAMILY_TANH_DRIFT = 2,
  /* Eikonal equation of Section 6.1, phi_t + s c(x)|grad phi|_2 = 0: H = s c(x)|p|_2
   * with the speed c(x) = c0 + c1 exp(-c2 |x - x_b|^2) (the paper's bump: c0 = 1,
   * c1 = 3, c2 = 4, x_b = (1, 1, 0, ...)).  dyn (host, 4 + d doubles):
   * s (+1 or -1), c0 > 0, c1 >= 0, c2 >= 0, x_b[d].  d = 1..4096.  The dual step
   * is the shrink_2 operator.  s = -1 is solved as in Section 6.1: phi = -psi
   * with psi the s = +1 solution for the initial data -g (concave; its x_0
   * proximal map needs tau W_i^2 < 1, HJ_ERR_STEP_SIZE otherwise), and V and
   * the returned p are those of phi.  Lax form only.  With 4 + 2d doubles the
   * last d are a bump velocity v_b: H(x, p, s) = c(x - s v_b)|p|_2 at the node
   * times s_j = j delta (Section 6.1's state-and-time-dependent example, v_b =
   * (-1, 1)); a nonzero v_b runs in the register kernel only (d in {2, 10}),
   * backward Euler.                                                         */
  HJ_FAMILY_EIKONAL = 3,
  /* Difference-of-norms differential game of Section 6.2 (Algorithm 3):
   * state z = (x, y), x = z[0..d1) the minimising player, y = z[d1..d) the
   * maximising one, costates (p, q) stored in that order; H(z, p, q) =
   * c1(z)|p|_2 - c2(z)|q|_2 with c1(z) = c0 + a exp(-b |z - z_b|^2) and its mirror
   * c2(z) = c1(-z).  dyn (host, 4 + d doubles): d1 (integer, 1..d-1), c0 > 0,
   * a >= 0, b >= 0, z_b[d].  d = 2 or 7 (the paper's cases; other d are
   * HJ_ERR_UNSUPPORTED at solve time).  V = g(z_0) + sum <p_j, dx_j>
   * - sum <q_j, dy_j> - delta sum H; g is convex in both players, so the
   * maximiser's y_0 step is the ascent prox of g (needs tau W_i^2 < 1 on the
   * maximiser's coordinates, HJ_ERR_STEP_SIZE otherwise).  Lax form, one
   * gradient step per primal block (inner_steps = 1), no gradient entry point. */
  HJ_FAMILY_GAME_NORMS = 4
};

/* Iterate precision.  With FP32 iterates the stopping test's squared
 * increments (each lane's or thread's partial in FP32, summed over its warp in
 * FP32) are accumulated over the point in FP64 and compared with tol in FP64,
 * the value's terms are summed in FP64, and the optional residual (kkt) is
 * evaluated in FP64, except the quadcopter's, which is evaluated in FP32 (its
 * error stays below the FP32 iterates' own rounding: see hj_kkt_residual);
 * FP64 runs everything in double.                                           */
enum { HJ_PREC_FP32 = 0, HJ_PREC_FP64 = 1 };

/* Saddle problem solved (hj_solver_opts.formulation).
 *   HJ_FORM_LAX   Algorithm 1, Eq. (disclaxBE): unknowns x_0..x_{N-1}, p_1..p_N.
 *   HJ_FORM_HOPF  Algorithm 2, Eq. (dischopf): x_0 eliminated through the convex
 *                 conjugate, min_{x_0} g(x_0) - <p_1, x_0> = -g*(p_1) with
 *                 g*(p) = <p, c> + 1/2 sum_i p_i^2 / W_i^2 (every W_i nonzero);
 *                 the j = 1 dual step is the joint prox of g* and delta H (the
 *                 appendix's Hopf tutorial algorithm).  For convex g both have
 *                 the same saddle value.                                        */
enum { HJ_FORM_LAX = 0, HJ_FORM_HOPF = 1 };

/* Time discretisation of the Lax form (hj_solver_opts.scheme).  With the
 * costate of interval [s_{j-1}, s_j] stored at node j (traj_p[b][j], j = 1..N),
 * every scheme solves
 *   max_p min_x g(x_0) + sum_{j=1}^N <p_j, x_j - x_{j-1}>
 *               - delta sum_{j=1}^N (wR H(x_j, p_j) + wL H(x_{j-1}, p_j))
 * with weights on the two ends of each interval:
 *   HJ_SCHEME_BE    (wR, wL) = (1, 0): backward Euler, Eq. (disclaxBE).
 *   HJ_SCHEME_FE    (0, 1): forward Euler, Eq. (disclaxFE); its costate p_{j-1}
 *                   (the paper's index) is stored at node j.
 *   HJ_SCHEME_TRAP  (1/2, 1/2): the average of the two Euler forms, which the
 *                   paper proposes for higher accuracy (end of Section 5 and
 *                   Section 7); second order in delta where both are first.
 * The PDHG steps are Algorithm 1's with H at x^k: the dual step is the prox of
 * sigma delta (wR H(x_j, .) + wL H(x_{j-1}, .)); x_j (1 <= j < N) takes one
 * gradient step on -delta (wR H(x_j, p_j) + wL H(x_j, p_{j+1})); x_0, on which
 * both g and (for wL > 0) H act, takes one gradient step on -delta wL H(x_0, p_1)
 * followed by the exact prox of g.  For the game (HJ_FAMILY_GAME_NORMS) the
 * same weights apply to both players in Algorithm 3's order: the y-block's H
 * terms, y_0's included, are taken at (x^{k+1}, y^k).  FE and TRAP run with
 * the Lax form and inner_steps = 1 in every kernel but the tiled FP32 one:
 * the register-resident kernel (quadcopter, tanh drift d in {2, 4}, eikonal
 * d in {2, 10}, the game d in {2, 7}; N <= 128 in FP64), the shared-memory
 * tanh-drift kernel (any other d, and d = 4 with N > 128 in FP64) and the
 * coordinate-parallel eikonal kernel (any other d, static bump); the quadratic
 * family, whose H does not depend on x, has the same problem under every
 * scheme.  Other cases (the quadcopter or the game in FP64 with N > 128, a
 * moving bump) return HJ_ERR_UNSUPPORTED.                                    */
enum { HJ_SCHEME_BE = 0, HJ_SCHEME_FE = 1, HJ_SCHEME_TRAP = 2 };

/* Per-point outcome written to status[].  HJ_POINT_INVALID marks a point whose
 * own N was outside the range of the kernel it was routed to (ragged batches:
 * N[b] outside 1..256); such a point is not iterated.  HJ_POINT_TIMEOUT marks a
 * point the launch did not solve because its budget (hj_solver_opts
 * time_budget_ms, iter_budget) had run out when the point came up: it is not
 * iterated, iters = 0, V = NaN, and its trajectory rows are not written.      */
enum { HJ_POINT_CONVERGED = 0, HJ_POINT_MAX_ITER = 1, HJ_POINT_NONFINITE = 2,
       HJ_POINT_INVALID = 3, HJ_POINT_VALUE_STOP = 4, HJ_POINT_TIMEOUT = 5 };

typedef struct hj_problem_s* hj_problem;

/* Create a problem: Hamiltonian family + terminal cost g(x) = 1/2 sum_i W_i^2 (x_i - c_i)^2
 * (a constant added to g adds the same constant to V: the caller adds it).
 *   out      (host) receives the handle; set to NULL on error.
 *   family   HJ_FAMILY_*;  d state dimension (1..128; 12 for the quadcopter;
 *            1..4096 for the eikonal family).
 *   dyn      (host) n_dyn doubles, layout per family above (may be NULL if n_dyn = 0).
 *   W, c     (host) d doubles each.
 * Copies every parameter to device memory owned by the handle (allocates on the
 * current device; the handle must be used on that device).
 * Errors: HJ_ERR_INVALID_ARG (bad family, d, n_dyn, non-finite values),
 *         HJ_ERR_OOM, HJ_ERR_CUDA.                                          */
hj_status hj_problem_create(hj_problem* out, int32_t family, int32_t d,
                            const double* dyn, int64_t n_dyn,
                            const double* W, const double* c);

/* Destroy a handle (NULL is accepted).  Synchronises the handle's device
 * before freeing, so pending solves on the handle complete first.          */
hj_status hj_problem_destroy(hj_problem prob);

/* Solver options (host struct, read during the call).
 *   sigma, tau   PDHG step sizes, sigma * tau < 1/4 (||D||^2 < 4, Appendix A.1).
 *   theta        over-relaxation, z = x^{k+1} + theta (x^{k+1} - x^k), in [0, 1].
 *   tol          stop when |x^{k+1}-x^k|_2^2 < tol and |p^{k+1}-p^k|_2^2 < tol
 *                (squared norms over the whole stacked vectors, Section 6).
 *   max_iter     iteration cap (>= 1).
 *   check_every  the stopping test runs after every check_every-th iteration
 *                and after iteration max_iter.
 *   inner_steps  gradient steps per x-update (1 = Section 5.3's single step;
 *                more approach the argmin of Appendix Algorithm A.1).
 *   precision    HJ_PREC_FP32 or HJ_PREC_FP64.
 *   seed         seed of the counter-based initial guess.
 *   init_radius  x_j^0 = x + r u, p_j^0 = r u', u, u' in [-1, 1)^d (Section 6).
 *   point_offset global index of the batch's first point: the initial guess of
 *                point b depends on (seed, point_offset + b) only, so a batch
 *                split into slices reproduces the unsplit run.
 *   formulation  HJ_FORM_LAX (0, the default of a zeroed struct) or HJ_FORM_HOPF;
 *                Hopf needs every W_i nonzero (HJ_ERR_INVALID_ARG otherwise).
 *   scheme       HJ_SCHEME_BE (0, the default), HJ_SCHEME_FE or HJ_SCHEME_TRAP
 *                (Lax form only).
 *   value_tol    0 (the default) or > 0: the value test of Section 6.2's slow
 *                points as well: at a test, a point whose fval moved by less
 *                than value_tol (absolute) since the previous test stops with
 *                status HJ_POINT_VALUE_STOP.  Backward-Euler Lax form in the
 *                register-resident kernel only (HJ_ERR_UNSUPPORTED otherwise).
 *   time_budget_ms, iter_budget
 *                budget of one kernel launch (0, the default: none): the
 *                milliseconds since the launch's first point was drawn (the
 *                device's global timer), and the iterations of the points it
 *                has finished.  Once either is used up, every point drawn after
 *                that is marked HJ_POINT_TIMEOUT instead of solved, so the launch
 *                drains its batch and ends; points already being solved finish
 *                (each is bounded by max_iter).  A ragged plan applies it to each
 *                bucket's launch.  The call itself stays asynchronous: the
 *                outcome is in status[].                                      */
typedef struct {
  double sigma, tau, theta, tol;
  int32_t max_iter, check_every, inner_steps, precision;
  uint64_t seed;
  double init_radius;
  int64_t point_offset;
  int32_t formulation;
  int32_t scheme;
  double value_tol;
  double time_budget_ms;
  int64_t iter_budget;
} hj_solver_opts;

/* Solve B independent points with a common N (Algorithm 1, Eq. (disclaxBE); with
 * opts->formulation = HJ_FORM_HOPF, Algorithm 2, Eq. (dischopf)).  Points with
 * their own N, or their own problem, go through a ragged plan
 * (hj_ragged_plan_create) instead of per-point N and trajectory offsets here:
 * the plan sorts them into buckets by N class once, gives each bucket its own
 * launch shape, and replays the buckets as one CUDA graph, which a single call
 * with a common launch shape could not do without running every point at the
 * largest N's shape.
 *   xq       (device) [B][d] double: query points x (x_N is pinned to them).
 *   t        (device) [B] double: horizons t > 0; delta = t / N per point.
 *   N        number of time steps, 1..256 (nodes j = 0..N).
 *   V        (device) [B] double out: fval of Algorithm 1 at the last iterate,
 *            summed in FP64.
 *   iters    (device) [B] int32 out: iterations run.
 *   status   (device) [B] int8 out: HJ_POINT_*.
 *   kkt      (device, may be NULL) [B] double out: the residual of the discrete
 *            characteristic equations at the returned iterates (Section 4, the
 *            stationarity conditions of Eq. (disclaxBE): x' = H_p, p' = -H_x,
 *            p(0) = grad g in discrete form), evaluated as hj_kkt_residual does:
 *              max over j, k of |x_j - x_{j-1} - delta grad_p H(x_j, p_j)|,
 *              |p_1 - grad g(x_0)| and |p_{j+1} - p_j + delta grad_x H(x_j, p_j)|.
 *            Zero at a saddle, so it certifies each point without a reference
 *            solver (see hj_kkt_residual for the eikonal conventions).  It is
 *            hj_kkt_residual's kernel run after the solve on traj_x, traj_p (or on
 *            a stream-ordered workspace when those are NULL).  Backward Euler
 *            only, families quadratic, quadcopter, tanh drift and eikonal
 *            (HJ_ERR_UNSUPPORTED otherwise).  Every point gets the residual of the
 *            iterate it returned, converged or not.
 *   traj_x   (device, may be NULL) [B][N+1][d] out: x_0..x_N (Hopf: x_0 is the
 *            minimiser grad g*(p_1) = c + p_1 / W^2 of g(x_0) - <p_1, x_0>).
 *   traj_p   (device, may be NULL) [B][N+1][d] out: p_0 (= 0), p_1..p_N
 *            (p_j: the costate of interval [s_{j-1}, s_j], see HJ_SCHEME_*).
 *   warm_x, warm_p (device, may both be NULL) [B][N+1][d] in: initial iterate
 *            instead of the random guess (resume from traj_x, traj_p as written,
 *            so for the negative eikonal equation warm_p is the costate of phi,
 *            like traj_p); warm_x[b][N] is ignored
 *            (x_N = x) and warm_p[b][0] is ignored (p_0 = 0); Hopf also
 *            ignores warm_x[b][0].
 *   The trajectory and warm-start arrays have the element type of `precision`.
 * Errors: HJ_ERR_INVALID_ARG, HJ_ERR_STEP_SIZE, HJ_ERR_UNSUPPORTED, HJ_ERR_CUDA.
 * Calls that share one handle must be ordered on one stream (the handle owns
 * the work counter the persistent kernels draw points from).                */
hj_status hj_solve_batch(hj_problem prob, int64_t B,
                         const double* xq, const double* t, int32_t N,
                         const hj_solver_opts* opts,
                         double* V, int32_t* iters, int8_t* status, double* kkt,
                         void* traj_x, void* traj_p,
                         const void* warm_x, const void* warm_p,
                         void* stream);

/* Residual of the discrete characteristic equations (Section 4) at given
 * trajectories, per point: the kkt output of hj_solve_batch for trajectories
 * from any source (a ragged plan, retry rounds, a warm start).  Evaluated in
 * FP64, except the quadcopter's FP32 trajectories, which are evaluated in FP32
 * with the accurate sincosf: the error is then below about 16 units of 2^-24
 * times the magnitudes entering each term (|x_j - x_{j-1}|, |p_{j+1} - p_j|,
 * delta times the terms of grad H), under the rounding of the FP32 iterates
 * themselves.  The result is a double either way.
 *   t        (device) [B] horizons, delta = t / N.
 *   traj_x, traj_p (device) [B][N+1][d] in the type of `precision`, in the
 *            layout hj_solve_batch writes (traj_p[b][0] ignored).
 *   kkt      (device) [B] double out: max over j, k of
 *              |x_j - x_{j-1} - delta grad_p H(x_j, p_j, s_j)| (j = 1..N),
 *              |p_1 - grad g(x_0)|,
 *              |p_{j+1} - p_j + delta grad_x H(x_j, p_j, s_j)| (j = 1..N-1),
 *            s_j = j delta.  For the negative eikonal equation (dyn[0] = -1)
 *            the equations are those of the solver's variables (costate -p,
 *            initial data -g; Section 6.1 solves phi = -psi), whose residuals
 *            have the magnitudes of phi's own.  Where the eikonal H = c(x)|p| is
 *            not differentiable (p_j = 0) the first term is the distance from
 *            x_j - x_{j-1} to delta times the subdifferential, the ball of
 *            radius delta c(x_j).
 * Backward-Euler equations; families quadratic, quadcopter, tanh drift and
 * eikonal (HJ_ERR_UNSUPPORTED for the game).
 * Errors: HJ_ERR_INVALID_ARG, HJ_ERR_UNSUPPORTED, HJ_ERR_CUDA.               */
hj_status hj_kkt_residual(hj_problem prob, int64_t B, const double* t, int32_t N,
                          int32_t precision, const void* traj_x, const void* traj_p,
                          double* kkt, void* stream);

/* Gradient of L = sum_b w_b V_b at solved points (the adjoint of the value).
 * At a saddle of Eq. (disclaxBE) (trajectories of HJ_SCHEME_BE, Lax or Hopf
 * form) every total derivative of V equals the partial
 * derivative of its Lagrangian (envelope theorem), so from the trajectories of
 * a converged hj_solve_batch call (same problem, t, N, precision):
 *   dV/dW_i = W_i (x_0i - c_i)^2,   dV/dc_i = -W_i^2 (x_0i - c_i),
 *   dV/dtheta = -delta sum_{j=1..N} dH/dtheta(x_j, p_j)     (theta = dyn parameters),
 *   dV/dx_q   = p_N - delta grad_x H(x_N, p_N)              (x_N = x_q is pinned),
 * which for H independent of x is the costate p_N (Section 2: p = grad_x phi).
 * The same formulas hold at a Hopf saddle with x_0 = grad g*(p_1), the node 0
 * that hj_solve_batch writes for HJ_FORM_HOPF (-g*(p_1) has the derivatives
 * p_1^2 / W^3 and -p_1 in W and c).
 *   t        (device) [B] horizons; traj_x, traj_p (device) [B][N+1][d] in the
 *            precision's type (as written by hj_solve_batch).
 *   dL_dV    (device) [B] weights w_b (e.g. 1/B for the mean value).
 *   dW, dc   (device) [d] double out: sum_b w_b dV_b/dW, dV_b/dc (zeroed first).
 *   ddyn     (device) [n_dyn] double out, the family's dyn layout (quadcopter:
 *            m, a_h, g_z, eps; tanh drift: A row-major; eikonal: 0 for the
 *            sign, then c0, c1, c2, x_b, and v_b for a moving bump; NULL for
 *            quadratic).
 *   dxq      (device, may be NULL) [B][d] double out: w_b dV_b/dx_q.
 * Node arithmetic runs in the trajectory type, all sums in FP64.  The result is
 * the gradient of the value at the given iterates; it equals the derivative of
 * the converged value to the accuracy the iterates satisfy the saddle
 * conditions (Appendix A.1 stopping rule).
 * Errors: HJ_ERR_INVALID_ARG, HJ_ERR_UNSUPPORTED (tanh drift with d > 128; the
 * game), HJ_ERR_CUDA.                                                        */
hj_status hj_solve_grad(hj_problem prob, int64_t B, const double* t, int32_t N,
                        int32_t precision, const void* traj_x, const void* traj_p,
                        const double* dL_dV, double* dW, double* dc, double* ddyn, double* dxq,
                        void* stream);

/* The same gradient, exact for the value after the iterations actually run:
 * reverse-mode differentiation of Algorithm 1's K_b iterations of each point
 * (K_b = iters[b] of the forward solve with the same options), with the
 * iterates (x, p, z) checkpointed every checkpoint_every iterations and each
 * iterate rebuilt from its checkpoint during the reverse sweep (no iterate is
 * stored beyond the checkpoints).  The initial guess x^0 = x + r u and the
 * pinned x_N = x both carry dV/dx.  At a converged point the result agrees
 * with hj_solve_grad to the stopping accuracy.
 *   xq, t, N, opts   (device, device, host, host) as in the forward solve.
 *   iters            (device) [B] iterations of the forward solve.
 *   max_iters        (host) an upper bound of iters[] (sizes the workspace);
 *                    a point above it gets dxq = NaN.
 *   dL_dV, dW, dc, ddyn, dxq  as hj_solve_grad (dxq required).
 * Families: quadcopter (ddyn: m, a_h, g_z, eps) and quadratic with d <= 4;
 * N <= 256, and N <= 128 for the quadcopter in FP64; opts->inner_steps == 1
 * opts->formulation == HJ_FORM_LAX and opts->scheme == HJ_SCHEME_BE
 * (HJ_ERR_UNSUPPORTED otherwise).
 * Allocates a workspace of about 3 (N+1) d (max_iters/checkpoint_every + 1)
 * values per CTA of a grid of 4 CTAs per SM, and synchronises `stream`.
 * Errors: HJ_ERR_INVALID_ARG, HJ_ERR_STEP_SIZE, HJ_ERR_UNSUPPORTED, HJ_ERR_OOM,
 * HJ_ERR_CUDA.                                                               */
hj_status hj_solve_grad_unrolled(hj_problem prob, int64_t B, const double* xq, const double* t,
                                 int32_t N, const hj_solver_opts* opts, const int32_t* iters,
                                 int32_t max_iters, int32_t checkpoint_every, const double* dL_dV,
                                 double* dW, double* dc, double* ddyn, double* dxq, void* stream);

/* Launch shape of the register-resident kernel (quadratic d <= 4, quadcopter,
 * tanh drift d in {2, 4}, eikonal d in {2, 10}, the game d in {2, 7}): a group
 * of `warps_per_point` warps (1, 2, 4, 8) solves one point, each lane holding
 * `nodes_per_lane` time nodes (1 or 2; 1 for FP64), so
 * N <= 32 * warps_per_point * nodes_per_lane; warps_per_point = 0 selects half
 * a warp (16 lanes, nodes_per_lane = 1, N <= 16): two points per warp.  The
 * default is one node per lane over as few warps as N needs (two nodes per lane
 * for H = |p|^2/2, half a warp for N <= 16); hj_autotune times every
 * instantiated shape.  The shape does not
 * change any result, only the speed (the nodes a lane owns and the exchange
 * between lanes are the same arithmetic).  The shape is stored on the handle for
 * (precision, N) and used by later solves with that N.
 * Errors: HJ_ERR_INVALID_ARG, HJ_ERR_UNSUPPORTED (no such instantiation).     */
hj_status hj_set_launch_shape(hj_problem prob, int32_t precision, int32_t N,
                              int32_t warps_per_point, int32_t nodes_per_lane);

/* The launch shape solves with (precision, N) will use (host outputs).      */
hj_status hj_get_launch_shape(hj_problem prob, int32_t precision, int32_t N,
                              int32_t* warps_per_point, int32_t* nodes_per_lane);

/* Autotuner: times every instantiated launch shape on the caller's sample
 * (xq, t device arrays of B points, options as for hj_solve_batch), `repeats`
 * timed runs each after one warm-up, stores the fastest on the handle for
 * (opts->precision, N) and returns it (host outputs, each may be NULL).
 * Synchronises `stream`; allocates and frees its own scratch outputs.
 * Errors: as hj_solve_batch; HJ_ERR_UNSUPPORTED when the family/d has no
 * register-resident kernel (the shared-memory kernel has no shape to tune). */
hj_status hj_autotune(hj_problem prob, int64_t B, const double* xq, const double* t, int32_t N,
                      const hj_solver_opts* opts, int32_t repeats, int32_t* warps_per_point,
                      int32_t* nodes_per_lane, float* best_ms, void* stream);

/* Persisted launch shapes (the tuning of hj_autotune kept across processes).
 * hj_shapes_save writes every (precision, N) shape stored on the handle to the
 * text file `path` (host, NUL-terminated), one line per shape keyed by the
 * device's name, the family, d, the precision and N; lines of the file with
 * another key are kept, lines with the same key are replaced (the file is
 * rewritten through a temporary file next to it).  hj_shapes_load applies the
 * file's lines whose device name, family and d match the handle (through the
 * checks of hj_set_launch_shape, so a line naming a shape this build lacks is
 * skipped) and reports how many it applied (host, may be NULL).  A missing
 * file loads nothing.  The paper has no counterpart; it is configuration.
 * Errors: HJ_ERR_INVALID_ARG (null arguments, a file that cannot be written),
 * HJ_ERR_CUDA.                                                               */
hj_status hj_shapes_save(hj_problem prob, const char* path);
hj_status hj_shapes_load(hj_problem prob, const char* path, int32_t* n_loaded);

/* ---------------------------------------------------------------- ragged batches
 * A ragged batch mixes points of several problems (family, d) and their own
 * number of time steps N (Algorithm 1 per point, as hj_solve_batch).  A plan
 * fixes the batch's structure once; every solve with it is one CUDA-graph
 * launch in which each (problem, N class) bucket of points runs its own
 * persistent kernel as a parallel branch.  The paper has no ragged batches; the
 * arithmetic per point is exactly that of hj_solve_batch.                    */
typedef struct hj_ragged_plan_s* hj_ragged_plan;

/* Build a plan.
 *   probs    (host) n_prob problem handles, all on the current device; they must
 *            outlive the plan.
 *   prob_of  (host) [B] int32: problem index of each point (0..n_prob-1).
 *   N_of     (host) [B] int32: time steps of each point (1..256).
 *   opts     (host) options shared by every point; point b's initial guess uses
 *            global index opts->point_offset + b.
 * Packed layouts (offsets from hj_ragged_plan_layout): the query points are
 * xq[xq_off[b] .. xq_off[b] + d_b) (doubles), the trajectories
 * traj[traj_off[b] .. traj_off[b+1]) as [N_b+1][d_b] (iterate type).
 * The plan owns device copies of N, the offsets and the bucket index lists,
 * one work counter per bucket and four side streams.
 * Errors: HJ_ERR_INVALID_ARG, HJ_ERR_STEP_SIZE, HJ_ERR_OOM, HJ_ERR_CUDA;
 * HJ_ERR_UNSUPPORTED when a bucket served by the shared-memory kernel does not
 * fit its 227 KB (FP64 tanh drift: 4 (N+1) d + d^2 doubles, e.g. d = 32 allows
 * N <= 200).                                                                */
hj_status hj_ragged_plan_create(hj_ragged_plan* out, int32_t n_prob, const hj_problem* probs,
                                int64_t B, const int32_t* prob_of, const int32_t* N_of,
                                const hj_solver_opts* opts);

/* Host outputs, each may be NULL: xq_offsets[B+1] (doubles), traj_offsets[B+1]
 * (elements), number of buckets.                                            */
hj_status hj_ragged_plan_layout(hj_ragged_plan plan, int64_t* xq_offsets, int64_t* traj_offsets,
                                int32_t* n_buckets);

/* Host outputs for bucket i (each may be NULL): its problem index, largest N,
 * number of points, launch shape (0, 0 = shared-memory kernel) and inner
 * gradient steps per x-update.                                              */
hj_status hj_ragged_plan_bucket(hj_ragged_plan plan, int32_t i, int32_t* problem, int32_t* n_max,
                                int64_t* n_points, int32_t* warps_per_point,
                                int32_t* nodes_per_lane, int32_t* inner_steps);

/* Solve the batch: xq (device, packed), t (device, [B]); V, iters, status
 * (device, [B]); traj_x, traj_p (device, packed, may be NULL).  The first call
 * with a given set of buffers captures the graph on a stream the plan owns;
 * every call launches it on `stream` (the legacy default stream is accepted).
 * Later calls with the same buffers replay the graph without capturing.  Solves
 * on one plan must be ordered on one stream.
 * Errors: HJ_ERR_INVALID_ARG, HJ_ERR_CUDA.                                   */
hj_status hj_ragged_solve(hj_ragged_plan plan, const double* xq, const double* t, double* V,
                          int32_t* iters, int8_t* status, void* traj_x, void* traj_p,
                          void* stream);

/* Autotune every bucket that runs the register-resident kernel: time each
 * instantiated launch shape on the bucket's own points (`repeats` timed runs
 * after one warm-up) and keep the fastest.  With max_inner_steps > 1 the
 * inner gradient steps per x-update (1..max_inner_steps, families whose H
 * depends on x) are tuned too: they change the iterates and iteration counts,
 * not the fixed point; 1 keeps the plan's option (Section 5.3's single step).
 * Synchronises `stream`; allocates and frees scratch outputs; drops the
 * captured graph.                                                            */
hj_status hj_ragged_autotune(hj_ragged_plan plan, const double* xq, const double* t,
                             int32_t repeats, int32_t max_inner_steps, void* stream);

/* Destroy a plan (NULL accepted); synchronises its device first.            */
hj_status hj_ragged_plan_destroy(hj_ragged_plan plan);

/* ---------------------------------------------------------------- retry rounds
 * The paper's handling of points that reach the iteration cap: Section 6.2
 * raises sigma by 20 and sets tau = 0.25 / sigma (here: step_product / sigma)
 * for such game points; Section 6.1 reruns such eikonal points.
 *   rounds        extra rounds, 0..127 (0: the plain hj_solve_batch).
 *   sigma_step    round r runs sigma_r = opts->sigma + r * sigma_step.
 *   step_product  tau_r = step_product / sigma_r; 0 keeps opts->sigma * opts->tau.
 *   warm          0: round r reruns the point from a fresh random guess drawn
 *                 with seed + r; 1: it continues from the point's last iterate
 *                 (z restarts at x).
 *   value_tol     > 0: the last round also applies the value test
 *                 (hj_solver_opts.value_tol), the paper's switch to a value
 *                 criterion after a maximum count; 0: off.                     */
typedef struct {
  int32_t rounds;
  double sigma_step;
  double step_product;
  int32_t warm;
  double value_tol;
} hj_retry_policy;

/* hj_solve_batch, then up to policy->rounds more rounds, each over the points
 * whose status is still HJ_POINT_MAX_ITER, with that round's sigma, tau and
 * seed (opts->max_iter iterations per round).  A retried point's outputs are
 * those of its last round; iters[] is its total over all rounds; rounds[]
 * (device, may be NULL) [B] int8 out: the last round the point ran in.
 * traj_x, traj_p may be NULL (with warm = 1 the library then keeps them in a
 * workspace).  Every round's options must pass the checks of hj_solve_batch
 * (sigma_r > 0, 4 sigma_r tau_r < 1, ...) or nothing runs.  Allocates a
 * stream-ordered workspace of 2B int32 (+ 2 or 4 trajectory arrays with
 * warm = 1) and synchronises `stream` once per extra round (to read how many
 * points it retries).
 * Errors: those of hj_solve_batch, HJ_ERR_OOM.                               */
hj_status hj_solve_batch_retry(hj_problem prob, int64_t B, const double* xq, const double* t,
                               int32_t N, const hj_solver_opts* opts, const hj_retry_policy* policy,
                               double* V, int32_t* iters, int8_t* status, int8_t* rounds,
                               void* traj_x, void* traj_p, void* stream);

/* ---------------------------------------------------------------- no device allocation
 * hj_solve_batch for callers that cannot allocate device memory: code running
 * under a device-memory budget fixed before it starts (an allocator owned by a
 * host framework), a real-time loop that forbids allocation after start-up, or
 * a plug-in that only receives buffers it did not allocate.  hj_problem_create
 * allocates (the parameter copies and the persistent kernels' work counter);
 * this entry point allocates nothing: it copies the problem's parameters and
 * keeps the work counter in one fixed array of hj_static_scratch_bytes() bytes
 * that the library declares in device memory (every GPU that loads the library
 * holds it until the process exits), then runs the same kernels as
 * hj_solve_batch.  The paper has no counterpart; it is a deployment variant.
 *   family, d, dyn, n_dyn, W, c   (host) as hj_problem_create.
 *   B, xq, t, N, opts, V, iters, status, traj_x, traj_p, stream
 *                                 as hj_solve_batch (no warm start; the launch
 *                                 shape is the default for (precision, N)).
 * The first call on a device looks up the array's device address (set-up, once
 * per device, with that device current).  Every call shares the one array and
 * overwrites it (the work counter is cleared on each call): calls that overlap
 * on the GPU, from any stream or thread, race and must be serialised by the
 * caller.
 * Errors: as hj_solve_batch; HJ_ERR_UNSUPPORTED when the parameters do not fit
 * the array (tanh drift: 3d + 3d^2 doubles for FP64, 3d + 2d^2 doubles for
 * FP32, plus alignment: d <= 51 in FP64, d <= 62 in FP32).                   */
int64_t hj_static_scratch_bytes(void);
hj_status hj_solve_batch_static(int32_t family, int32_t d, const double* dyn, int64_t n_dyn,
                                const double* W, const double* c, int64_t B, const double* xq,
                                const double* t, int32_t N, const hj_solver_opts* opts,
                                double* V, int32_t* iters, int8_t* status, void* traj_x,
                                void* traj_p, void* stream);

/* Diagnostic, with no counterpart in the method: the device's FP32 FMA
 * throughput, measured by one launch of independent FMA chains that fills every
 * SM (after one warm-up launch).  It is the measured denominator of the
 * roofline fraction of the FP32 iteration kernels, which the FP32 FMA pipe bounds.
 *   iters   (host) >= 1; every thread runs 8 chains of 16 * iters FMAs
 *           (50000 runs for ~50 ms on a GB300).
 *   packed  (host) 0: scalar fmaf; 1: the packed two-wide FMA (2 FMAs each).
 *   tflops  (host) out: 2 * FMAs / elapsed seconds / 1e12 (CUDA events).
 * Allocates a small stream-ordered scratch buffer; synchronises `stream`.
 * Errors: HJ_ERR_INVALID_ARG, HJ_ERR_OOM, HJ_ERR_CUDA.                       */
hj_status hj_probe_fp32_fma(int64_t iters, int32_t packed, double* tflops, void* stream);

/* Human-readable name of a status code (static storage). */
const char* hj_status_str(hj_status s);

/* Library version (major * 10000 + minor * 100 + patch). */
int32_t hj_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HJPDHG_H */
