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
  HJ_FAMILY_TANH_DRIFT = 2
};

/* Iterate precision.  FP32 iterates keep the increment reductions and the
 * value sum in FP64; FP64 runs everything in double.                        */
enum { HJ_PREC_FP32 = 0, HJ_PREC_FP64 = 1 };

/* Per-point outcome written to status[]. */
enum { HJ_POINT_CONVERGED = 0, HJ_POINT_MAX_ITER = 1, HJ_POINT_NONFINITE = 2 };

typedef struct hj_problem_s* hj_problem;

/* Create a problem: Hamiltonian family + terminal cost g(x) = 1/2 sum_i W_i^2 (x_i - c_i)^2.
 *   out      (host) receives the handle; set to NULL on error.
 *   family   HJ_FAMILY_*;  d state dimension (1..128; 12 for the quadcopter).
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
 *                split into slices reproduces the unsplit run.                */
typedef struct {
  double sigma, tau, theta, tol;
  int32_t max_iter, check_every, inner_steps, precision;
  uint64_t seed;
  double init_radius;
  int64_t point_offset;
} hj_solver_opts;

/* Solve B independent points with a common N (Algorithm 1, Eq. (disclaxBE)).
 *   xq       (device) [B][d] double: query points x (x_N is pinned to them).
 *   t        (device) [B] double: horizons t > 0; delta = t / N per point.
 *   N        number of time steps, 1..256 (nodes j = 0..N).
 *   V        (device) [B] double out: fval of Algorithm 1 at the last iterate,
 *            summed in FP64.
 *   iters    (device) [B] int32 out: iterations run.
 *   status   (device) [B] int8 out: HJ_POINT_*.
 *   traj_x   (device, may be NULL) [B][N+1][d] out: x_0..x_N.
 *   traj_p   (device, may be NULL) [B][N+1][d] out: p_0 (= 0), p_1..p_N.
 *   warm_x, warm_p (device, may both be NULL) [B][N+1][d] in: initial iterate
 *            instead of the random guess (resume); warm_x[b][N] is ignored
 *            (x_N = x) and warm_p[b][0] is ignored (p_0 = 0).
 *   The trajectory and warm-start arrays have the element type of `precision`.
 * Errors: HJ_ERR_INVALID_ARG, HJ_ERR_STEP_SIZE, HJ_ERR_UNSUPPORTED, HJ_ERR_CUDA.
 * Calls that share one handle must be ordered on one stream (the handle owns
 * the work counter the persistent kernels draw points from).                */
hj_status hj_solve_batch(hj_problem prob, int64_t B,
                         const double* xq, const double* t, int32_t N,
                         const hj_solver_opts* opts,
                         double* V, int32_t* iters, int8_t* status,
                         void* traj_x, void* traj_p,
                         const void* warm_x, const void* warm_p,
                         void* stream);

/* Human-readable name of a status code (static storage). */
const char* hj_status_str(hj_status s);

/* Library version (major * 10000 + minor * 100 + patch). */
int32_t hj_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HJPDHG_H */
