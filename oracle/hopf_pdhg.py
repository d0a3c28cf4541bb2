"""Algorithm 2 (Hopf formula, backward Euler) in FP64, one step at a time.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The saddle problem (Eq. dischopf): with delta = t/N and x_N = x_target,
    phi(x, t) ~ max_{p_1..p_N} min_{x_1..x_{N-1}}
        -g*(p_1) + <p_N, x_target> + sum_{j=1}^{N-1} <p_j - p_{j+1}, x_j>
        - delta sum_{j=1}^N H(x_j, p_j),
obtained from Eq. (disclaxBE) by minimising over x_0 in closed form
(min_{x_0} g(x_0) - <p_1, x_0> = -g*(p_1)), so for convex g it has the same
saddle value as the Lax problem.  For g(x) = 1/2 sum_i W_i^2 (x_i - c_i)^2,
g*(p) = <p, c> + 1/2 sum_i p_i^2 / W_i^2 (all W_i must be nonzero).

One iteration (appendix tutorial algorithm for the Hopf formula), with the
difference operator of the Hopf form ((D^T z)_1 = z_1, (D^T z)_j = z_j - z_{j-1}
for j >= 2, (D p)_j = p_j - p_{j+1}):
  dual, j = 1   p_1 <- argmin_p g*(p) + delta H(x_1^k, p) + |p - (p_1^k + sigma z_1^k)|^2/(2 sigma)
  dual, j >= 2  p_j <- argmin_p delta H(x_j^k, p) + |p - (p_j^k + sigma (z_j^k - z_{j-1}^k))|^2/(2 sigma)
  x_j           x_j <- x_j^k - tau (p_j^{k+1} - p_{j+1}^{k+1}) + tau delta grad_x H(x_j^k, p_j^{k+1}),
                j = 1..N-1 (one gradient step on -delta H, as in the Lax oracle)
  x_N           stays x_target
  relax         z = x^{k+1} + theta (x^{k+1} - x^k),  j = 1..N
  stop          as the Lax oracle (squared increments of x_1..x_{N-1} and p_1..p_N)
  value         fval = -g*(p_1) + <p_N, x_target> + sum_{j=1}^{N-1} <p_j - p_{j+1}, x_j>
                       - delta sum_j H(x_j, p_j)
The same readings as the Lax oracle (delta = t/N, p^{k+1} in the x-step, H at x^k
in the dual step, one gradient step, p_N free).  The j = 1 step is the exact
joint prox the appendix algorithm writes (the Section 5.3 variant instead takes
a gradient step on g*); every family here has H quadratic in p, so the prox is
the linear system
    (I + sigma diag(1/W^2) + lam M(x)) p = v - sigma c - lam grad_p H(x, 0),
    M(x) p = grad_p H(x, p) - grad_p H(x, 0),  lam = sigma delta,
solved as written.  The returned trajectory stores, at node 0, the x_0 that
attains the conjugate: x_0 = grad g*(p_1) = c + p_1 / W^2.
"""
import numpy as np

from .families import QuadCost, make_family
from .lax_pdhg import CONVERGED, MAX_ITER, NONFINITE, initial_guess


def conj_g(cost, p):
    """g*(p) = <p, c> + 1/2 sum_i p_i^2 / W_i^2."""
    return np.sum(p * cost.c, axis=-1) + 0.5 * np.sum(p * p / cost.w2, axis=-1)


def grad_conj_g(cost, p):
    return cost.c + p / cost.w2


def prox_first(fam, cost, x1, v, lam, sigma):
    """argmin_p sigma g*(p) + lam H(x1, p) + |p - v|^2 / 2 for x1, v [B, d], lam [B]."""
    B, d = v.shape
    zero = np.zeros_like(v)
    f0 = fam.grad_p(x1, zero)
    M = np.empty((B, d, d))
    for k in range(d):
        e = np.zeros_like(v)
        e[:, k] = 1.0
        M[:, :, k] = fam.grad_p(x1, e) - f0
    A = np.eye(d)[None] * (1.0 + sigma / cost.w2)[None, None, :] \
        + lam[:, None, None] * M
    rhs = v - sigma * cost.c - lam[:, None] * f0
    return np.linalg.solve(A, rhs[..., None])[..., 0]


def hopf_value(fam, cost, x, p, xq, delta):
    """fval of the Hopf algorithm for stacked x, p [B, N+1, d] (x_N = x_target)."""
    N = x.shape[1] - 1
    pair = np.sum(p[:, N, :] * xq, axis=-1) \
        + np.sum((p[:, 1:N, :] - p[:, 2:N + 1, :]) * x[:, 1:N, :], axis=(1, 2))
    ham = np.sum(fam.H(x[:, 1:, :], p[:, 1:, :]), axis=1)
    return -conj_g(cost, p[:, 1, :]) + pair - delta * ham


def solve_hopf(w, *, N=None, sigma=None, tau=None, theta=1.0, tol=None, max_iter=None,
               check_every=None, inner_steps=1, seed=None, init_radius=None,
               x_init=None, p_init=None, activation="tanh"):
    """Run the Hopf algorithm on every query point of workload `w` (uniform N).

    Same arguments and result layout as lax_pdhg.solve; x[:, 0, :] holds
    grad g*(p_1) and p[:, 0, :] = 0.
    """
    if w["family"] == "eikonal":
        raise ValueError("the Hopf form here needs H quadratic in p (not the eikonal family)")
    fam = make_family(w, activation=activation)
    if getattr(fam, "time_dependent", False):
        raise ValueError("a time-dependent H is solved in the backward-Euler Lax form only")
    cost = QuadCost(w["W"], w["c"])
    if np.any(cost.w2 == 0.0):
        raise ValueError("the Hopf form needs every W_i nonzero (g* finite)")
    N = int(w["N"] if N is None else N)
    sigma = float(w["sigma"] if sigma is None else sigma)
    tau = float(w["tau"] if tau is None else tau)
    tol = float(w["tol"] if tol is None else tol)
    max_iter = int(w["max_iter"] if max_iter is None else max_iter)
    check_every = int(w["check_every"] if check_every is None else check_every)
    seed = int(w["seed"] if seed is None else seed)
    radius = float(w["init_radius"] if init_radius is None else init_radius)

    xq = np.asarray(w["xq"], dtype=np.float64)
    B, d = xq.shape
    pidx = w.get("point_index", np.arange(B))
    delta_all = np.asarray(w["t"], dtype=np.float64) / N

    if x_init is None:
        x_all, p_all = initial_guess(xq, N, seed, radius, pidx)
    else:
        x_all = np.array(x_init, dtype=np.float64)
        p_all = np.array(p_init, dtype=np.float64)
    x_all[:, N, :] = xq
    x_all[:, 0, :] = 0.0                   # x_0 is not a variable of the Hopf form
    p_all[:, 0, :] = 0.0
    z_all = x_all.copy()
    iters = np.zeros(B, dtype=np.int64)
    status = np.full(B, MAX_ITER, dtype=np.int64)
    rx_all = np.full(B, np.inf)
    rp_all = np.full(B, np.inf)

    act = np.arange(B)
    x, p, z, delta = x_all[act], p_all[act], z_all[act], delta_all[act]
    k = 0
    while act.size and k < max_iter:
        lam = sigma * delta
        # dual step: j = 1 joint prox of g* and delta H, j >= 2 prox of delta H (H at x^k)
        p_new = np.empty_like(p)
        p_new[:, 0, :] = 0.0
        v1 = p[:, 1, :] + sigma * z[:, 1, :]
        p_new[:, 1, :] = prox_first(fam, cost, x[:, 1, :], v1, lam, sigma)
        if N >= 2:
            v = p[:, 2:, :] + sigma * (z[:, 2:, :] - z[:, 1:-1, :])
            lam_j = np.broadcast_to(lam[:, None], v.shape[:2])
            p_new[:, 2:, :] = fam.prox_p(x[:, 2:, :], v, lam_j)
        # primal step, x_j for j = 1..N-1
        x_new = x.copy()
        base = x[:, 1:N, :] - tau * (p_new[:, 1:N, :] - p_new[:, 2:N + 1, :])
        xj = x[:, 1:N, :]
        for _ in range(inner_steps):
            xj = base + tau * delta[:, None, None] * fam.grad_x(xj, p_new[:, 1:N, :])
        x_new[:, 1:N, :] = xj
        z = x_new + theta * (x_new - x)
        z[:, 0, :] = 0.0
        rx = np.sum((x_new - x) ** 2, axis=(1, 2))
        rp = np.sum((p_new - p) ** 2, axis=(1, 2))
        x, p = x_new, p_new
        k += 1
        if k % check_every == 0 or k == max_iter:
            bad = ~(np.isfinite(rx) & np.isfinite(rp))
            conv = (rx < tol) & (rp < tol) & ~bad
            stop = bad | conv | (k == max_iter)
            if np.any(stop):
                ids = act[stop]
                x_all[ids], p_all[ids], z_all[ids] = x[stop], p[stop], z[stop]
                iters[ids] = k
                rx_all[ids], rp_all[ids] = rx[stop], rp[stop]
                status[ids] = np.where(bad[stop], NONFINITE,
                                       np.where(conv[stop], CONVERGED, MAX_ITER))
                keep = ~stop
                act = act[keep]
                x, p, z, delta = x[keep], p[keep], z[keep], delta[keep]
    V = hopf_value(fam, cost, x_all, p_all, xq, delta_all)
    x_all[:, 0, :] = grad_conj_g(cost, p_all[:, 1, :])
    return dict(V=V, iters=iters, status=status, x=x_all, p=p_all,
                rx=rx_all, rp=rp_all)
