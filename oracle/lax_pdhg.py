"""Algorithm 1 (Lax formula, backward Euler) in FP64, one step at a time.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The saddle problem (Eq. disclaxBE): with delta = t/N, x_N = x_target,
    phi(x, t) ~ max_{p_1..p_N} min_{x_0..x_{N-1}}
        g(x_0) + sum_{j=1}^N <p_j, x_j - x_{j-1}> - delta sum_{j=1}^N H(x_j, p_j).

One iteration (Appendix Algorithm A.1 with the updates of Section 5.3):
  dual    p_j <- argmin_p delta H(x_j^k, p) + |p - (p_j^k + sigma (z_j^k - z_{j-1}^k))|^2/(2 sigma),
          j = 1..N                               ((D z)_j = z_j - z_{j-1})
  x_0     x_0 <- prox_{tau g}(x_0^k - tau (D^T p^{k+1})_0),  (D^T p)_0 = -p_1  (p_0 = 0)
  x_j     x_j <- x_j^k - tau (p_j^{k+1} - p_{j+1}^{k+1}) + tau delta grad_x H(x_j^k, p_j^{k+1}),
          j = 1..N-1  (one gradient step on -delta H; `inner_steps` > 1 repeats it at the
          new x, approaching the exact argmin of Algorithm A.1 with the same fixed point)
  x_N     stays x_target
  relax   z = x^{k+1} + theta (x^{k+1} - x^k)
  stop    |x^{k+1} - x^k|_2^2 < tol and |p^{k+1} - p^k|_2^2 < tol (Section 6), tested
          after every `check_every`-th iteration, or when max_iter iterations are done.
  value   fval = g(x_0) + sum_j <p_j, x_j - x_{j-1}> - delta sum_j H(x_j, p_j).

Readings of the paper taken here (each also listed in the design notes):
  * delta = t/N with nodes j = 0..N (Appendix), not N = t/delta + 1.
  * The x-step uses p^{k+1} (Algorithm 1 and Section 5.3), not p^k.
  * The dual prox evaluates H at x^k (Appendix), the same point as grad_x H.
  * p_N is a free dual variable updated like the others; x_N is pinned.
Initial guess (Section 6): x_j^0 = x_target + r u (j < N), p_j^0 = r u' (j >= 1), with
u, u' in [-1, 1) from the counter-based generator in counter_rng.

Negative eikonal equation (Section 6.1): phi_t - c(x)|grad phi| = 0 with initial
data g is solved as -psi, psi the positive equation's solution with initial
data -g (concave: its proximal map is the "stretch" of Section 6.1); the
returned V and p are those of phi (V = -V_psi, p = -p_psi), x is shared.
"""
import numpy as np

from .counter_rng import uniform_pm1
from .families import Eikonal, QuadCost, make_family

CONVERGED, MAX_ITER, NONFINITE = 0, 1, 2
VALUE_STOP = 4     # stopped by the value test (the paper's switch for slow points)


def eikonal_sign(w):
    """-1 for the negative eikonal equation (dyn[0] = -1), else +1."""
    if w["family"] == "eikonal" and float(np.asarray(w["dyn"])[0]) < 0:
        return -1.0
    return 1.0


def initial_guess(xq, N, seed, radius, point_index):
    """x^0 [B, N+1, d] and p^0 [B, N+1, d] (p^0_0 = 0) for Section 6's random init."""
    B, d = xq.shape
    P = np.asarray(point_index, dtype=np.uint64)[:, None, None]
    J = np.arange(N + 1, dtype=np.uint64)[None, :, None]
    C = np.arange(d, dtype=np.uint64)[None, None, :]
    x0 = xq[:, None, :] + radius * uniform_pm1(seed, P, 0, J, C)
    x0[:, N, :] = xq
    p0 = radius * uniform_pm1(seed, P, 1, J, C)
    p0[:, 0, :] = 0.0
    return x0, p0


def node_times(delta, N):
    """s_j = j delta, j = 0..N (uniform nodes, s_N = t), shape [B, N+1]."""
    return np.arange(N + 1)[None, :] * np.asarray(delta, dtype=np.float64)[:, None]


def lax_value(fam, cost, x, p, delta):
    """fval of Algorithm 1 for stacked x [B, N+1, d], p [B, N+1, d] (p_0 unused)."""
    dx = x[:, 1:, :] - x[:, :-1, :]
    pair = np.sum(p[:, 1:, :] * dx, axis=(1, 2))
    S = node_times(delta, x.shape[1] - 1)
    ham = np.sum(fam.H(x[:, 1:, :], p[:, 1:, :], s=S[:, 1:]), axis=1)
    return cost.g(x[:, 0, :]) + pair - delta * ham


def solve(w, *, N=None, sigma=None, tau=None, theta=1.0, tol=None, max_iter=None,
          check_every=None, inner_steps=1, seed=None, init_radius=None,
          x_init=None, p_init=None, activation="tanh", value_tol=0.0):
    """Run Algorithm 1 on every query point of workload `w` (uniform N).

    Returns dict(V [B], iters [B], status [B], x [B, N+1, d], p [B, N+1, d],
    rx [B], rp [B]) where rx, rp are the last squared increments.

    value_tol > 0 adds the paper's other stopping rule for slow points
    (Section 6.2): at a test, a point whose value fval moved by less than
    value_tol since the previous test stops with status VALUE_STOP.
    """
    fam = make_family(w, activation=activation)
    sign = eikonal_sign(w)
    cost = QuadCost(w["W"], w["c"], sign=sign)
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
        p_all = sign * np.array(p_init, dtype=np.float64)    # p_init as returned (phi's costate)
        x_all[:, N, :] = xq
        p_all[:, 0, :] = 0.0
    z_all = x_all.copy()
    iters = np.zeros(B, dtype=np.int64)
    status = np.full(B, MAX_ITER, dtype=np.int64)
    rx_all = np.full(B, np.inf)
    rp_all = np.full(B, np.inf)

    act = np.arange(B)                     # points still iterating
    x, p, z, delta = x_all[act], p_all[act], z_all[act], delta_all[act]
    vprev = np.full(B, np.nan)             # fval at the previous test
    lam = sigma * delta[:, None]           # sigma * delta for every node j = 1..N
    k = 0
    while act.size and k < max_iter:
        # dual step, j = 1..N, H evaluated at x^k (and the node times s_j = j delta)
        S = node_times(delta, N)
        v = p[:, 1:, :] + sigma * (z[:, 1:, :] - z[:, :-1, :])
        p_new = np.empty_like(p)
        p_new[:, 0, :] = 0.0
        p_new[:, 1:, :] = fam.prox_p(x[:, 1:, :], v, lam, s=S[:, 1:])
        # primal step, x_0: prox of g, (D^T p)_0 = -p_1
        x_new = np.empty_like(x)
        x_new[:, 0, :] = cost.prox(x[:, 0, :] + tau * p_new[:, 1, :], tau)
        # primal step, x_j for j = 1..N-1: gradient step on -delta H
        base = x[:, 1:N, :] - tau * (p_new[:, 1:N, :] - p_new[:, 2:N + 1, :])
        xj = x[:, 1:N, :]
        for _ in range(inner_steps):
            xj = base + tau * delta[:, None, None] * fam.grad_x(xj, p_new[:, 1:N, :], s=S[:, 1:N])
        x_new[:, 1:N, :] = xj
        x_new[:, N, :] = x[:, N, :]
        # over-relaxation
        z = x_new + theta * (x_new - x)
        rx = np.sum((x_new - x) ** 2, axis=(1, 2))
        rp = np.sum((p_new - p) ** 2, axis=(1, 2))
        x, p = x_new, p_new
        k += 1
        if k % check_every == 0 or k == max_iter:
            bad = ~(np.isfinite(rx) & np.isfinite(rp))
            conv = (rx < tol) & (rp < tol) & ~bad
            vstop = np.zeros_like(conv)
            if value_tol > 0:
                v = lax_value(fam, cost, x, p, delta)
                vstop = (np.abs(v - vprev) < value_tol) & ~bad & ~conv
                vprev = v
            stop = bad | conv | vstop | (k == max_iter)
            if np.any(stop):
                ids = act[stop]
                x_all[ids], p_all[ids], z_all[ids] = x[stop], p[stop], z[stop]
                iters[ids] = k
                rx_all[ids], rp_all[ids] = rx[stop], rp[stop]
                status[ids] = np.where(bad[stop], NONFINITE,
                                       np.where(conv[stop], CONVERGED,
                                                np.where(vstop[stop], VALUE_STOP, MAX_ITER)))
                keep = ~stop
                act = act[keep]
                x, p, z, delta = x[keep], p[keep], z[keep], delta[keep]
                lam = lam[keep]
                vprev = vprev[keep]
    V = lax_value(fam, cost, x_all, p_all, delta_all)
    return dict(V=sign * V, iters=iters, status=status, x=x_all, p=sign * p_all,
                rx=rx_all, rp=rp_all)


def kkt_residual(w, x, p, activation="tanh", parts=False):
    """Max-norm residual of the discrete characteristic equations at (x, p), the
    stationarity conditions of the Lagrangian of Eq. disclaxBE (the discrete form
    of x' = H_p, p' = -H_x with p(0) = grad g(x(0)), Section 4):
        r1_j = x_j - x_{j-1} - delta grad_p H(x_j, p_j)           j = 1..N
        r2   = p_1 - grad g(x_0)
        r3_j = p_{j+1} - p_j + delta grad_x H(x_j, p_j)           j = 1..N-1
    Zero at every saddle.  x, p are as `solve` returns them; for the negative
    eikonal equation p is phi's costate and the equations are taken in the
    solver's variables (psi = -phi: costate -p, initial data -g), which have the
    same residual magnitudes as phi's own characteristic equations.  Where the
    eikonal H = c(x)|p| is not differentiable (p_j = 0), r1_j is the distance from
    x_j - x_{j-1} to delta times the subdifferential, the ball of radius c(x_j).
    Returns [B], or with parts=True the three maxima (r1, r2, r3), each [B]."""
    fam = make_family(w, activation=activation)
    sign = eikonal_sign(w)
    cost = QuadCost(w["W"], w["c"], sign=sign)
    q = sign * np.asarray(p, dtype=np.float64)          # the solver's costate
    x = np.asarray(x, dtype=np.float64)
    N = x.shape[1] - 1
    delta = (np.asarray(w["t"], dtype=np.float64) / N)[:, None, None]
    S = node_times(delta[:, 0, 0], N)
    dx = x[:, 1:] - x[:, :-1]
    r1 = dx - delta * fam.grad_p(x[:, 1:], q[:, 1:], s=S[:, 1:])
    if isinstance(fam, Eikonal):
        # p_j = 0: distance of dx_j to the ball of radius delta c(x_j)
        c, _ = fam.speed(x[:, 1:], S[:, 1:])
        n = np.sqrt(np.sum(dx * dx, axis=-1))
        out = np.maximum(0.0, 1.0 - delta[..., 0] * c / np.where(n > 0, n, 1.0))
        zero = np.all(q[:, 1:] == 0.0, axis=-1)
        r1 = np.where(zero[..., None], dx * out[..., None], r1)
    r2 = q[:, 1] - cost.grad(x[:, 0])
    r3 = q[:, 2:] - q[:, 1:N] + delta * fam.grad_x(x[:, 1:N], q[:, 1:N], s=S[:, 1:N])
    m1 = np.max(np.abs(r1), axis=(1, 2))
    m2 = np.max(np.abs(r2), axis=1)
    m3 = np.max(np.abs(r3), axis=(1, 2)) if N > 1 else np.zeros_like(m1)
    if parts:
        return m1, m2, m3
    return np.maximum(m1, np.maximum(m2, m3))
