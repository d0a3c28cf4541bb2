"""The Lax saddle problem with the forward-Euler discretisation (Eq. disclaxFE)
and its trapezoid average with backward Euler (Section 5, after Algorithm 1;
Section 7), solved by the PDHG iteration of Algorithm 1, in FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Indexing follows Eq. disclaxFE: costates p_0..p_{N-1}, p_j belonging to the
interval [s_j, s_{j+1}], states x_0..x_N with x_N = x_target.  With weights
(wL, wR) on the two ends of each interval the saddle function is
    g(x_0) + sum_{j=0}^{N-1} <p_j, x_{j+1} - x_j>
           - delta sum_{j=0}^{N-1} (wL H(x_j, p_j) + wR H(x_{j+1}, p_j)),
  forward Euler      (wL, wR) = (1, 0)     (Eq. disclaxFE)
  trapezoid          (wL, wR) = (1/2, 1/2) (the average of the two Euler forms)
  backward Euler     (wL, wR) = (0, 1)     (Eq. disclaxBE with p_j renamed p_{j+1})

One iteration, the steps of Algorithm 1 with H at x^k as in the
backward-Euler solver (lax_pdhg.py):
  dual   p_j <- argmin_p delta (wL H(x_j^k, p) + wR H(x_{j+1}^k, p))
                        + |p - (p_j^k + sigma (z_{j+1} - z_j))|^2 / (2 sigma)    j = 0..N-1
  x_0    x_0 <- prox_{tau g}(x_0^k + tau p_0 + tau delta wL grad_x H(x_0^k, p_0))
         (g and H both act on x_0 here; the H part takes one gradient step, as
         Algorithm 1 does for every x_j, and g keeps its exact proximal map)
  x_j    x_j <- x_j^k - tau (p_{j-1} - p_j)
                + tau delta (wL grad_x H(x_j^k, p_j) + wR grad_x H(x_j^k, p_{j-1}))  j = 1..N-1
  relax  z = x^{k+1} + theta (x^{k+1} - x^k)
  stop   |x^{k+1} - x^k|^2 < tol and |p^{k+1} - p^k|^2 < tol, every check_every-th
         iteration (Section 6)
  value  the saddle function above at the last iterate.
Initial guess: x^0 as in lax_pdhg.initial_guess; p_j^0 is the draw that the
backward-Euler solver uses for its node j + 1 (the same interval).
The negative eikonal equation goes through phi = -psi as in lax_pdhg.py.
"""
import numpy as np

from .families import QuadCost, make_family
from .lax_pdhg import CONVERGED, MAX_ITER, NONFINITE, eikonal_sign, initial_guess

SCHEMES = {"fe": (1.0, 0.0), "trap": (0.5, 0.5), "be": (0.0, 1.0)}


def scheme_value(fam, cost, x, p, delta, wl, wr):
    """The saddle function for x [B, N+1, d], p [B, N, d] (interval costates)."""
    pair = np.sum(p * (x[:, 1:, :] - x[:, :-1, :]), axis=(1, 2))
    ham = np.zeros(x.shape[0])
    if wl:
        ham = ham + wl * np.sum(fam.H(x[:, :-1, :], p), axis=1)
    if wr:
        ham = ham + wr * np.sum(fam.H(x[:, 1:, :], p), axis=1)
    return cost.g(x[:, 0, :]) + pair - delta * ham


def solve_scheme(w, scheme, *, N=None, sigma=None, tau=None, theta=1.0, tol=None,
                 max_iter=None, check_every=None, seed=None, init_radius=None,
                 activation="tanh"):
    """Run the iteration above on every query point of workload `w` (uniform N).

    Returns dict(V [B], iters, status, x [B, N+1, d], p [B, N, d] (p_j of interval
    [s_j, s_{j+1}]), rx, rp).
    """
    wl, wr = SCHEMES[scheme]
    fam = make_family(w, activation=activation)
    if getattr(fam, "time_dependent", False):
        raise ValueError("a time-dependent H is solved in the backward-Euler Lax form only")
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
    x_all, p_nodes = initial_guess(xq, N, seed, radius, pidx)
    p_all = p_nodes[:, 1:, :].copy()          # interval j <- the draw of node j + 1
    z_all = x_all.copy()
    iters = np.zeros(B, dtype=np.int64)
    status = np.full(B, MAX_ITER, dtype=np.int64)
    rx_all = np.full(B, np.inf)
    rp_all = np.full(B, np.inf)

    act = np.arange(B)
    x, p, z, delta = x_all[act], p_all[act], z_all[act], delta_all[act]
    k = 0
    while act.size and k < max_iter:
        dl = delta[:, None, None]
        lam = sigma * delta[:, None]
        # dual step on every interval, H at the two ends of x^k
        v = p + sigma * (z[:, 1:, :] - z[:, :-1, :])
        p_new = fam.prox_p_mix(x[:, :-1, :], x[:, 1:, :], wl, wr, v, lam)
        x_new = x.copy()
        # x_0: one gradient step on -delta wL H(., p_0), then the prox of g
        v0 = x[:, 0, :] + tau * p_new[:, 0, :]
        if wl:
            v0 = v0 + tau * delta[:, None] * wl * fam.grad_x(x[:, 0, :], p_new[:, 0, :])
        x_new[:, 0, :] = cost.prox(v0, tau)
        # x_j, j = 1..N-1: p_{j-1} on its left interval, p_j on its right one
        if N > 1:
            xj = x[:, 1:N, :]
            pl, pr = p_new[:, 0:N - 1, :], p_new[:, 1:N, :]
            gH = np.zeros_like(xj)
            if wl:
                gH = gH + wl * fam.grad_x(xj, pr)
            if wr:
                gH = gH + wr * fam.grad_x(xj, pl)
            x_new[:, 1:N, :] = xj - tau * (pl - pr) + tau * dl * gH
        z = x_new + theta * (x_new - x)
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
    V = scheme_value(fam, cost, x_all, p_all, delta_all, wl, wr)
    return dict(V=sign * V, iters=iters, status=status, x=x_all, p=sign * p_all,
                rx=rx_all, rp=rp_all)
