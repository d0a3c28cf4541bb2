"""Algorithm 3 for the difference-of-norms game with the forward-Euler and
trapezoid discretisations (the averaging Section 7 proposes for the Lax
discretisations of both the control and the game problems), in FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Indexing as in Eq. disclaxFE: costates P_j = (p_j, q_j) of the interval
[s_j, s_{j+1}], j = 0..N-1, states z_j = (x_j, y_j), j = 0..N, z_N = target.
With weights (wL, wR) on the interval's two ends the saddle function is
    g(z_0) + sum_j (<p_j, x_{j+1} - x_j> - <q_j, y_{j+1} - y_j>)
           - delta sum_j (wL H(z_j, P_j) + wR H(z_{j+1}, P_j)),
H(z, p, q) = c1(z)|p| - c2(z)|q|; (1, 0) forward Euler, (1/2, 1/2) trapezoid,
(0, 1) backward Euler (game_pdhg.py with P_j renamed P_{j+1}).

One iteration, Algorithm 3's order with one gradient step per primal block:
  p_j <- shrink_2(p_j + sigma (xbar_{j+1} - xbar_j), sigma delta (wL c1(z_j^k) + wR c1(z_{j+1}^k)))
  q_j <- shrink_2(q_j + sigma (ybar_{j+1} - ybar_j), sigma delta (wL c2(z_j^k) + wR c2(z_{j+1}^k)))
  x_0 <- prox_{tau g_x}(x_0 + tau p_0 + tau delta wL d_x H(z_0^k, P_0))
  x_j <- x_j - tau (p_{j-1} - p_j) + tau delta (wL d_x H(z_j^k, P_j) + wR d_x H(z_j^k, P_{j-1}))
  with m_j = (x_j^{k+1}, y_j^k):
  y_0 <- ascent prox of g_y at y_0 + tau q_0 - tau delta wL d_y H(m_0, P_0)
  y_j <- y_j - tau (q_{j-1} - q_j) - tau delta (wL d_y H(m_j, P_j) + wR d_y H(m_j, P_{j-1}))
  relax, stop and initial guess as in game_pdhg.py (P_j^0: the draw of node j + 1).
"""
import numpy as np

from .families import QuadCost
from .game_pdhg import make_game, shrink2
from .lax_pdhg import CONVERGED, MAX_ITER, NONFINITE, initial_guess
from .lax_schemes import SCHEMES


def game_scheme_value(game, cost, z, P, delta, wl, wr):
    d1 = game.d1
    dz = z[:, 1:, :] - z[:, :-1, :]
    pair = np.sum(P[..., :d1] * dz[..., :d1], axis=(1, 2)) \
        - np.sum(P[..., d1:] * dz[..., d1:], axis=(1, 2))
    ham = np.zeros(z.shape[0])
    if wl:
        ham = ham + wl * np.sum(game.H(z[:, :-1, :], P), axis=1)
    if wr:
        ham = ham + wr * np.sum(game.H(z[:, 1:, :], P), axis=1)
    return cost.g(z[:, 0, :]) + pair - delta * ham


def solve_game_scheme(w, scheme, *, N=None, sigma=None, tau=None, theta=1.0, tol=None,
                      max_iter=None, check_every=None, seed=None, init_radius=None):
    """Returns dict(V, iters, status, x [B, N+1, d] (z), p [B, N, d] ((p, q) per
    interval), rx, rp)."""
    wl, wr = SCHEMES[scheme]
    game = make_game(w)
    d1 = game.d1
    cost = QuadCost(w["W"], w["c"])
    N = int(w["N"] if N is None else N)
    sigma = float(w["sigma"] if sigma is None else sigma)
    tau = float(w["tau"] if tau is None else tau)
    tol = float(w["tol"] if tol is None else tol)
    max_iter = int(w["max_iter"] if max_iter is None else max_iter)
    check_every = int(w["check_every"] if check_every is None else check_every)
    seed = int(w["seed"] if seed is None else seed)
    radius = float(w["init_radius"] if init_radius is None else init_radius)
    if np.any(tau * cost.w2[d1:] >= 1.0):
        raise ValueError("the ascent prox of y_0 needs tau W_y^2 < 1")

    zq = np.asarray(w["xq"], dtype=np.float64)
    B, d = zq.shape
    pidx = w.get("point_index", np.arange(B))
    delta_all = np.asarray(w["t"], dtype=np.float64) / N
    z_all, P_nodes = initial_guess(zq, N, seed, radius, pidx)
    P_all = P_nodes[:, 1:, :].copy()
    zb_all = z_all.copy()
    iters = np.zeros(B, dtype=np.int64)
    status = np.full(B, MAX_ITER, dtype=np.int64)
    rx_all = np.full(B, np.inf)
    rp_all = np.full(B, np.inf)
    w2x, w2y = cost.w2[:d1], cost.w2[d1:]
    cx, cy = cost.c[:d1], cost.c[d1:]

    def gradH(zz, PP):
        return game.grad_z(zz, PP)

    act = np.arange(B)
    z, P, zb, delta = z_all[act], P_all[act], zb_all[act], delta_all[act]
    k = 0
    while act.size and k < max_iter:
        dl = delta[:, None]
        td = tau * delta[:, None, None]
        c1l, c2l, _, _ = game.speeds(z[:, :-1, :])
        c1r, c2r, _, _ = game.speeds(z[:, 1:, :])
        v = P + sigma * (zb[:, 1:, :] - zb[:, :-1, :])
        Pn = np.empty_like(P)
        Pn[..., :d1] = shrink2(v[..., :d1], sigma * dl * (wl * c1l + wr * c1r))
        Pn[..., d1:] = shrink2(v[..., d1:], sigma * dl * (wl * c2l + wr * c2r))
        zn = z.copy()
        # x-block at z^k
        gx0 = gradH(z[:, 0, :], Pn[:, 0, :])[..., :d1] if wl else 0.0
        zn[:, 0, :d1] = (z[:, 0, :d1] + tau * Pn[:, 0, :d1] + tau * delta[:, None] * wl * gx0
                         + tau * w2x * cx) / (1.0 + tau * w2x)
        if N > 1:
            pl, pr = Pn[:, 0:N - 1, :], Pn[:, 1:N, :]
            g = np.zeros_like(z[:, 1:N, :])
            if wl:
                g = g + wl * gradH(z[:, 1:N, :], pr)
            if wr:
                g = g + wr * gradH(z[:, 1:N, :], pl)
            zn[:, 1:N, :d1] = z[:, 1:N, :d1] - tau * (pl[..., :d1] - pr[..., :d1]) + td * g[..., :d1]
        # y-block at m = (x^{k+1}, y^k)
        m = np.concatenate([zn[:, :, :d1], z[:, :, d1:]], axis=-1)
        gy0 = gradH(m[:, 0, :], Pn[:, 0, :])[..., d1:] if wl else 0.0
        zn[:, 0, d1:] = (z[:, 0, d1:] + tau * Pn[:, 0, d1:] - tau * delta[:, None] * wl * gy0
                         - tau * w2y * cy) / (1.0 - tau * w2y)
        if N > 1:
            g = np.zeros_like(z[:, 1:N, :])
            if wl:
                g = g + wl * gradH(m[:, 1:N, :], pr)
            if wr:
                g = g + wr * gradH(m[:, 1:N, :], pl)
            zn[:, 1:N, d1:] = z[:, 1:N, d1:] - tau * (pl[..., d1:] - pr[..., d1:]) - td * g[..., d1:]
        zb = zn + theta * (zn - z)
        rx = np.sum((zn - z) ** 2, axis=(1, 2))
        rp = np.sum((Pn - P) ** 2, axis=(1, 2))
        z, P = zn, Pn
        k += 1
        if k % check_every == 0 or k == max_iter:
            bad = ~(np.isfinite(rx) & np.isfinite(rp))
            conv = (rx < tol) & (rp < tol) & ~bad
            stop = bad | conv | (k == max_iter)
            if np.any(stop):
                ids = act[stop]
                z_all[ids], P_all[ids] = z[stop], P[stop]
                iters[ids] = k
                rx_all[ids], rp_all[ids] = rx[stop], rp[stop]
                status[ids] = np.where(bad[stop], NONFINITE,
                                       np.where(conv[stop], CONVERGED, MAX_ITER))
                keep = ~stop
                act = act[keep]
                z, P, zb, delta = z[keep], P[keep], zb[keep], delta[keep]
    V = game_scheme_value(game, cost, z_all, P_all, delta_all, wl, wr)
    return dict(V=V, iters=iters, status=status, x=z_all, p=P_all, rx=rx_all, rp=rp_all)
