"""Algorithm 3 (Lax form for differential games) in FP64, one step at a time,
for the difference-of-norms game of Section 6.2.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

State z = (x, y), x in R^d1 (the minimising player), y in R^d2 (the maximising
one), costates (p, q).  With the dynamics x' = c1(z) alpha, y' = c2(z) beta,
|alpha|, |beta| <= 1, the Hamiltonian is H(z, p, q) = c1(z)|p|_2 - c2(z)|q|_2 and
the discrete problem (Eq. discgenlaxhopfdg) is
    phi(x, y, t) ~ min_q max_p min_x max_y
        g(z_0) + sum_j <p_j, x_j - x_{j-1}> - sum_j <q_j, y_j - y_{j-1}>
        - delta sum_j (c1(z_j)|p_j| - c2(z_j)|q_j|),
with z_N = (x_target, y_target).  The speeds are Section 6.2's:
c1(z) = c0 + a exp(-b |z - z_b|^2) and its mirror c2(z) = c1(-z).

One iteration (Algorithm 3 with one gradient step for each primal block, as in
Section 6.2's runs; H at z^k for the dual steps and the x-step, at
(x^{k+1}, y^k) for the y-step, following the order of the listing):
  p_j <- shrink_2(p_j + sigma (xbar_j - xbar_{j-1}), sigma delta c1(z_j^k))     j = 1..N
  q_j <- shrink_2(q_j + sigma (ybar_j - ybar_{j-1}), sigma delta c2(z_j^k))
  x_0 <- (x_0 + tau p_1 + tau W_x^2 c_x) / (1 + tau W_x^2)              (prox of tau g)
  x_j <- x_j - tau (p_j - p_{j+1}) + tau delta d_x H(z_j^k, p_j, q_j)       j = 1..N-1
  y_0 <- (y_0 + tau q_1 - tau W_y^2 c_y) / (1 - tau W_y^2)     (ascent prox, tau W^2 < 1)
  y_j <- y_j - tau (q_j - q_{j+1}) - tau delta d_y H((x_j^{k+1}, y_j^k), p_j, q_j)
  relax zbar = z^{k+1} + theta (z^{k+1} - z^k)
  stop  |z^{k+1} - z^k|^2 < tol and |(p, q)^{k+1} - (p, q)^k|^2 < tol
  value fval = g(z_0) + sum <p_j, dx_j> - sum <q_j, dy_j> - delta sum (c1|p_j| - c2|q_j|)
Arrays hold z = (x, y) and (p, q) stacked on the coordinate axis.
"""
import numpy as np

from .families import QuadCost
from .lax_pdhg import CONVERGED, MAX_ITER, NONFINITE, VALUE_STOP, initial_guess


class NormsGame:
    """c1(z)|p| - c2(z)|q| with c1(z) = c0 + a exp(-b |z - z_b|^2), c2(z) = c1(-z)."""

    def __init__(self, d1, c0, a, b, zb):
        self.d1 = int(d1)
        self.c0, self.a, self.b = float(c0), float(a), float(b)
        self.zb = np.asarray(zb, dtype=np.float64)

    def speeds(self, z):
        """c1, c2 and their gradients in z."""
        y1, y2 = z - self.zb, z + self.zb
        e1 = np.exp(-self.b * np.sum(y1 * y1, -1))
        e2 = np.exp(-self.b * np.sum(y2 * y2, -1))
        g1 = (-2.0 * self.a * self.b * e1)[..., None] * y1
        g2 = (-2.0 * self.a * self.b * e2)[..., None] * y2
        return self.c0 + self.a * e1, self.c0 + self.a * e2, g1, g2

    def H(self, z, P):
        c1, c2, _, _ = self.speeds(z)
        return c1 * np.linalg.norm(P[..., :self.d1], axis=-1) \
            - c2 * np.linalg.norm(P[..., self.d1:], axis=-1)

    def grad_z(self, z, P):
        _, _, g1, g2 = self.speeds(z)
        return np.linalg.norm(P[..., :self.d1], axis=-1)[..., None] * g1 \
            - np.linalg.norm(P[..., self.d1:], axis=-1)[..., None] * g2


def shrink2(v, t):
    n = np.linalg.norm(v, axis=-1)
    return (np.maximum(n - t, 0.0) / np.where(n > 0, n, 1.0))[..., None] * v


def game_value(game, cost, z, P, delta):
    d1 = game.d1
    dz = z[:, 1:, :] - z[:, :-1, :]
    pair = np.sum(P[:, 1:, :d1] * dz[..., :d1], axis=(1, 2)) \
        - np.sum(P[:, 1:, d1:] * dz[..., d1:], axis=(1, 2))
    ham = np.sum(game.H(z[:, 1:, :], P[:, 1:, :]), axis=1)
    return cost.g(z[:, 0, :]) + pair - delta * ham


def make_game(w):
    dyn = np.asarray(w["dyn"], dtype=np.float64)
    d = int(w["d"])
    return NormsGame(int(dyn[0]), dyn[1], dyn[2], dyn[3], dyn[4:4 + d])


def solve_game(w, *, N=None, sigma=None, tau=None, theta=1.0, tol=None, max_iter=None,
               check_every=None, seed=None, init_radius=None, x_init=None, p_init=None,
               value_tol=0.0):
    """Run Algorithm 3 on every query point (x, y) of workload `w` (uniform N),
    from the random initial guess or from (x_init, p_init) as returned.
    value_tol > 0: the value test of lax_pdhg.solve (status VALUE_STOP).

    Returns dict(V, iters, status, x [B, N+1, d] (z = (x, y)), p [B, N+1, d]
    ((p, q); index 0 is 0), rx, rp) like lax_pdhg.solve.
    """
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
    if x_init is None:
        z_all, P_all = initial_guess(zq, N, seed, radius, pidx)
    else:                                     # resume from returned iterates
        z_all = np.array(x_init, dtype=np.float64)
        P_all = np.array(p_init, dtype=np.float64)
        z_all[:, N, :] = zq
        P_all[:, 0, :] = 0.0
    zb_all = z_all.copy()
    iters = np.zeros(B, dtype=np.int64)
    status = np.full(B, MAX_ITER, dtype=np.int64)
    rx_all = np.full(B, np.inf)
    rp_all = np.full(B, np.inf)
    w2x, w2y = cost.w2[:d1], cost.w2[d1:]
    cx, cy = cost.c[:d1], cost.c[d1:]

    act = np.arange(B)
    z, P, zb, delta = z_all[act], P_all[act], zb_all[act], delta_all[act]
    vprev = np.full(B, np.nan)
    k = 0
    while act.size and k < max_iter:
        dl = delta[:, None]
        c1, c2, _, _ = game.speeds(z[:, 1:, :])
        # dual steps at z^k
        v = P[:, 1:, :] + sigma * (zb[:, 1:, :] - zb[:, :-1, :])
        P_new = np.zeros_like(P)
        P_new[:, 1:, :d1] = shrink2(v[..., :d1], sigma * dl * c1)
        P_new[:, 1:, d1:] = shrink2(v[..., d1:], sigma * dl * c2)
        z_new = z.copy()
        # x-step at z^k
        gx = game.grad_z(z[:, 1:N, :], P_new[:, 1:N, :])[..., :d1]
        z_new[:, 1:N, :d1] = z[:, 1:N, :d1] - tau * (P_new[:, 1:N, :d1] - P_new[:, 2:, :d1]) \
            + tau * delta[:, None, None] * gx
        z_new[:, 0, :d1] = (z[:, 0, :d1] + tau * P_new[:, 1, :d1] + tau * w2x * cx) \
            / (1.0 + tau * w2x)
        # y-step at (x^{k+1}, y^k)
        zmid = np.concatenate([z_new[:, 1:N, :d1], z[:, 1:N, d1:]], axis=-1)
        gy = game.grad_z(zmid, P_new[:, 1:N, :])[..., d1:]
        z_new[:, 1:N, d1:] = z[:, 1:N, d1:] - tau * (P_new[:, 1:N, d1:] - P_new[:, 2:, d1:]) \
            - tau * delta[:, None, None] * gy
        z_new[:, 0, d1:] = (z[:, 0, d1:] + tau * P_new[:, 1, d1:] - tau * w2y * cy) \
            / (1.0 - tau * w2y)
        zb = z_new + theta * (z_new - z)
        rx = np.sum((z_new - z) ** 2, axis=(1, 2))
        rp = np.sum((P_new - P) ** 2, axis=(1, 2))
        z, P = z_new, P_new
        k += 1
        if k % check_every == 0 or k == max_iter:
            bad = ~(np.isfinite(rx) & np.isfinite(rp))
            conv = (rx < tol) & (rp < tol) & ~bad
            vstop = np.zeros_like(conv)
            if value_tol > 0:
                v = game_value(game, cost, z, P, delta)
                vstop = (np.abs(v - vprev) < value_tol) & ~bad & ~conv
                vprev = v
            stop = bad | conv | vstop | (k == max_iter)
            if np.any(stop):
                ids = act[stop]
                z_all[ids], P_all[ids] = z[stop], P[stop]
                iters[ids] = k
                rx_all[ids], rp_all[ids] = rx[stop], rp[stop]
                status[ids] = np.where(bad[stop], NONFINITE,
                                       np.where(conv[stop], CONVERGED,
                                                np.where(vstop[stop], VALUE_STOP, MAX_ITER)))
                keep = ~stop
                act = act[keep]
                z, P, zb, delta = z[keep], P[keep], zb[keep], delta[keep]
                vprev = vprev[keep]
    V = game_value(game, cost, z_all, P_all, delta_all)
    return dict(V=V, iters=iters, status=status, x=z_all, p=P_all, rx=rx_all, rp=rp_all)
