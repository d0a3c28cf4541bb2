"""Hamiltonians and terminal cost for the oracle (FP64, numpy, batched).

The paper's convention (Section 2): the control problem runs backwards in
time, x'(s) = f(x, u, s), x(t) = x_target, cost g(x(0)) + int L, so that
H(x, p) = max_u { <f(x, u), p> - L(x, u) } and phi_t + H(x, grad phi) = 0,
phi(x, 0) = g(x).  All three families below have L = |u|^2 / 2 and
control-affine dynamics f = f0(x) + B(x) u, so H = <p, f0> + |B^T p|^2 / 2.

Every array argument has the coordinate axis last: x, p have shape [..., d].
prox_p(x, v, lam) returns argmin_p { lam * H(x, p) + |p - v|^2 / 2 }, the
dual proximal map of Algorithm 1 with lam = sigma * delta.
A time-dependent H (the moving-bump eikonal of Section 6.1) takes the node
time s (shape x.shape[:-1]) as the keyword s; the other families ignore it.
prox_p_mix(xl, xr, wl, wr, v, lam) returns
argmin_p { lam (wl H(xl, p) + wr H(xr, p)) + |p - v|^2 / 2 }, the dual map of
the forward-Euler (wl = 1, wr = 0) and trapezoid (wl = wr = 1/2) forms.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
import numpy as np


class Quadratic:
    """H(x, p) = |p|^2 / 2  (f = u, L = |u|^2/2): the closed-form case."""

    def __init__(self, d):
        self.d = d

    def H(self, x, p, s=None):
        return 0.5 * np.sum(p * p, axis=-1)

    def grad_p(self, x, p, s=None):
        return p.copy()

    def grad_x(self, x, p, s=None):
        return np.zeros_like(p)

    def prox_p(self, x, v, lam, s=None):
        # lam * p + (p - v) = 0
        return v / (1.0 + lam[..., None])

    def prox_p_mix(self, xl, xr, wl, wr, v, lam):
        # lam (wl + wr) p + (p - v) = 0
        return v / (1.0 + (wl + wr) * lam[..., None])


class TanhDrift:
    """H(x, p) = <p, tanh(A x)> + |p|^2 / 2  (f = tanh(Ax) + u, L = |u|^2/2).

    `activation="identity"` gives the linear drift f = Ax + u used by the
    discrete Riccati pin; the tanh form is the high-dimensional workload.
    """

    def __init__(self, A, activation="tanh"):
        self.A = np.asarray(A, dtype=np.float64)
        self.d = self.A.shape[0]
        self.activation = activation

    def _act(self, x):
        y = x @ self.A.T                      # (A x)_i = sum_k A_ik x_k
        if self.activation == "identity":
            return y, np.ones_like(y)
        a = np.tanh(y)
        return a, 1.0 - a * a                 # value and derivative of tanh

    def H(self, x, p, s=None):
        a, _ = self._act(x)
        return np.sum(p * a, axis=-1) + 0.5 * np.sum(p * p, axis=-1)

    def grad_p(self, x, p, s=None):
        a, _ = self._act(x)
        return a + p

    def grad_x(self, x, p, s=None):
        _, da = self._act(x)
        return (da * p) @ self.A              # A^T (tanh'(Ax) * p)

    def prox_p(self, x, v, lam, s=None):
        # lam * (a + p) + (p - v) = 0
        a, _ = self._act(x)
        lam = lam[..., None]
        return (v - lam * a) / (1.0 + lam)

    def prox_p_mix(self, xl, xr, wl, wr, v, lam):
        # lam (wl (a(xl) + p) + wr (a(xr) + p)) + (p - v) = 0
        al, _ = self._act(xl)
        ar, _ = self._act(xr)
        lam = lam[..., None]
        return (v - lam * (wl * al + wr * ar)) / (1.0 + (wl + wr) * lam)


class Quadcopter:
    """12-D quadcopter (Section 6.4 dynamics, thrust measured from hover).

    H(x, p) = <p, f0(x)> + |B(x)^T p|^2 / 2 + eps |p|^2 / 2.
    The last term is an additive full-state disturbance input w with cost
    |w|^2 / (2 eps).  With eps = 0, B has rank 4 in R^12 and H is not bounded
    below in p, which Section 5.1.1 names as the case where the Lax form does
    not converge; eps > 0 makes H strongly convex in p.

    State order follows the paper: (x, y, z, psi, theta, phi) positions and
    Euler angles, then their rates.  With thrust m*a_h + u (a_h = hover gain)
    and torques tau_psi, tau_theta, tau_phi as the four controls:
        f0(x) = (v_pos, v_ang, a_h * a(psi, theta, phi) - g_z e3, 0)
        B(x)  = [ (0_6; a/m; 0_3) | e_10 | e_11 | e_12 ]            (12 x 4)
    with the thrust direction
        a = ( s_phi s_psi + c_phi c_psi s_theta,
             -c_psi s_phi + c_phi s_theta s_psi,
              c_theta c_phi ).
    """

    def __init__(self, m, a_h, g_z, eps):
        self.m, self.a_h, self.g_z = float(m), float(a_h), float(g_z)
        self.eps = float(eps)
        self.d = 12

    @staticmethod
    def thrust_dir(x):
        psi, th, ph = x[..., 3], x[..., 4], x[..., 5]
        sps, cps = np.sin(psi), np.cos(psi)
        sth, cth = np.sin(th), np.cos(th)
        sph, cph = np.sin(ph), np.cos(ph)
        a = np.stack([sph * sps + cph * cps * sth,
                      -cps * sph + cph * sth * sps,
                      cth * cph], axis=-1)
        # J[..., r, c] = d a_r / d (psi, theta, phi)_c
        J = np.empty(x.shape[:-1] + (3, 3), dtype=np.result_type(x, float))
        J[..., 0, 0] = sph * cps - cph * sps * sth
        J[..., 0, 1] = cph * cps * cth
        J[..., 0, 2] = cph * sps - sph * cps * sth
        J[..., 1, 0] = sps * sph + cph * sth * cps
        J[..., 1, 1] = cph * cth * sps
        J[..., 1, 2] = -cps * cph - sph * sth * sps
        J[..., 2, 0] = 0.0
        J[..., 2, 1] = -sth * cph
        J[..., 2, 2] = -cth * sph
        return a, J

    def f0(self, x):
        a, _ = self.thrust_dir(x)
        out = np.zeros_like(x)
        out[..., 0:3] = x[..., 6:9]
        out[..., 3:6] = x[..., 9:12]
        out[..., 6:9] = self.a_h * a
        out[..., 8] -= self.g_z
        return out

    def Bmat(self, x):
        a, _ = self.thrust_dir(x)
        Bm = np.zeros(x.shape[:-1] + (12, 4), dtype=np.result_type(x, float))
        Bm[..., 6:9, 0] = a / self.m
        Bm[..., 9, 1] = 1.0
        Bm[..., 10, 2] = 1.0
        Bm[..., 11, 3] = 1.0
        return Bm

    def H(self, x, p, s=None):
        u = np.einsum("...ik,...i->...k", self.Bmat(x), p)
        return (np.sum(p * self.f0(x), axis=-1) + 0.5 * np.sum(u * u, axis=-1)
                + 0.5 * self.eps * np.sum(p * p, axis=-1))

    def grad_p(self, x, p, s=None):
        Bm = self.Bmat(x)
        u = np.einsum("...ik,...i->...k", Bm, p)
        return self.f0(x) + np.einsum("...ik,...k->...i", Bm, u) + self.eps * p

    def grad_x(self, x, p, s=None):
        a, J = self.thrust_dir(x)
        q = p[..., 6:9]
        u0 = np.sum(a * q, axis=-1) / self.m              # thrust control B_0 . p
        g = np.zeros_like(p)
        # d/d(angles) of  a_h <a, q>  +  (<a, q>/m)^2 / 2
        g[..., 3:6] = (self.a_h + u0 / self.m)[..., None] \
            * np.einsum("...rc,...r->...c", J, q)
        g[..., 6:9] = p[..., 0:3]                          # d/dv_pos of <p_pos, v_pos>
        g[..., 9:12] = p[..., 3:6]                         # d/dv_ang of <p_ang, v_ang>
        return g

    def prox_p(self, x, v, lam, s=None):
        # lam (f0 + B B^T p + eps p) + (p - v) = 0
        #   ->  ((1 + lam eps) I + lam B B^T) p = v - lam f0
        Bm = self.Bmat(x)
        lam = lam[..., None]
        M = (1.0 + lam[..., None] * self.eps) * np.eye(12) \
            + lam[..., None] * np.einsum("...ik,...jk->...ij", Bm, Bm)
        rhs = v - lam * self.f0(x)
        return np.linalg.solve(M, rhs[..., None])[..., 0]

    def prox_p_mix(self, xl, xr, wl, wr, v, lam):
        # lam (wl grad_p H(xl, p) + wr grad_p H(xr, p)) + (p - v) = 0, a linear system
        # with matrix (1 + lam eps (wl + wr)) I + lam (wl B_l B_l^T + wr B_r B_r^T)
        Bl, Br = self.Bmat(xl), self.Bmat(xr)
        lam = lam[..., None]
        BB = wl * np.einsum("...ik,...jk->...ij", Bl, Bl) \
            + wr * np.einsum("...ik,...jk->...ij", Br, Br)
        M = (1.0 + lam[..., None] * self.eps * (wl + wr)) * np.eye(12) + lam[..., None] * BB
        rhs = v - lam * (wl * self.f0(xl) + wr * self.f0(xr))
        return np.linalg.solve(M, rhs[..., None])[..., 0]


class Eikonal:
    """H(x, p, s) = c(x - s v_b) |p|_2 with the speed of Section 6.1,
    c(y) = c0 + c1 exp(-c2 |y - x_b|^2) (a bump of height c1 at x_b on a floor c0).
    v_b (default none: 0) moves the bump with velocity v_b as time s grows,
    Section 6.1's state-and-time-dependent example (v_b = (-1, 1)).

    The dual proximal map is the shrink_2 operator of Section 6.1:
    argmin_p lam c |p| + |p - v|^2 / 2 = v max(|v| - lam c, 0) / |v|.
    grad_x H = |p| grad c; H is not differentiable in p at p = 0, and
    grad_p H is only used away from it.
    """

    def __init__(self, c0, c1, c2, xb, vb=None):
        self.c0, self.c1, self.c2 = float(c0), float(c1), float(c2)
        self.xb = np.asarray(xb, dtype=np.float64)
        self.d = self.xb.shape[0]
        self.vb = None if vb is None or not np.any(vb) else np.asarray(vb, dtype=np.float64)
        self.time_dependent = self.vb is not None

    def speed(self, x, s=None):
        """c and grad c at x (node time s for a moving bump)."""
        y = x - self.xb
        if self.vb is not None:
            y = y - np.asarray(s)[..., None] * self.vb
        e = np.exp(-self.c2 * np.sum(y * y, axis=-1))
        return self.c0 + self.c1 * e, (-2.0 * self.c1 * self.c2 * e)[..., None] * y

    def H(self, x, p, s=None):
        c, _ = self.speed(x, s)
        return c * np.sqrt(np.sum(p * p, axis=-1))

    def grad_p(self, x, p, s=None):
        c, _ = self.speed(x, s)
        n = np.sqrt(np.sum(p * p, axis=-1))
        return np.where(n[..., None] > 0, c[..., None] * p / np.where(n > 0, n, 1.0)[..., None], 0.0)

    def grad_x(self, x, p, s=None):
        _, gc = self.speed(x, s)
        return np.sqrt(np.sum(p * p, axis=-1))[..., None] * gc

    def prox_p(self, x, v, lam, s=None):
        c, _ = self.speed(x, s)
        n = np.sqrt(np.sum(v * v, axis=-1))
        keep = np.maximum(n - lam * c, 0.0) / np.where(n > 0, n, 1.0)
        return keep[..., None] * v

    def prox_p_mix(self, xl, xr, wl, wr, v, lam):
        # (wl c(xl) + wr c(xr)) |p|: shrink_2 with the weighted speed
        if self.time_dependent:
            raise ValueError("the moving bump is solved in the backward-Euler form only")
        cl, _ = self.speed(xl)
        cr, _ = self.speed(xr)
        n = np.sqrt(np.sum(v * v, axis=-1))
        keep = np.maximum(n - lam * (wl * cl + wr * cr), 0.0) / np.where(n > 0, n, 1.0)
        return keep[..., None] * v


class QuadCost:
    """g(x) = 1/2 sum_i W_i^2 (x_i - c_i)^2 (terminal / initial cost).

    sign = -1 gives the concave -g: the eikonal family's negative equation is
    solved as the positive one with initial data -g (Section 6.1), whose
    proximal map ("stretch") needs 1 - tau W_i^2 > 0.
    """

    def __init__(self, W, c, sign=1.0):
        self.w2 = float(sign) * np.asarray(W, dtype=np.float64) ** 2
        self.c = np.asarray(c, dtype=np.float64)

    def g(self, x):
        return 0.5 * np.sum(self.w2 * (x - self.c) ** 2, axis=-1)

    def grad(self, x):
        return self.w2 * (x - self.c)

    def prox(self, v, tau):
        # argmin_x tau*g(x) + |x - v|^2/2  ->  tau w2 (x - c) + x - v = 0
        return (v + tau * self.w2 * self.c) / (1.0 + tau * self.w2)


def make_family(w, activation="tanh"):
    """Oracle Hamiltonian for a workload dict (see workloads.py)."""
    fam, d, dyn = w["family"], w["d"], np.asarray(w["dyn"], dtype=np.float64)
    if fam == "quadratic":
        return Quadratic(d)
    if fam == "tanh_drift":
        return TanhDrift(dyn.reshape(d, d), activation=activation)
    if fam == "quadcopter":
        return Quadcopter(*dyn[:4])
    if fam == "eikonal":
        # dyn = (s, c0, c1, c2, x_b[, v_b]): s = +1 the positive equation, -1 the
        # negative; v_b (optional) the bump's velocity
        vb = dyn[4 + d:4 + 2 * d] if dyn.size >= 4 + 2 * d else None
        return Eikonal(dyn[1], dyn[2], dyn[3], dyn[4:4 + d], vb)
    raise ValueError(fam)
