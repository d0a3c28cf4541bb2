"""Pins for the eikonal family of the FP64 oracle (Section 6.1: H = +/- c(x)|p|_2,
the shrink_2 dual step, the negative equation through the sign identity),
each against something that is not the oracle.

Constant speed c = c0 makes the discrete problem exact: the max over p_j of
<p_j, x_j - x_{j-1}> - delta c0 |p_j| is 0 when |x_j - x_{j-1}| <= delta c0 and
+inf otherwise, so x_0 ranges over the ball of radius N delta c0 = t c0 around
the query and V = min of g over that ball (positive equation) or, through
phi = -psi, max of g over it (negative equation).

No GPU is needed; every case is small.
"""
import numpy as np
from scipy.optimize import brentq, minimize, minimize_scalar

from oracle import lax_pdhg as O
from oracle.families import Eikonal
from test_oracle_pins import _cs_grad


def _eik(d, xq, t, N, sign, sigma, c=(1.0, 3.0, 4.0), xb=None, W=None, cc=None, tol=1e-22,
         max_iter=200000):
    xb = np.zeros(d) if xb is None else np.asarray(xb, float)
    W = np.ones(d) if W is None else np.asarray(W, float)
    cc = np.zeros(d) if cc is None else np.asarray(cc, float)
    xq = np.atleast_2d(np.asarray(xq, float))
    return dict(family="eikonal", d=d, dyn=np.concatenate([[sign], c, xb]), W=W, c=cc, xq=xq,
                t=np.full(len(xq), float(t)), N=N, sigma=sigma, tau=0.24 / sigma, tol=tol,
                max_iter=max_iter, check_every=8, seed=5, init_radius=0.1)


def test_shrink_prox_stationarity_and_grad_x():
    """|v| > lam c: lam c p/|p| + p - v = 0; |v| <= lam c: p = 0 (0 is in the
    subdifferential).  grad_x H = |p| grad c by complex step of c(x)|p| written out."""
    r = np.random.default_rng(41)
    d = 5
    xb = r.standard_normal(d)
    fam = Eikonal(0.7, 2.0, 1.3, xb)
    x = r.standard_normal((6, d))
    v = r.standard_normal((6, d)) * np.array([3, 3, 3, 0.01, 0.02, 3.0])[:, None]
    lam = np.full(6, 0.4)
    p = fam.prox_p(x, v, lam)
    c = 0.7 + 2.0 * np.exp(-1.3 * np.sum((x - xb) ** 2, -1))
    big = np.linalg.norm(v, axis=1) > lam * c
    assert big.any() and (~big).any()
    n = np.linalg.norm(p[big], axis=1)
    np.testing.assert_allclose(lam[big, None] * c[big, None] * p[big] / n[:, None] + p[big] - v[big],
                               0.0, atol=1e-13)
    assert np.all(p[~big] == 0.0)
    q = r.standard_normal((6, d))
    H = lambda xx: (0.7 + 2.0 * np.exp(-1.3 * np.sum((xx - xb) ** 2, -1))) \
        * np.sqrt(np.sum(q * q, -1))
    np.testing.assert_allclose(fam.grad_x(x, q), _cs_grad(H, x), rtol=1e-12, atol=1e-13)


def _ball_min(q, cc, x, R):
    """min over |y - x| <= R of 1/2 sum q_i (y_i - cc_i)^2, q > 0 (Lagrange multiplier
    mu >= 0: y = (q cc + mu x) / (q + mu))."""
    if np.linalg.norm(cc - x) <= R:
        return 0.0
    y = lambda mu: (q * cc + mu * x) / (q + mu)
    mu = brentq(lambda m: np.linalg.norm(y(m) - x) - R, 0.0, 1e12)
    yy = y(mu)
    return 0.5 * np.sum(q * (yy - cc) ** 2)


def test_constant_speed_positive_is_a_ball_constrained_minimum():
    r = np.random.default_rng(42)
    d, N, t = 3, 8, 0.6
    W = np.array([0.6, 1.1, 1.7])
    cc = r.standard_normal(d)
    xq = cc + 1.5 * r.standard_normal((4, d))
    w = _eik(d, xq, t, N, +1, sigma=0.5, c=(1.3, 0.0, 1.0), W=W, cc=cc)
    o = O.solve(w)
    assert np.all(o["status"] == O.CONVERGED)
    ref = [_ball_min(W ** 2, cc, x, t * 1.3) for x in xq]
    np.testing.assert_allclose(o["V"], ref, rtol=0, atol=1e-9)


def test_constant_speed_negative_is_a_ball_constrained_maximum():
    """Through phi = -psi the negative equation gives max of g over the ball; in
    d = 2 the maximiser lies on the circle, found by a dense angle search."""
    d, N, t, c0 = 2, 6, 0.5, 1.0
    W = np.array([0.4, 1.0])
    xq = np.array([[0.3, 1.2], [-1.0, 0.4], [0.8, -0.9]])
    w = _eik(d, xq, t, N, -1, sigma=100.0, c=(c0, 0.0, 1.0), W=W)
    o = O.solve(w)
    assert np.all(o["status"] == O.CONVERGED)
    R = t * c0
    for b, x in enumerate(xq):
        g = lambda th: 0.5 * np.sum(W ** 2 * (x + R * np.array([np.cos(th), np.sin(th)])) ** 2)
        ths = np.linspace(0, 2 * np.pi, 20001)
        k = int(np.argmax([g(th) for th in ths]))
        opt = minimize_scalar(lambda th: -g(th), bounds=(ths[max(k - 1, 0)], ths[min(k + 1, 20000)]),
                              method="bounded", options=dict(xatol=1e-12))
        assert abs(o["V"][b] - g(opt.x)) < 1e-9, (b, o["V"][b], g(opt.x))


def test_bump_speed_positive_direct_collocation():
    """The paper's speed c(x) = 1 + 3 exp(-4 |x - (1,1)|^2): the primal problem
    min g(x_0) subject to |x_j - x_{j-1}| <= delta c(x_j), x_N = x, solved by SLSQP
    from the oracle-independent straight-line start, matches the oracle's value."""
    d, N, t = 2, 5, 0.3
    W = np.array([1 / 2.5, 1.0])
    xb = np.array([1.0, 1.0])
    xq = np.array([[0.6, 0.8], [1.6, 0.2], [-0.5, 1.4]])
    w = _eik(d, xq, t, N, +1, sigma=0.5, xb=xb, W=W)
    o = O.solve(w)
    assert np.all(o["status"] == O.CONVERGED)
    delta = t / N
    cfun = lambda y: 1.0 + 3.0 * np.exp(-4.0 * np.sum((y - xb) ** 2))
    for b, x in enumerate(xq):
        def unpack(z):
            return np.vstack([z.reshape(N, d), x])
        cons = [{"type": "ineq",
                 "fun": (lambda z, j=j: (delta * cfun(unpack(z)[j])) ** 2
                         - np.sum((unpack(z)[j] - unpack(z)[j - 1]) ** 2))}
                for j in range(1, N + 1)]
        z0 = np.repeat(x[None], N, 0).ravel()
        res = minimize(lambda z: 0.5 * np.sum(W ** 2 * unpack(z)[0] ** 2), z0, method="SLSQP",
                       constraints=cons, options=dict(ftol=1e-15, maxiter=2000))
        assert res.success
        assert abs(res.fun - o["V"][b]) < 1e-7, (b, res.fun, o["V"][b])


def test_moving_bump_direct_collocation():
    """Section 6.1's state-and-time-dependent eikonal, c(x - s(-1, 1)) |p|: the
    primal problem min g(x_0) subject to |x_j - x_{j-1}| <= delta c(x_j - s_j v),
    s_j = j delta, x_N = x, solved by SLSQP from the straight-line start, matches
    the oracle's value (a node time shifted by one step fails it)."""
    d, N, t = 2, 5, 0.4
    W = np.array([1 / 2.5, 1.0])
    xb, vb = np.array([1.0, 1.0]), np.array([-1.0, 1.0])
    xq = np.array([[0.6, 0.8], [1.6, 0.2], [-0.5, 1.4]])
    w = _eik(d, xq, t, N, +1, sigma=0.5, xb=xb, W=W)
    w["dyn"] = np.concatenate([w["dyn"], vb])
    o = O.solve(w)
    assert np.all(o["status"] == O.CONVERGED)
    delta = t / N
    cfun = lambda y, s: 1.0 + 3.0 * np.exp(-4.0 * np.sum((y - s * vb - xb) ** 2))
    for b, x in enumerate(xq):
        def unpack(z):
            return np.vstack([z.reshape(N, d), x])
        cons = [{"type": "ineq",
                 "fun": (lambda z, j=j: (delta * cfun(unpack(z)[j], j * delta)) ** 2
                         - np.sum((unpack(z)[j] - unpack(z)[j - 1]) ** 2))}
                for j in range(1, N + 1)]
        z0 = np.repeat(x[None], N, 0).ravel()
        res = minimize(lambda z: 0.5 * np.sum(W ** 2 * unpack(z)[0] ** 2), z0, method="SLSQP",
                       constraints=cons, options=dict(ftol=1e-15, maxiter=2000))
        assert res.success
        assert abs(res.fun - o["V"][b]) < 1e-7, (b, res.fun, o["V"][b])


def test_zero_velocity_is_the_static_bump():
    w = _eik(2, [[0.6, 0.8], [-1.0, 0.4]], 0.3, 6, +1, sigma=0.5, xb=[1.0, 1.0])
    a = O.solve(w, tol=0.0, max_iter=50, check_every=50)
    w["dyn"] = np.concatenate([w["dyn"], [0.0, 0.0]])
    b = O.solve(w, tol=0.0, max_iter=50, check_every=50)
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["V"], b["V"])
