"""Pins for the FP64 oracle: each test checks the oracle against something that
is not the oracle (a closed form, a textbook recursion, an independent solver,
a definition written from the paper's dynamics), chosen so that a dropped term,
a wrong sign, a wrong time index or a transposed operand fails one of them.

No GPU is needed; every case is small.
"""
import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import lax_pdhg as O
from oracle import counter_rng
from paper_1803_01215_gb300 import workloads as W

TIGHT = 1e-26


def _w(family, d, dyn, Wt, c, xq, t, N, sigma=1.0, **kw):
    base = dict(family=family, d=d, dyn=np.asarray(dyn, dtype=float), W=np.asarray(Wt, float),
                c=np.asarray(c, float), xq=np.atleast_2d(np.asarray(xq, float)),
                t=np.asarray(t, float), N=N, sigma=sigma, tau=0.24 / sigma, tol=TIGHT,
                max_iter=200000, check_every=1, seed=11, init_radius=0.1)
    base.update(kw)
    return base


# ---------------------------------------------------------------- generator
def test_splitmix64_reference_values():
    # splitmix64 seeded with 0: its first three outputs (published reference sequence)
    z = counter_rng.splitmix64_at(0, np.arange(3, dtype=np.uint64))
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_draws_range_and_moments():
    u = counter_rng.uniform_pm1(5, np.arange(2000)[:, None], 0, np.arange(50)[None, :], 3)
    assert u.min() >= -1.0 and u.max() < 1.0
    assert abs(u.mean()) < 0.01 and abs(u.var() - 1.0 / 3.0) < 0.01


def test_initial_guess_matches_section6():
    xq = np.array([[0.3, -1.2, 2.0]])
    x0, p0 = O.initial_guess(xq, 7, seed=3, radius=0.1, point_index=[5])
    assert np.all(np.abs(x0[:, :7] - xq[:, None]) <= 0.1)
    assert np.array_equal(x0[:, 7], xq)
    assert np.all(p0[:, 0] == 0.0) and np.all(np.abs(p0) <= 0.1)
    assert np.std(x0[:, :7] - xq[:, None]) > 0.02      # actually random


# ---------------------------------------------------------------- closed form
@pytest.mark.parametrize("sigma", [0.5, 2.0])
def test_quadratic_closed_form(sigma):
    """H = |p|^2/2, g = 1/2 sum W^2 (x-c)^2: the discrete problem is solved by the
    straight path; V = sum W^2 (x-c)^2 / (2 (1 + W^2 t)) exactly (Hopf-Lax)."""
    r = np.random.default_rng(0)
    d, N = 3, 9
    Wt, c = np.array([0.7, 1.0, 1.6]), np.array([0.2, -0.4, 0.0])
    xq = r.uniform(-2, 2, (5, d))
    t = np.array([0.3, 1.0, 1.7, 0.9, 2.5])
    w = _w("quadratic", d, [], Wt, c, xq, t, N, sigma=sigma)
    res = O.solve(w)
    assert np.all(res["status"] == O.CONVERGED)
    w2 = Wt ** 2
    V = np.sum(w2 * (xq - c) ** 2 / (2 * (1 + w2 * t[:, None])), axis=1)
    np.testing.assert_allclose(res["V"], V, rtol=0, atol=1e-11)
    x0 = (xq + t[:, None] * w2 * c) / (1 + t[:, None] * w2)
    s = np.arange(N + 1)[None, :, None] / N
    np.testing.assert_allclose(res["x"], x0[:, None] + s * (xq - x0)[:, None], atol=1e-10)
    np.testing.assert_allclose(res["p"][:, 1:], np.repeat(((xq - x0) / t[:, None])[:, None], N, 1),
                               atol=1e-10)


# ---------------------------------------------------------------- discrete Riccati
def test_linear_drift_discrete_riccati():
    """f = A x + u, L = |u|^2/2, g = 1/2 x^T P0 x.  Backward Euler gives
    x_{j-1} = M x_j - delta u_j, M = I - delta A, so the dynamic program is
    V_j(x) = 1/2 (Mx)^T P_{j-1}(I + delta P_{j-1})^{-1} (Mx)  (textbook LQR recursion)."""
    r = np.random.default_rng(1)
    d, N, t = 3, 8, 1.3
    A = 0.6 * r.standard_normal((d, d))
    Wt = np.array([0.8, 1.3, 1.9])
    xq = r.standard_normal((4, d))
    w = _w("tanh_drift", d, A.reshape(-1), Wt, np.zeros(d), xq, np.full(4, t), N)
    res = O.solve(w, activation="identity")
    assert np.all(res["status"] == O.CONVERGED)
    delta = t / N
    P = np.diag(Wt ** 2)
    M = np.eye(d) - delta * A
    for _ in range(N):
        P = M.T @ P @ np.linalg.inv(np.eye(d) + delta * P) @ M
    V = 0.5 * np.einsum("bi,ij,bj->b", xq, P, xq)
    np.testing.assert_allclose(res["V"], V, rtol=1e-10, atol=1e-11)


# ---------------------------------------------------------------- tanh drift: direct collocation
def test_tanh_drift_direct_collocation():
    """f = tanh(Ax) + u, L = |u|^2/2.  The primal problem of Eq. (disclaxBE) is
    min over x_0..x_{N-1} of g(x_0) + delta/2 sum |(x_j - x_{j-1})/delta - tanh(A x_j)|^2
    (the max over p written out); minimise it directly with BFGS."""
    r = np.random.default_rng(2)
    d, N, t = 3, 6, 0.8
    A = r.standard_normal((d, d)) / np.sqrt(d)
    c = r.standard_normal(d)
    xq = r.standard_normal((3, d))
    w = _w("tanh_drift", d, A.reshape(-1), np.ones(d), c, xq, np.full(3, t), N)
    res = O.solve(w)
    assert np.all(res["status"] == O.CONVERGED)
    delta = t / N
    for b in range(3):
        def J(z):
            X = np.vstack([z.reshape(N, d), xq[b]])
            u = (X[1:] - X[:-1]) / delta - np.tanh(X[1:] @ A.T)
            return 0.5 * np.sum((X[0] - c) ** 2) + 0.5 * delta * np.sum(u * u)
        z0 = np.repeat(xq[b][None], N, 0).ravel()
        opt = minimize(J, z0, method="BFGS", options=dict(gtol=1e-12, maxiter=20000))
        assert abs(opt.fun - res["V"][b]) < 1e-9
        np.testing.assert_allclose(opt.x.reshape(N, d), res["x"][b, :N], atol=2e-6)


def test_value_independent_of_step_sizes():
    """The fixed point does not depend on sigma, tau (Section 3.2); only the path to it."""
    w = W.tanh_drift(4, B=6, seed=9, N=10)
    w.update(tol=TIGHT, max_iter=200000, check_every=1)
    a = O.solve(w, sigma=0.5, tau=0.24 / 0.5)
    b = O.solve(w, sigma=2.0, tau=0.1)
    np.testing.assert_allclose(a["V"], b["V"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(a["x"], b["x"], atol=1e-9)


# ---------------------------------------------------------------- quadcopter from the paper's ODE
def _qc_dynamics(x, u_thrust, tq, wdist, m, a_h, g_z):
    """Section 6.4's first-order quadcopter system, thrust m*a_h + u_thrust,
    plus the additive disturbance input.  Written coordinate by coordinate."""
    x1, y1, z1, psi, th, phi, x2, y2, z2, psi2, th2, phi2 = [x[..., i] for i in range(12)]
    T = a_h + u_thrust / m
    out = [x2, y2, z2, psi2, th2, phi2,
           T * (np.sin(phi) * np.sin(psi) + np.cos(phi) * np.cos(psi) * np.sin(th)),
           T * (-np.cos(psi) * np.sin(phi) + np.cos(phi) * np.sin(th) * np.sin(psi)),
           T * np.cos(th) * np.cos(phi) - g_z,
           tq[..., 0], tq[..., 1], tq[..., 2]]
    return np.stack(out, axis=-1) + wdist


def _qc_H(x, p, m, a_h, g_z, eps):
    """H = max over (u, tau, w) of <f, p> - |u|^2/2 - |tau|^2/2 - |w|^2/(2 eps).
    f is affine in the controls, so its columns come from differences of f; the
    maximiser of the concave quadratic is (columns . p) scaled by the cost."""
    z1 = np.zeros(x.shape[:-1])
    z3 = np.zeros(x.shape[:-1] + (3,))
    z12 = np.zeros(x.shape[:-1] + (12,))
    f00 = _qc_dynamics(x, z1, z3, z12, m, a_h, g_z)
    b_th = _qc_dynamics(x, z1 + 1.0, z3, z12, m, a_h, g_z) - f00
    u = np.sum(b_th * p, axis=-1)
    tq = p[..., 9:12]
    wd = eps * p
    f = _qc_dynamics(x, u, tq, wd, m, a_h, g_z)
    L = 0.5 * u * u + 0.5 * np.sum(tq * tq, -1) + 0.5 * np.sum(wd * wd, -1) / eps
    return np.sum(f * p, axis=-1) - L


def _cs_grad(fun, x, h=1e-30):
    """Complex-step gradient along the last axis (exact to round-off)."""
    g = np.zeros(x.shape)
    for k in range(x.shape[-1]):
        e = np.zeros(x.shape, dtype=complex)
        e[..., k] = 1j * h
        g[..., k] = np.imag(fun(x + e)) / h
    return g


QC_PAR = (1.0, 9.81, 9.81, 1.0)


def test_quadcopter_H_and_derivatives_match_dynamics():
    from oracle.families import Quadcopter
    r = np.random.default_rng(3)
    x = r.standard_normal((7, 12))
    p = r.standard_normal((7, 12))
    fam = Quadcopter(*QC_PAR)
    np.testing.assert_allclose(fam.H(x, p), _qc_H(x, p, *QC_PAR), rtol=1e-13, atol=1e-12)
    gx = _cs_grad(lambda xx: _qc_H(xx, p, *QC_PAR), x)
    gp = _cs_grad(lambda pp: _qc_H(x, pp, *QC_PAR), p)
    np.testing.assert_allclose(fam.grad_x(x, p), gx, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(fam.grad_p(x, p), gp, rtol=1e-12, atol=1e-12)
    # prox: stationarity lam grad_p H(x, p*) + p* - v = 0
    v = r.standard_normal((7, 12))
    lam = np.full(7, 0.37)
    ps = fam.prox_p(x, v, lam)
    gps = _cs_grad(lambda pp: _qc_H(x, pp, *QC_PAR), ps)
    np.testing.assert_allclose(lam[:, None] * gps + ps - v, 0.0, atol=1e-12)


def test_quadcopter_kkt_and_value_identity():
    """At the converged saddle the discrete characteristic equations hold with
    derivatives of the H built from the ODE, and fval equals the primal cost
    g(x_0) + delta sum L(u_j) with the optimal controls recovered from p_j."""
    w = W.quadcopter(B=3, seed=4, N=12, t=0.5)
    w.update(tol=1e-28, max_iter=200000, check_every=1)
    res = O.solve(w)
    assert np.all(res["status"] == O.CONVERGED)
    x, p = res["x"], res["p"]
    N = 12
    delta = 0.5 / N
    m, a_h, g_z, eps = QC_PAR
    Hf = lambda xx, pp: _qc_H(xx, pp, m, a_h, g_z, eps)
    gp = _cs_grad(lambda pp: Hf(x[:, 1:], pp), p[:, 1:])
    gx = _cs_grad(lambda xx: Hf(xx, p[:, 1:N]), x[:, 1:N])
    w2 = w["W"] ** 2
    np.testing.assert_allclose(x[:, 1:] - x[:, :-1], delta * gp, atol=1e-11)
    np.testing.assert_allclose(p[:, 1], w2 * x[:, 0], atol=1e-11)
    np.testing.assert_allclose(p[:, 2:] - p[:, 1:N], -delta * gx, atol=1e-11)
    # primal cost from the controls that attain the max in H
    z1 = np.zeros(x[:, 1:].shape[:-1])
    z3 = np.zeros(x[:, 1:].shape[:-1] + (3,))
    z12 = np.zeros(x[:, 1:].shape)
    b_th = _qc_dynamics(x[:, 1:], z1 + 1.0, z3, z12, m, a_h, g_z) \
        - _qc_dynamics(x[:, 1:], z1, z3, z12, m, a_h, g_z)
    u = np.sum(b_th * p[:, 1:], -1)
    L = 0.5 * u ** 2 + 0.5 * np.sum(p[:, 1:, 9:12] ** 2, -1) + 0.5 * eps * np.sum(p[:, 1:] ** 2, -1)
    Vp = 0.5 * np.sum(w2 * x[:, 0] ** 2, -1) + delta * np.sum(L, -1)
    np.testing.assert_allclose(res["V"], Vp, rtol=1e-11, atol=1e-11)


# ---------------------------------------------------------------- brute force, tiny
def test_tiny_brute_force_saddle():
    """d = 1, N = 2, tanh drift: the value min over (x_0, x_1) of the primal cost,
    found by dense grid search refined by Nelder-Mead, equals the oracle's fval."""
    A = np.array([[0.9]])
    xq = np.array([[0.7]])
    t = 0.6
    w = _w("tanh_drift", 1, A.reshape(-1), [1.2], [-0.3], xq, [t], 2)
    res = O.solve(w)
    delta = t / 2

    def J(z):
        X = np.array([z[0], z[1], xq[0, 0]])
        u = (X[1:] - X[:-1]) / delta - np.tanh(0.9 * X[1:])
        return 0.5 * 1.44 * (X[0] + 0.3) ** 2 + 0.5 * delta * np.sum(u * u)
    g = np.linspace(-2, 2, 401)
    G = np.array([[J((a, b)) for b in g] for a in g])
    i, j = np.unravel_index(np.argmin(G), G.shape)
    opt = minimize(J, [g[i], g[j]], method="Nelder-Mead",
                   options=dict(xatol=1e-12, fatol=1e-15, maxiter=20000))
    assert abs(opt.fun - res["V"][0]) < 1e-10


# ---------------------------------------------------------------- loop control
def test_stopping_rule_checks_only_every_k():
    w = W.tanh_drift(4, B=5, seed=9, N=10)
    res = O.solve(w, tol=1e-8, check_every=8, max_iter=100000)
    assert np.all(res["status"] == O.CONVERGED)
    assert np.all(res["iters"] % 8 == 0)
    assert np.all(res["rx"] < 1e-8) and np.all(res["rp"] < 1e-8)
    res2 = O.solve(w, tol=1e-8, check_every=8, max_iter=13)
    assert np.all(res2["status"] == O.MAX_ITER) and np.all(res2["iters"] == 13)


def test_warm_start_resumes_the_same_iteration():
    """Restarting from the iterate after k steps with z = x (as Algorithm 1's
    initialisation prescribes) reaches the same fixed point."""
    w = W.tanh_drift(4, B=4, seed=9, N=10)
    w.update(tol=TIGHT, check_every=1, max_iter=200000)
    full = O.solve(w)
    part = O.solve(w, max_iter=40)
    res = O.solve(w, x_init=part["x"], p_init=part["p"])
    np.testing.assert_allclose(res["V"], full["V"], atol=1e-10)
