"""Pins for the forward-Euler (Eq. disclaxFE) and trapezoid forms of the FP64
oracle (oracle/lax_schemes.py), each against something that is not that oracle:

  * backward-Euler weights reproduce the separately pinned backward-Euler solver
    iterate for iterate (index bookkeeping of the interval costates);
  * state-independent H: every form has the Hopf-Lax closed form;
  * constant-speed eikonal: every form gives the ball-constrained minimum;
  * tanh drift: the value equals direct collocation of the ODE with the
    forward-Euler or trapezoid rule (BFGS on the primal cost);
  * quadcopter: the gradient of the saddle function, written here from Eq.
    disclaxFE with H built from the ODE and differentiated by complex step,
    vanishes at the converged point;
  * linear drift: against the exact value from the continuous Riccati equation,
    both Euler forms converge at first order in delta, their first-order error
    terms cancel in the sum, and the trapezoid form is second order.

No GPU is needed; every case is small.
"""
import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.optimize import minimize

from oracle import lax_pdhg as O
from oracle import lax_schemes as S
from paper_1803_01215_gb300 import workloads as W
from test_oracle_eikonal_pins import _ball_min, _eik
from test_oracle_pins import QC_PAR, _qc_H, _w


@pytest.mark.parametrize("make", [
    lambda: W.tanh_drift(3, B=5, seed=21, N=7),
    lambda: W.quadcopter(B=3, seed=22, N=9, t=0.6),
    lambda: _eik(2, [[0.6, 0.8], [1.6, 0.2]], 0.3, 5, +1, sigma=0.5, xb=[1.0, 1.0]),
])
def test_backward_weights_reproduce_backward_euler(make):
    w = make()
    K = 60
    a = O.solve(w, tol=0.0, max_iter=K, check_every=K)
    b = S.solve_scheme(w, "be", tol=0.0, max_iter=K, check_every=K)
    np.testing.assert_allclose(b["x"], a["x"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(b["p"], a["p"][:, 1:], rtol=0, atol=1e-13)
    np.testing.assert_allclose(b["V"], a["V"], rtol=0, atol=1e-12)


@pytest.mark.parametrize("scheme", ["fe", "trap"])
def test_state_independent_H_closed_form(scheme):
    """H = |p|^2/2 does not see x, so both ends of an interval give the same H and
    every form is the backward-Euler problem: V = sum W^2 (x-c)^2 / (2 (1 + W^2 t))."""
    r = np.random.default_rng(23)
    d, N = 3, 9
    Wt, c = np.array([0.7, 1.0, 1.6]), np.array([0.2, -0.4, 0.0])
    xq = r.uniform(-2, 2, (4, d))
    t = np.array([0.3, 1.0, 1.7, 2.5])
    w = _w("quadratic", d, [], Wt, c, xq, t, N)
    res = S.solve_scheme(w, scheme)
    assert np.all(res["status"] == O.CONVERGED)
    w2 = Wt ** 2
    V = np.sum(w2 * (xq - c) ** 2 / (2 * (1 + w2 * t[:, None])), axis=1)
    np.testing.assert_allclose(res["V"], V, rtol=0, atol=1e-11)


@pytest.mark.parametrize("scheme", ["fe", "trap"])
def test_constant_speed_eikonal_ball_minimum(scheme):
    r = np.random.default_rng(24)
    d, N, t = 3, 8, 0.6
    Wt = np.array([0.6, 1.1, 1.7])
    cc = r.standard_normal(d)
    xq = cc + 1.5 * r.standard_normal((3, d))
    w = _eik(d, xq, t, N, +1, sigma=0.5, c=(1.3, 0.0, 1.0), W=Wt, cc=cc)
    res = S.solve_scheme(w, scheme)
    assert np.all(res["status"] == O.CONVERGED)
    ref = [_ball_min(Wt ** 2, cc, x, t * 1.3) for x in xq]
    np.testing.assert_allclose(res["V"], ref, rtol=0, atol=1e-9)


@pytest.mark.parametrize("scheme", ["fe", "trap"])
def test_tanh_drift_direct_collocation(scheme):
    """f = tanh(Ax) + u, L = |u|^2/2.  Forward Euler steps x_{j+1} = x_j +
    delta (f(x_j) + u_j); the trapezoid rule averages f over the two ends.  With
    cost g(x_0) + delta sum |u_j|^2/2 and x_N = x, minimise over x_0..x_{N-1}."""
    r = np.random.default_rng(25)
    d, N, t = 3, 6, 0.8
    A = r.standard_normal((d, d)) / np.sqrt(d)
    c = r.standard_normal(d)
    xq = r.standard_normal((3, d))
    w = _w("tanh_drift", d, A.reshape(-1), np.ones(d), c, xq, np.full(3, t), N)
    res = S.solve_scheme(w, scheme)
    assert np.all(res["status"] == O.CONVERGED)
    delta = t / N
    for b in range(3):
        def J(z):
            X = np.vstack([z.reshape(N, d), xq[b]])
            fl, fr = np.tanh(X[:-1] @ A.T), np.tanh(X[1:] @ A.T)
            f = fl if scheme == "fe" else 0.5 * (fl + fr)
            u = (X[1:] - X[:-1]) / delta - f
            return 0.5 * np.sum((X[0] - c) ** 2) + 0.5 * delta * np.sum(u * u)
        z0 = np.repeat(xq[b][None], N, 0).ravel()
        opt = minimize(J, z0, method="BFGS", options=dict(gtol=1e-12, maxiter=20000))
        assert abs(opt.fun - res["V"][b]) < 1e-9, (b, opt.fun, res["V"][b])
        np.testing.assert_allclose(opt.x.reshape(N, d), res["x"][b, :N], atol=2e-6)


@pytest.mark.parametrize("scheme", ["fe", "trap"])
def test_quadcopter_saddle_is_stationary(scheme):
    """The saddle function of Eq. disclaxFE (trapezoid: H averaged over the two
    ends of each interval), written here with the H of the ODE, has zero gradient
    in every free x_j (j = 0..N-1) and every p_j (j = 0..N-1) at the oracle's
    converged point."""
    N, t = 8, 0.5
    w = W.quadcopter(B=2, seed=26, N=N, t=t)
    w.update(tol=1e-28, max_iter=200000, check_every=1)
    res = S.solve_scheme(w, scheme)
    assert np.all(res["status"] == O.CONVERGED)
    x, p = res["x"], res["p"]
    delta = t / N
    w2 = w["W"] ** 2
    Hf = lambda xx, pp: _qc_H(xx, pp, *QC_PAR)

    def L(xf, pp):
        X = np.concatenate([xf, x[:, N:N + 1]], axis=1)
        Hs = Hf(X[:, :-1], pp) if scheme == "fe" else 0.5 * (Hf(X[:, :-1], pp) + Hf(X[:, 1:], pp))
        return 0.5 * np.sum(w2 * X[:, 0] ** 2, -1) \
            + np.sum(pp * (X[:, 1:] - X[:, :-1]), axis=(1, 2)) - delta * np.sum(Hs, -1)

    h = 1e-30
    for j in range(N):
        for k in range(12):
            e = np.zeros(x[:, :N].shape, dtype=complex)
            e[:, j, k] = 1j * h
            gx = np.imag(L(x[:, :N] + e, p)) / h
            e = np.zeros(p.shape, dtype=complex)
            e[:, j, k] = 1j * h
            gp = np.imag(L(x[:, :N].astype(complex), p + e)) / h
            assert np.max(np.abs(gx)) < 1e-10 and np.max(np.abs(gp)) < 1e-10, (j, k, gx, gp)


def test_linear_drift_orders_against_continuous_riccati():
    """f = A x + u, L = |u|^2/2, g = 1/2 x^T diag(W^2) x: the exact value is
    1/2 x^T P(t) x with P' = -(P A + A^T P) - P^2, P(0) = diag(W^2).  Both Euler
    forms are first order in delta and their first-order error terms cancel in
    the sum; the trapezoid form is second order."""
    r = np.random.default_rng(27)
    d, t = 3, 1.0
    A = 0.6 * r.standard_normal((d, d))
    Wt = np.array([0.8, 1.3, 1.9])
    xq = r.standard_normal((3, d))
    rhs = lambda s, y: (-(y.reshape(d, d) @ A + A.T @ y.reshape(d, d))
                        - y.reshape(d, d) @ y.reshape(d, d)).ravel()
    sol = solve_ivp(rhs, (0.0, t), np.diag(Wt ** 2).ravel(), method="DOP853",
                    rtol=1e-13, atol=1e-14)
    P = sol.y[:, -1].reshape(d, d)
    Vex = 0.5 * np.einsum("bi,ij,bj->b", xq, P, xq)
    err = {}
    for scheme in ("be", "fe", "trap"):
        e = []
        for N in (8, 16, 32):
            w = _w("tanh_drift", d, A.reshape(-1), Wt, np.zeros(d), xq, np.full(3, t), N,
                   check_every=16)
            res = S.solve_scheme(w, scheme, activation="identity")
            assert np.all(res["status"] == O.CONVERGED)
            e.append(res["V"] - Vex)
        err[scheme] = np.array(e)
    ratio = lambda e: np.log2(np.abs(e[1] / e[2]))              # observed order, N = 16 -> 32
    mx = {s: np.max(np.abs(err[s]), axis=1) for s in err}
    assert 0.7 < ratio(mx["be"]) < 1.3 and 0.7 < ratio(mx["fe"]) < 1.3, (mx["be"], mx["fe"])
    assert np.all(ratio(err["trap"]) > 1.85), err["trap"]
    # the first-order terms of the two Euler forms cancel
    assert np.all(ratio(err["be"] + err["fe"]) > 1.85), err["be"] + err["fe"]
    assert mx["trap"][2] < 0.1 * min(mx["be"][2], mx["fe"][2])
