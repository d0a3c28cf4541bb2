"""Pins for the FP64 oracle of the Hopf form (Eq. dischopf, the appendix's Hopf
tutorial algorithm): each test checks it against something that is not that
oracle — a closed form, a textbook recursion, the separately written Lax oracle
(same discrete saddle for convex g), an identity between the two value
formulas, or derivatives of the quadcopter H written from its ODE.

No GPU is needed; every case is small.
"""
import numpy as np

from oracle import hopf_pdhg as HO
from oracle import lax_pdhg as O
from oracle.families import QuadCost, make_family
from paper_1803_01215_gb300 import workloads as W
from test_oracle_pins import QC_PAR, _cs_grad, _qc_H, _w


def test_hopf_quadratic_closed_form():
    """H = |p|^2/2, g = 1/2 sum W_i^2 (x_i - c_i)^2: V = sum W^2 (x - c)^2 / (2 (1 + W^2 t)),
    x_0 = grad g*(p_1) = (x + t W^2 c) / (1 + t W^2), p_j constant."""
    r = np.random.default_rng(21)
    d, N = 3, 7
    Wt = np.array([0.7, 1.2, 2.0])
    c = r.standard_normal(d)
    xq = r.standard_normal((5, d))
    t = r.uniform(0.4, 1.6, 5)
    w = _w("quadratic", d, [], Wt, c, xq, t, N, sigma=0.8)
    res = HO.solve_hopf(w)
    assert np.all(res["status"] == O.CONVERGED)
    w2 = Wt ** 2
    V = np.sum(w2 * (xq - c) ** 2 / (2 * (1 + w2 * t[:, None])), axis=1)
    np.testing.assert_allclose(res["V"], V, rtol=0, atol=1e-11)
    x0 = (xq + t[:, None] * w2 * c) / (1 + t[:, None] * w2)
    np.testing.assert_allclose(res["x"][:, 0], x0, atol=1e-10)
    np.testing.assert_allclose(res["p"][:, 1:], np.repeat(((xq - x0) / t[:, None])[:, None], N, 1),
                               atol=1e-10)


def test_hopf_value_formula_equals_lax_formula_at_any_iterate():
    """With x_0 = grad g*(p_1), -g*(p_1) = g(x_0) - <p_1, x_0> (Fenchel equality)
    and summation by parts turns the Hopf objective into the Lax objective, at
    any (x, p), not only at the saddle."""
    r = np.random.default_rng(22)
    w = W.tanh_drift(4, B=3, seed=23)
    N = 9
    fam = make_family(w)
    cost = QuadCost(w["W"] * r.uniform(0.5, 2.0, 4), w["c"])
    x = r.standard_normal((3, N + 1, 4))
    p = r.standard_normal((3, N + 1, 4))
    xq = x[:, N, :]
    delta = r.uniform(0.05, 0.2, 3)
    v_hopf = HO.hopf_value(fam, cost, x, p, xq, delta)
    x_lax = x.copy()
    x_lax[:, 0, :] = cost.c + p[:, 1, :] / cost.w2
    v_lax = O.lax_value(fam, cost, x_lax, p, delta)
    np.testing.assert_allclose(v_hopf, v_lax, rtol=1e-12, atol=1e-12)


def test_hopf_and_lax_reach_the_same_saddle():
    """Convex g: both discrete problems have the same saddle; tanh drift and the
    quadcopter (eps = 1) converge to the same value, trajectory and costate."""
    wt = W.tanh_drift(3, B=4, seed=24)
    wt["N"] = 10
    wq = W.quadcopter(B=3, seed=25, N=12, t=0.5)
    for w in (wt, wq):
        a = O.solve(w, tol=1e-26, max_iter=200000, check_every=8)
        b = HO.solve_hopf(w, tol=1e-26, max_iter=200000, check_every=8)
        assert np.all(a["status"] == O.CONVERGED) and np.all(b["status"] == O.CONVERGED)
        np.testing.assert_allclose(b["V"], a["V"], rtol=0, atol=1e-10)
        np.testing.assert_allclose(b["x"], a["x"], atol=1e-9)
        np.testing.assert_allclose(b["p"][:, 1:], a["p"][:, 1:], atol=1e-9)


def test_hopf_linear_drift_discrete_riccati():
    """f = A x + u: the Hopf value equals the textbook LQR recursion
    P_j = M^T P_{j-1} (I + delta P_{j-1})^{-1} M, M = I - delta A."""
    r = np.random.default_rng(26)
    d, N, t = 3, 8, 1.1
    A = 0.6 * r.standard_normal((d, d))
    Wt = np.array([0.9, 1.4, 1.7])
    xq = r.standard_normal((4, d))
    w = _w("tanh_drift", d, A.reshape(-1), Wt, np.zeros(d), xq, np.full(4, t), N)
    res = HO.solve_hopf(w, activation="identity")
    assert np.all(res["status"] == O.CONVERGED)
    delta = t / N
    P = np.diag(Wt ** 2)
    M = np.eye(d) - delta * A
    for _ in range(N):
        P = M.T @ P @ np.linalg.inv(np.eye(d) + delta * P) @ M
    np.testing.assert_allclose(res["V"], 0.5 * np.einsum("bi,ij,bj->b", xq, P, xq),
                               rtol=1e-10, atol=1e-11)


def test_hopf_first_prox_stationarity_quadcopter():
    """The j = 1 step: sigma grad g*(p) + lam grad_p H(x_1, p) + p - v = 0 at the
    result, with grad_p H by complex step of the H written from the ODE."""
    r = np.random.default_rng(27)
    x = r.standard_normal((5, 12))
    v = r.standard_normal((5, 12))
    Wt = r.uniform(0.5, 2.0, 12)
    c = r.standard_normal(12)
    w = dict(family="quadcopter", d=12, dyn=np.array(QC_PAR), W=Wt, c=c)
    fam = make_family(w)
    cost = QuadCost(Wt, c)
    lam = np.full(5, 0.21)
    sigma = 0.9
    ps = HO.prox_first(fam, cost, x, v, lam, sigma)
    gp = _cs_grad(lambda pp: _qc_H(x, pp, *QC_PAR), ps)
    resid = sigma * (c + ps / Wt ** 2) + lam[:, None] * gp + ps - v
    np.testing.assert_allclose(resid, 0.0, atol=1e-12)


def test_hopf_discrete_characteristics_quadcopter():
    """At the converged Hopf saddle: x_j - x_{j-1} = delta grad_p H(x_j, p_j) for
    j = 1..N with x_0 = grad g*(p_1), and p_{j+1} - p_j = -delta grad_x H(x_j, p_j)
    for j = 1..N-1 (derivatives of the H built from the ODE)."""
    w = W.quadcopter(B=3, seed=28, N=10, t=0.4)
    w.update(tol=1e-28, max_iter=200000, check_every=1)
    res = HO.solve_hopf(w)
    assert np.all(res["status"] == O.CONVERGED)
    x, p = res["x"], res["p"]
    N, delta = 10, 0.4 / 10
    Hf = lambda xx, pp: _qc_H(xx, pp, *QC_PAR)
    gp = _cs_grad(lambda pp: Hf(x[:, 1:], pp), p[:, 1:])
    gx = _cs_grad(lambda xx: Hf(xx, p[:, 1:N]), x[:, 1:N])
    np.testing.assert_allclose(x[:, 0], w["c"] + p[:, 1] / w["W"] ** 2, atol=1e-12)
    np.testing.assert_allclose(x[:, 1:] - x[:, :-1], delta * gp, atol=1e-11)
    np.testing.assert_allclose(p[:, 2:] - p[:, 1:N], -delta * gx, atol=1e-11)
