"""Pins for the oracle's kkt_residual (the discrete characteristic equations,
the stationarity conditions of Eq. disclaxBE's Lagrangian, Section 4).

Each saddle below is built without the oracle's solver or its residual: from
the closed form of H = |p|^2/2 (Hopf-Lax, exact in the discrete problem), from
the dynamic-programming recursion of a linear-quadratic problem (the optimal
control of each step found by minimisation, not by the characteristic
equations), and from the ball extremum of the constant-speed eikonal problem
(Section 6.1).  The residual must vanish there.  Planted perturbations of one
x_j, one p_j, x_0 and p_N must then move each of the three residual parts by
the size that the equations fix by hand, so that dropping a part, flipping the
sign of a gradient term, or taking the wrong node fails a test.

No GPU is needed.
"""
import numpy as np
import pytest

from oracle import lax_pdhg as O


def _w(family, d, dyn, Wt, c, t, N, B):
    return dict(family=family, d=d, dyn=np.asarray(dyn, dtype=float), W=np.asarray(Wt, float),
                c=np.asarray(c, float), t=np.asarray(t, float), N=N, xq=np.zeros((B, d)))


# ---------------------------------------------------------------- closed-form saddle
def _quadratic_saddle(Wt, c, xq, t, N):
    """H = |p|^2/2, g = 1/2 sum W^2 (x - c)^2: x_0 = (x + t W^2 c) / (1 + t W^2), the
    path is straight and the costate constant, p = W^2 (x_0 - c) = (x - x_0) / t."""
    w2 = Wt ** 2
    x0 = (xq + t[:, None] * w2 * c) / (1 + t[:, None] * w2)
    s = np.arange(N + 1)[None, :, None] / N
    x = x0[:, None] + s * (xq - x0)[:, None]
    p = np.repeat((w2 * (x0 - c))[:, None], N + 1, 1)
    p[:, 0] = 0.0
    return x, p


QW = np.array([0.7, 1.3, 1.6])
QC = np.array([0.2, -0.4, 0.0])
QT = np.array([0.3, 1.0, 1.7, 0.9])
QN = 9


def _quadratic_case():
    r = np.random.default_rng(0)
    xq = r.uniform(-2, 2, (4, 3))
    w = _w("quadratic", 3, [], QW, QC, QT, QN, 4)
    x, p = _quadratic_saddle(QW, QC, xq, QT, QN)
    return w, x, p


def test_closed_form_saddle_has_zero_residual():
    w, x, p = _quadratic_case()
    r1, r2, r3 = O.kkt_residual(w, x, p, parts=True)
    assert max(r1.max(), r2.max(), r3.max()) <= 1e-13
    assert O.kkt_residual(w, x, p).max() <= 1e-13


@pytest.mark.parametrize("what", ["x_j", "p_j", "x_0", "p_N"])
def test_planted_perturbations_closed_form(what):
    """On the closed-form saddle (grad_x H = 0, grad_p H = p): a perturbation eps
    of one coordinate k moves the three parts by
        x_j (0 < j < N):  r1 = eps (nodes j and j+1), r2 = 0, r3 = 0
        p_j (1 < j < N):  r1 = delta eps, r2 = 0, r3 = eps (nodes j-1 and j)
        x_0:              r1 = eps (node 1), r2 = W_k^2 eps, r3 = 0
        p_N:              r1 = delta eps, r2 = 0, r3 = eps (node N-1)."""
    w, x, p = _quadratic_case()
    eps, k, j = 1e-3, 1, 4
    delta = QT / QN
    x, p = x.copy(), p.copy()
    if what == "x_j":
        x[:, j, k] += eps
        want = (np.full(4, eps), np.zeros(4), np.zeros(4))
    elif what == "p_j":
        p[:, j, k] += eps
        want = (delta * eps, np.zeros(4), np.full(4, eps))
    elif what == "x_0":
        x[:, 0, k] += eps
        want = (np.full(4, eps), np.full(4, QW[k] ** 2 * eps), np.zeros(4))
    else:
        p[:, QN, k] += eps
        want = (delta * eps, np.zeros(4), np.full(4, eps))
    got = O.kkt_residual(w, x, p, parts=True)
    for g, e in zip(got, want):
        np.testing.assert_allclose(g, e, rtol=1e-9, atol=1e-13)
    np.testing.assert_allclose(O.kkt_residual(w, x, p), np.maximum(np.maximum(*want[:2]), want[2]),
                               rtol=1e-9, atol=1e-13)


# ---------------------------------------------------------------- Riccati (dynamic programming) saddle
def _lq_saddle(A, Wt, xq, t, N):
    """f = A x + u, L = |u|^2/2, g = 1/2 x^T diag(W^2) x, backward Euler
    x_{j-1} = M x_j - delta u_j with M = I - delta A.  Dynamic programming:
    V_j(x) = min_u V_{j-1}(M x - delta u) + delta |u|^2/2 = 1/2 x^T P_j x.  The
    optimal control of step j minimises that quadratic in u:
    (I + delta P_{j-1}) u = P_{j-1} M x_j.  Walking from x_N = x down to x_0
    gives the optimal path; the costate of interval j is the gradient of the
    value-to-go at its left end, p_j = P_{j-1} x_{j-1} (Section 2: p = grad phi)."""
    d = A.shape[0]
    delta = t / N
    M = np.eye(d) - delta * A
    P = [np.diag(Wt ** 2)]
    for _ in range(N):
        Pj = P[-1]
        P.append(M.T @ Pj @ np.linalg.inv(np.eye(d) + delta * Pj) @ M)
    x = np.zeros((N + 1, d))
    p = np.zeros((N + 1, d))
    x[N] = xq
    for j in range(N, 0, -1):
        Pm = P[j - 1]
        u = np.linalg.solve(np.eye(d) + delta * Pm, Pm @ M @ x[j])
        x[j - 1] = M @ x[j] - delta * u
        p[j] = Pm @ x[j - 1]
    return x, p


def _lq_case():
    r = np.random.default_rng(1)
    d, N, t, B = 3, 8, 1.3, 3
    A = 0.6 * r.standard_normal((d, d))
    Wt = np.array([0.8, 1.3, 1.9])
    xq = r.standard_normal((B, d))
    w = _w("tanh_drift", d, A.reshape(-1), Wt, np.zeros(d), np.full(B, t), N, B)
    xs, ps = zip(*[_lq_saddle(A, Wt, xq[b], t, N) for b in range(B)])
    return w, A, np.stack(xs), np.stack(ps), t / N


def test_riccati_saddle_has_zero_residual():
    w, _, x, p, _ = _lq_case()
    r1, r2, r3 = O.kkt_residual(w, x, p, activation="identity", parts=True)
    assert max(r1.max(), r2.max(), r3.max()) <= 1e-12


def test_planted_perturbations_linear_drift():
    """grad_p H = A x + p and grad_x H = A^T p: a perturbation eps e_k of x_j moves
    r1 by eps |e_k - delta A e_k| at node j and eps at node j+1, and nothing else;
    one of p_j moves r1 by delta eps (node j) and r3 by eps |e_k - delta A^T e_k|
    (node j) and eps (node j-1)."""
    w, A, x, p, delta = _lq_case()
    eps, k, j = 1e-4, 2, 3
    e = np.zeros(3)
    e[k] = 1.0
    xp = x.copy()
    xp[:, j, k] += eps
    r1, r2, r3 = O.kkt_residual(w, xp, p, activation="identity", parts=True)
    np.testing.assert_allclose(r1, eps * max(1.0, np.max(np.abs(e - delta * A @ e))), rtol=1e-6)
    assert r2.max() <= 1e-12 and r3.max() <= 1e-12
    pp = p.copy()
    pp[:, j, k] += eps
    r1, r2, r3 = O.kkt_residual(w, x, pp, activation="identity", parts=True)
    np.testing.assert_allclose(r1, delta * eps, rtol=1e-6)
    assert r2.max() <= 1e-12
    np.testing.assert_allclose(r3, eps * max(1.0, np.max(np.abs(e - delta * A.T @ e))), rtol=1e-6)


# ---------------------------------------------------------------- eikonal at constant speed
def _eik_w(sign, xq, t, N, Wt=1.5, c=0.3, c0=0.8):
    B = len(xq)
    w = _w("eikonal", 1, [sign, c0, 0.0, 4.0, 0.0], [Wt], [c], np.full(B, t), N, B)
    w["xq"] = np.asarray(xq, float)[:, None]
    return w


def _eik_saddle(sign, xq, t, N, Wt=1.5, c=0.3, c0=0.8):
    """d = 1, H = sign c0 |p|, g = W^2 (x - c)^2 / 2.  phi(x, t) is the minimum
    (sign +1) or the maximum (sign -1) of g over [x - t c0, x + t c0] (Section 6.1);
    the characteristic is straight from that extremum x_0 to x, and the costate
    is constant, p = g'(x_0).  With sign +1 and |x - c| <= t c0 the minimum is at
    c, where p = 0 and H is not differentiable in p."""
    xq = np.asarray(xq, float)
    away = np.where(xq >= c, 1.0, -1.0)
    if sign > 0:
        x0 = np.where(np.abs(xq - c) <= t * c0, c, xq - away * t * c0)
    else:
        x0 = xq + away * t * c0
    s = np.arange(N + 1)[None, :] / N
    x = (x0[:, None] + s * (xq - x0)[:, None])[..., None]
    p = np.repeat((Wt ** 2 * (x0 - c))[:, None], N + 1, 1)[..., None]
    p[:, 0] = 0.0
    return x, p


@pytest.mark.parametrize("sign", [1, -1])
def test_eikonal_constant_speed_saddle(sign):
    xq = np.array([-1.7, -0.2, 0.35, 0.9, 2.4])
    t, N = 0.6, 12
    w = _eik_w(sign, xq, t, N)
    x, p = _eik_saddle(sign, xq, t, N)
    if sign > 0:
        assert np.any(p[:, 1:] == 0.0)             # the subdifferential case is exercised
    assert O.kkt_residual(w, x, p).max() <= 1e-14


def test_eikonal_negative_equation_sign_matters():
    """The same constant-speed saddle read with the wrong equation (the positive
    one's costate sign) has a residual of order delta c0, not zero."""
    xq = np.array([-1.7, 0.9, 2.4])
    t, N = 0.6, 12
    x, p = _eik_saddle(-1, xq, t, N)
    r_pos = O.kkt_residual(_eik_w(1, xq, t, N), x, p)
    assert np.all(r_pos >= 0.5 * (t / N) * 0.8)


def test_converged_oracle_solves_have_zero_residual():
    """The residual vanishes at the oracle's own converged saddles for the
    negative eikonal equation with the paper's bump speed (d = 2) and the
    quadcopter (its saddle is pinned against the ODE by complex-step derivatives
    elsewhere): a wrong sign or node in the grad_x H term of r3 would not."""
    from paper_1803_01215_gb300 import workloads as W
    we = W.subset(W.eikonal(d=2, sign=-1, t=0.2, B=6, seed=3), np.arange(6))
    we.update(tol=1e-26, max_iter=400000, check_every=1)
    re = O.solve(we)
    assert np.all(re["status"] == O.CONVERGED)
    r1, r2, r3 = O.kkt_residual(we, re["x"], re["p"], parts=True)
    assert max(r1.max(), r2.max(), r3.max()) <= 1e-9
    wq = W.quadcopter(B=3, seed=4, N=12, t=0.5)
    wq.update(tol=1e-28, max_iter=200000, check_every=1)
    rq = O.solve(wq)
    assert np.all(rq["status"] == O.CONVERGED)
    r1, r2, r3 = O.kkt_residual(wq, rq["x"], rq["p"], parts=True)
    assert max(r1.max(), r2.max(), r3.max()) <= 1e-11
    # a quadcopter node's grad_x H is far from zero, so r3 is not trivially small
    from oracle.families import Quadcopter
    gx = Quadcopter(*wq["dyn"]).grad_x(rq["x"][:, 1:12], rq["p"][:, 1:12])
    assert np.max(np.abs(gx)) > 1e-2
