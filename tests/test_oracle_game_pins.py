"""Pins for the FP64 oracle of the difference-of-norms game (Section 6.2,
Algorithm 3), each against something that is not that oracle.

The converged runs stop at tol 1e-20: with sigma = 50 the dual steps amplify
FP64 rounding, and the squared increments of (p, q) stall near 1e-21.

No GPU is needed; every case is small.
"""
import numpy as np
from scipy.optimize import minimize_scalar

from oracle import game_pdhg as GO
from oracle import lax_pdhg as O
from test_oracle_eikonal_pins import _ball_min


def _game(d1, d, zq, t, N, sigma=50.0, speed=(1.0, 3.0, 4.0), zb=None, W=None, c=None,
          tol=1e-20, max_iter=200000):
    zb = np.zeros(d) if zb is None else np.asarray(zb, float)
    W = np.ones(d) if W is None else np.asarray(W, float)
    c = np.zeros(d) if c is None else np.asarray(c, float)
    zq = np.atleast_2d(np.asarray(zq, float))
    return dict(family="game_norms", d=d, dyn=np.concatenate([[d1], speed, zb]), W=W, c=c,
                xq=zq, t=np.full(len(zq), float(t)), N=N, sigma=sigma, tau=0.24 / sigma,
                tol=tol, max_iter=max_iter, check_every=8, seed=9, init_radius=0.1)


def test_constant_speed_game_decouples_into_ball_min_and_max():
    """a = 0: H = c0 (|p| - |q|) and g separable, so the discrete game splits:
    the minimiser's x_0 ranges over the ball of radius t c0 around x (V gets the
    min of g_x there) and the maximiser's y_0 over the ball around y (the max of
    g_y, found by a dense angle search in two dimensions)."""
    d1, d, t, N, c0 = 2, 4, 0.3, 6, 1.2
    W = np.array([0.7, 1.3, 0.5, 1.1])
    c = np.array([0.4, -0.3, 0.2, 0.1])
    zq = np.array([[1.1, 0.2, 0.6, -0.8], [-0.4, 1.3, -1.0, 0.5], [0.9, -1.2, 0.3, 1.4]])
    w = _game(d1, d, zq, t, N, sigma=20.0, speed=(c0, 0.0, 4.0), W=W, c=c)
    o = GO.solve_game(w)
    assert np.all(o["status"] == O.CONVERGED)
    R = t * c0
    for b, z in enumerate(zq):
        vmin = _ball_min(W[:2] ** 2, c[:2], z[:2], R)
        gy = lambda th: 0.5 * np.sum(W[2:] ** 2 * (z[2:] + R * np.array([np.cos(th), np.sin(th)])
                                                  - c[2:]) ** 2)
        ths = np.linspace(0, 2 * np.pi, 20001)
        k = int(np.argmax([gy(th) for th in ths]))
        opt = minimize_scalar(lambda th: -gy(th), bounds=(ths[max(k - 1, 0)], ths[min(k + 1, 20000)]),
                              method="bounded", options=dict(xatol=1e-12))
        assert abs(o["V"][b] - (vmin + gy(opt.x))) < 1e-9, (b, o["V"][b], vmin + gy(opt.x))


def _speed(z, zb, c0=1.0, a=3.0, b=4.0):
    """c(z) = c0 + a exp(-b |z - z_b|^2), written out for complex-step derivatives."""
    y = z - zb
    return c0 + a * np.exp(-b * np.sum(y * y, -1))


def _cs(f, z, h=1e-30):
    g = np.zeros(z.shape)
    for i in range(z.shape[-1]):
        zz = z.astype(complex)
        zz[..., i] += 1j * h
        g[..., i] = np.imag(f(zz)) / h
    return g


def test_bump_game_discrete_characteristics():
    """The paper's 2-D game (d1 = d2 = 1, bump at (1, 1), mirrored bump for the
    maximiser) at the converged saddle: dx_j = delta c1 sign(p_j),
    dy_j = delta c2 sign(q_j), p_{j+1} - p_j = -delta d_x H, q_{j+1} - q_j = delta d_y H,
    p_1 = d_x g(z_0), q_1 = -d_y g(z_0); speeds and their derivatives written
    independently (complex step).  At a stop of 1e-20 on the squared increments
    the residuals are of order 1e-10."""
    zb = np.array([1.0, 1.0])
    W = np.array([1 / 2.5, 1.0])
    zq = np.array([[-2.0, 0.3], [0.7, -1.5], [1.5, 1.2]])
    t, N = 0.1, 5
    w = _game(1, 2, zq, t, N, W=W, zb=zb)
    o = GO.solve_game(w)
    assert np.all(o["status"] == O.CONVERGED)
    z, P = o["x"], o["p"]
    delta = t / N
    p, q = P[:, 1:, 0], P[:, 1:, 1]
    c1 = _speed(z[:, 1:], zb)
    c2 = _speed(z[:, 1:], -zb)
    assert np.all(np.abs(p) > 1e-8) and np.all(np.abs(q) > 1e-8)
    np.testing.assert_allclose(z[:, 1:, 0] - z[:, :-1, 0], delta * c1 * np.sign(p), rtol=0, atol=1e-9)
    np.testing.assert_allclose(z[:, 1:, 1] - z[:, :-1, 1], delta * c2 * np.sign(q), rtol=0, atol=1e-9)
    Hf = lambda zz: _speed(zz, zb) * np.abs(p[:, :N - 1]) - _speed(zz, -zb) * np.abs(q[:, :N - 1])
    gH = _cs(Hf, z[:, 1:N])
    np.testing.assert_allclose(p[:, 1:] - p[:, :-1], -delta * gH[..., 0], rtol=0, atol=1e-9)
    np.testing.assert_allclose(q[:, 1:] - q[:, :-1], delta * gH[..., 1], rtol=0, atol=1e-9)
    np.testing.assert_allclose(p[:, 0], W[0] ** 2 * z[:, 0, 0], rtol=0, atol=1e-9)
    np.testing.assert_allclose(q[:, 0], -W[1] ** 2 * z[:, 0, 1], rtol=0, atol=1e-9)


def test_seven_dimensional_slice_equals_the_two_dimensional_game():
    """Section 6.2's 7-D case on the slice [-3, 3]^2 x {0}^5 (d1 = 1, bump centre
    (1, 1, 0, ...)): the extra maximiser coordinates have zero target, centre and
    data, so by symmetry they tend to zero and the value is the 2-D one.  The
    maximiser's five extra coordinates sit inside the non-smooth |q| shrink and
    settle slowly, so this comparison stops at 1e-14 and checks V to 1e-7."""
    zb2, W2 = np.array([1.0, 1.0]), np.array([1 / 2.5, 1.0])
    zq2 = np.array([[-0.5, 0.3], [0.7, 1.2]])
    w2 = _game(1, 2, zq2, 0.1, 5, W=W2, zb=zb2)
    zq7 = np.zeros((2, 7))
    zq7[:, :2] = zq2
    W7 = np.full(7, 2.0)
    W7[:2] = W2
    zb7 = np.zeros(7)
    zb7[:2] = zb2
    w7 = _game(1, 7, zq7, 0.1, 5, sigma=20.0, W=W7, zb=zb7, tol=1e-14)
    o2, o7 = GO.solve_game(w2), GO.solve_game(w7)
    assert np.all(o2["status"] == O.CONVERGED) and np.all(o7["status"] == O.CONVERGED)
    np.testing.assert_allclose(o7["V"], o2["V"], rtol=0, atol=1e-7)
