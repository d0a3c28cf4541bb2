"""Pins for the forward-Euler and trapezoid forms of Algorithm 3 for the
difference-of-norms game (oracle/game_schemes.py):

  * backward-Euler weights reproduce the separately pinned game oracle iterate
    for iterate (index bookkeeping of the interval costates);
  * constant speed: every form splits into the min of g_x and the max of g_y
    over balls of radius t c0 (exact for any time discretisation);
  * the paper's 2-D bump game: the saddle function, written here with speeds
    of its own and differentiated by complex step, is stationary at the
    converged point in every free state and every nonzero costate.

No GPU is needed; every case is small.
"""
import numpy as np
import pytest
from scipy.optimize import minimize_scalar

from oracle import game_pdhg as GO
from oracle import game_schemes as GS
from oracle import lax_pdhg as O
from test_oracle_eikonal_pins import _ball_min
from test_oracle_game_pins import _game, _speed


def test_backward_weights_reproduce_the_game_oracle():
    zq = np.array([[-0.5, 0.3], [0.7, 1.2], [1.4, -0.8]])
    w = _game(1, 2, zq, 0.2, 8, W=np.array([0.4, 1.0]), zb=np.array([1.0, 1.0]))
    K = 80
    a = GO.solve_game(w, tol=0.0, max_iter=K, check_every=K)
    b = GS.solve_game_scheme(w, "be", tol=0.0, max_iter=K, check_every=K)
    np.testing.assert_allclose(b["x"], a["x"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(b["p"], a["p"][:, 1:], rtol=0, atol=1e-12)
    np.testing.assert_allclose(b["V"], a["V"], rtol=0, atol=1e-12)


@pytest.mark.parametrize("scheme", ["fe", "trap"])
def test_constant_speed_game_is_scheme_independent(scheme):
    d1, d, t, N, c0 = 2, 4, 0.3, 6, 1.2
    W = np.array([0.7, 1.3, 0.5, 1.1])
    c = np.array([0.4, -0.3, 0.2, 0.1])
    zq = np.array([[1.1, 0.2, 0.6, -0.8], [-0.4, 1.3, -1.0, 0.5]])
    w = _game(d1, d, zq, t, N, sigma=20.0, speed=(c0, 0.0, 4.0), W=W, c=c)
    o = GS.solve_game_scheme(w, scheme)
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


@pytest.mark.parametrize("scheme", ["fe", "trap"])
def test_bump_game_saddle_is_stationary(scheme):
    zb = np.array([1.0, 1.0])
    W = np.array([1 / 2.5, 1.0])
    zq = np.array([[-2.0, 0.3], [0.7, -1.5], [1.5, 1.2]])
    t, N = 0.1, 5
    w = _game(1, 2, zq, t, N, W=W, zb=zb)
    o = GS.solve_game_scheme(w, scheme)
    assert np.all(o["status"] == O.CONVERGED)
    z, P = o["x"], o["p"]
    delta = t / N
    wl, wr = (1.0, 0.0) if scheme == "fe" else (0.5, 0.5)

    def H(zz, PP):
        # |v| written as v sign(Re v): analytic near v != 0, so the complex step applies
        a = lambda v: v * np.sign(np.real(v))
        return _speed(zz, zb) * a(PP[..., 0]) - _speed(zz, -zb) * a(PP[..., 1])

    def L(zf, PP):
        Z = np.concatenate([zf, z[:, N:N + 1]], axis=1)
        dZ = Z[:, 1:] - Z[:, :-1]
        pair = np.sum(PP[..., 0] * dZ[..., 0] - PP[..., 1] * dZ[..., 1], axis=1)
        ham = wl * H(Z[:, :-1], PP) + wr * H(Z[:, 1:], PP)
        return 0.5 * np.sum(W ** 2 * Z[:, 0] ** 2, -1) + pair - delta * np.sum(ham, -1)

    assert np.all(np.abs(P) > 1e-8)
    h = 1e-30
    for j in range(N):
        for k in range(2):
            e = np.zeros(z[:, :N].shape, dtype=complex)
            e[:, j, k] = 1j * h
            gz = np.imag(L(z[:, :N] + e, P.astype(complex))) / h
            e = np.zeros(P.shape, dtype=complex)
            e[:, j, k] = 1j * h
            gp = np.imag(L(z[:, :N].astype(complex), P + e)) / h
            assert np.max(np.abs(gz)) < 1e-9 and np.max(np.abs(gp)) < 1e-9, (j, k, gz, gp)
