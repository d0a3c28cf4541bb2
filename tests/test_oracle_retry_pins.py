"""Pins for the retry rounds of the oracle (oracle/retry.py): the paper's
handling of points that reach the iteration cap (Section 6.2: raise sigma by 20
and reset tau from the step-size bound; Section 6.1: rerun the point).

  * no extra round is the plain solve;
  * a fresh round of a point is the plain solve of that point alone with the
    round's seed and steps, its iterations added to the first round's;
  * a warm round is the plain solve resumed from the point's last iterate;
  * retried control points reach the converged saddle value (its value does
    not depend on sigma, tau or the starting point);
  * on Section 6.2's game, raising sigma turns some grid points that hit the
    cap into converged ones, as the paper reports (3 of these 12 within three
    raises; the rest oscillate, which the paper ascribes to non-unique optimal
    trajectories).

No GPU is needed; every case is small.
"""
import numpy as np

from oracle import game_pdhg as GO
from oracle import lax_pdhg as O
from oracle import retry as R
from paper_1803_01215_gb300 import workloads as W


def _td(max_iter=64):
    w = W.tanh_drift(4, B=12, seed=31, N=16)
    w.update(max_iter=max_iter, check_every=16, tol=1e-12)
    return w


def test_no_extra_round_is_the_plain_solve():
    w = _td()
    a = O.solve(w)
    b = R.solve_retry(w, rounds=0, sigma_step=0.5)
    for k in ("V", "iters", "status", "x", "p"):
        assert np.array_equal(a[k], b[k]), k
    assert np.all(b["rounds"] == 0)


def test_fresh_round_is_a_standalone_solve():
    w = _td()
    a = O.solve(w)
    ids = np.where(a["status"] == O.MAX_ITER)[0]
    assert ids.size >= 3
    b = R.solve_retry(w, rounds=1, sigma_step=0.5, step_product=0.24)
    sub = W.subset(w, ids)
    s = O.solve(sub, sigma=w["sigma"] + 0.5, tau=0.24 / (w["sigma"] + 0.5), seed=w["seed"] + 1)
    np.testing.assert_array_equal(b["V"][ids], s["V"])
    np.testing.assert_array_equal(b["x"][ids], s["x"])
    np.testing.assert_array_equal(b["iters"][ids], w["max_iter"] + s["iters"])
    assert np.all(b["rounds"][ids] == 1)
    keep = np.setdiff1d(np.arange(len(a["V"])), ids)
    np.testing.assert_array_equal(b["V"][keep], a["V"][keep])


def test_warm_round_resumes_the_last_iterate():
    w = _td()
    a = O.solve(w)
    ids = np.where(a["status"] == O.MAX_ITER)[0]
    b = R.solve_retry(w, rounds=1, sigma_step=0.0, warm=True)
    s = O.solve(W.subset(w, ids), x_init=a["x"][ids], p_init=a["p"][ids])
    np.testing.assert_array_equal(b["V"][ids], s["V"])
    np.testing.assert_array_equal(b["p"][ids], s["p"])


def test_retried_points_reach_the_converged_value():
    w = _td(max_iter=288)
    ref = O.solve(w, tol=1e-26, max_iter=200000, check_every=1)
    assert np.all(ref["status"] == O.CONVERGED)
    a = O.solve(w)
    assert np.mean(a["status"] == O.MAX_ITER) >= 0.3
    warm = R.solve_retry(w, rounds=4, sigma_step=0.25, step_product=0.24, warm=True)
    assert np.all(warm["status"] == O.CONVERGED) and warm["rounds"].max() >= 1
    np.testing.assert_allclose(warm["V"], ref["V"], rtol=0, atol=1e-6)
    fresh = R.solve_retry(w, rounds=4, sigma_step=-0.1, step_product=0.24)
    ok = fresh["status"] == O.CONVERGED
    assert np.mean(ok) > np.mean(a["status"] == O.CONVERGED) and fresh["rounds"].max() >= 1
    np.testing.assert_allclose(fresh["V"][ok], ref["V"][ok], rtol=0, atol=1e-6)


# Grid points of Section 6.2's 2-D game (t = 0.3, mesh 1/12 on [-3, 3]^2) that
# reach 20 000 iterations at sigma = 50 (found with the oracle, plain solve)
GAME_SLOW = [754, 832, 1339, 1417, 1560, 1781, 1924, 2002, 2067, 2145, 2210, 2223]


def test_game_sigma_raise_converges_slow_points():
    w = W.subset(W.game_norms(d=2, t=0.3), np.array(GAME_SLOW))
    a = GO.solve_game(w)
    assert np.all(a["status"] == O.MAX_ITER)
    b = R.solve_retry(w, rounds=3, sigma_step=20.0, step_product=0.24)
    assert np.mean(b["status"] == O.CONVERGED) >= 0.2
    # a converged point satisfies the stopping rule at its last iterate
    ok = b["status"] == O.CONVERGED
    assert np.all((b["rx"][ok] < w["tol"]) & (b["rp"][ok] < w["tol"]))


def _plain_values(solve, w, ks, **kw):
    return {k: solve(w, tol=0.0, max_iter=k, check_every=k, **kw)["V"] for k in ks}


def test_value_stop_is_the_first_test_with_a_small_value_change():
    """A point stopped by the value test at iteration k moved its value by less
    than value_tol between the tests at k - c and k, and by at least value_tol
    between the tests before (values from plain runs of k, k - c, k - 2c
    iterations)."""
    w = _td(max_iter=4000)
    w["tol"] = 1e-30                              # the residual test never fires
    vt = 1e-5
    o = O.solve(w, value_tol=vt)
    stopped = np.where(o["status"] == O.VALUE_STOP)[0]
    assert stopped.size == len(o["V"])
    c = w["check_every"]
    for b in stopped[:4]:
        k = int(o["iters"][b])
        sub = W.subset(w, np.array([b]))
        ks = [kk for kk in (k, k - c, k - 2 * c) if kk > 0]
        v = _plain_values(O.solve, sub, ks)
        np.testing.assert_allclose(o["V"][b], v[k][0], rtol=0, atol=1e-12)
        assert abs(v[k][0] - v[k - c][0]) < vt
        if k - 2 * c > 0:
            assert abs(v[k - c][0] - v[k - 2 * c][0]) >= vt


def test_value_stop_on_the_game_slow_points():
    """The paper's remedy for points that neither converge nor settle their
    trajectories: after the sigma raises, the last round stops on the value."""
    w = W.subset(W.game_norms(d=2, t=0.3), np.array(GAME_SLOW[:6]))
    b = R.solve_retry(w, rounds=1, sigma_step=20.0, step_product=0.24, value_tol=1e-5)
    assert np.mean(b["status"] == O.VALUE_STOP) >= 0.5
    assert np.all(b["iters"][b["status"] == O.VALUE_STOP] > w["max_iter"])   # in the last round
