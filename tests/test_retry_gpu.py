"""Retry rounds (hj_solve_batch_retry) on the CUDA path against the retry rounds
of the oracle (oracle/retry.py, pinned by tests/test_oracle_retry_pins.py).

FP64: the same rounds, iteration totals and values (1e-9) for the points whose
every round stops at the same iteration on both sides; FP32: values within 1e-4
of the FP64 oracle for the points both sides converge.
"""
import ctypes

import numpy as np
import pytest

from gpu_common import value_err
from oracle import lax_pdhg as O
from oracle import retry as R
from paper_1803_01215_gb300 import workloads as W
from test_oracle_retry_pins import GAME_SLOW, _td

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run(w, precision, rounds, sigma_step, step_product=0.24, warm=False, value_tol=0.0):
    from paper_1803_01215_gb300 import binding
    prob = binding.Problem.from_workload(w)
    opts = binding.make_opts(sigma=w["sigma"], tau=w["tau"], tol=w["tol"], max_iter=w["max_iter"],
                             check_every=w["check_every"], seed=w["seed"],
                             init_radius=w["init_radius"], precision=precision)
    pol = binding.RetryPolicy(rounds, sigma_step, step_product, int(warm), value_tol)
    xq = torch.as_tensor(w["xq"], device="cuda")
    t = torch.as_tensor(w["t"], device="cuda")
    out = binding.solve_batch_retry(prob, xq, t, int(w["N"]), opts, pol, return_traj=True)
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("warm", [False, True])
def test_retry_fp64_matches_the_oracle_rounds(warm):
    w = _td(max_iter=288)
    step = 0.25 if warm else -0.1
    g = _run(w, "fp64", 4, step, warm=warm)
    o = R.solve_retry(w, rounds=4, sigma_step=step, step_product=0.24, warm=warm)
    assert o["rounds"].max() >= 1
    same = (g["rounds"] == o["rounds"]) & (g["iters"] == o["iters"])
    assert np.mean(same) >= 0.8
    assert np.all(g["status"][same] == o["status"][same])
    assert value_err(g["V"][same], o["V"][same]).max() <= 1e-9
    assert np.max(np.abs(g["traj_x"][same] - o["x"][same])) <= 1e-9


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_game_sigma_raise_on_the_slow_grid_points(precision):
    """These grid points oscillate for 20 000 iterations at sigma = 50, so the
    two sides part ways through rounding long before any stop and cannot be
    compared iterate for iterate.  Instead: raising sigma converges a share of
    them, and every point the GPU reports converged sits where the oracle's
    Algorithm 3 stays: 16 more oracle iterations from the GPU's iterate, at that
    round's steps, keep the x increments under the stopping tolerance and move V
    by at most 1e-4 (restarting the relaxation at z = x perturbs the dual step
    by about sigma |dx|, so the (p, q) increments are not tested)."""
    from oracle import game_pdhg as GO
    w = W.subset(W.game_norms(d=2, t=0.3), np.array(GAME_SLOW))
    g = _run(w, precision, 3, 20.0)
    assert np.all(g["rounds"] >= 1)                       # every one hit the cap at sigma = 50
    ok = np.where(g["status"] == O.CONVERGED)[0]
    assert ok.size >= 0.2 * len(GAME_SLOW)
    for b in ok:
        sub = W.subset(w, np.array([b]))
        sig = w["sigma"] + 20.0 * g["rounds"][b]
        o = GO.solve_game(sub, sigma=sig, tau=0.24 / sig, max_iter=16, check_every=16,
                          x_init=g["traj_x"][b:b + 1].astype(np.float64),
                          p_init=g["traj_p"][b:b + 1].astype(np.float64))
        assert o["rx"][0] < w["tol"], (b, o["rx"], o["rp"])
        assert value_err(g["V"][b:b + 1], o["V"]).max() <= 1e-4, (b, g["V"][b], o["V"])


def test_no_extra_round_is_solve_batch():
    from gpu_common import gpu
    w = _td(max_iter=288)
    a = gpu(w, "fp32")
    b = _run(w, "fp32", 0, 1.0)
    for k in ("V", "iters", "status", "traj_x", "traj_p"):
        assert np.array_equal(a[k], b[k]), k
    assert np.all(b["rounds"] == 0)


def test_retry_argument_errors():
    from paper_1803_01215_gb300 import binding
    w = _td()
    prob = binding.Problem.from_workload(w)
    xq = torch.as_tensor(w["xq"], device="cuda")
    t = torch.as_tensor(w["t"], device="cuda")
    opts = binding.make_opts(sigma=1.0, tau=0.24)
    cases = [(binding.RetryPolicy(-1, 0.0, 0.0, 0, 0.0), 1),   # rounds < 0
             (binding.RetryPolicy(2, 0.0, 0.0, 3, 0.0), 1),    # warm not 0/1
             (binding.RetryPolicy(3, -0.5, 0.0, 0, 0.0), 1),   # sigma_3 < 0
             (binding.RetryPolicy(2, 1.0, 0.3, 0, 0.0), 3),    # 4 sigma tau >= 1
             (binding.RetryPolicy(2, 1.0, 0.0, 0, -1.0), 1)]   # value_tol < 0
    for pol, code in cases:
        with pytest.raises(binding.HJError) as e:
            binding.solve_batch_retry(prob, xq, t, int(w["N"]), opts, pol)
        assert e.value.code == code
    # the retry list holds 32-bit point indices: a batch above 2^31 - 1 points is
    # refused before any output pointer is looked at or anything runs
    pol = binding.RetryPolicy(1, 0.0, 0.0, 0, 0.0)
    r = binding._lib().hj_solve_batch_retry(prob.handle, 2 ** 31, None, None, int(w["N"]),
                                            ctypes.byref(opts), ctypes.byref(pol), None, None,
                                            None, None, None, None, None)
    assert r == binding.HJ_ERR_INVALID_ARG


@pytest.mark.parametrize("family", ["tanh_drift", "quadcopter"])
def test_value_stop_fp64_matches_the_oracle(family):
    """The value test in the kernel (summed by parts on test iterations, one
    group of warps for the 12-D N = 64 problem) stops at the oracle's test."""
    from gpu_common import gpu
    if family == "tanh_drift":
        w = _td(max_iter=4000)
    else:
        w = W.quadcopter(B=24, seed=33, N=64, t=1.0)
        w.update(max_iter=4000)
    w["tol"] = 1e-30                                   # only the value test can stop
    vt = 1e-5
    g = gpu(w, "fp64", value_tol=vt)
    o = O.solve(w, value_tol=vt)
    assert np.all(o["status"] == O.VALUE_STOP)
    assert np.all(g["status"] == O.VALUE_STOP)
    same = g["iters"] == o["iters"]
    assert np.mean(same) >= 0.8
    assert value_err(g["V"][same], o["V"][same]).max() <= 1e-9


def test_value_stop_fp32_and_game_retry():
    from gpu_common import gpu
    w = _td(max_iter=4000)
    w["tol"] = 1e-30
    g = gpu(w, "fp32", value_tol=1e-5)
    o = O.solve(w, value_tol=1e-5)
    assert np.all(g["status"] == O.VALUE_STOP)
    assert np.all(np.abs(g["iters"] - o["iters"]) <= 2 * w["check_every"])
    # the game's slow grid points: sigma raise, then the value test in the last round
    wg = W.subset(W.game_norms(d=2, t=0.3), np.array(GAME_SLOW[:6]))
    r = _run(wg, "fp64", 1, 20.0, value_tol=1e-5)
    assert np.mean(r["status"] == O.VALUE_STOP) >= 0.5
    assert np.all(r["iters"][r["status"] == O.VALUE_STOP] > wg["max_iter"])


def test_value_stop_argument_errors():
    from paper_1803_01215_gb300 import binding
    from test_parity_gpu import _custom
    w = _td()
    prob = binding.Problem.from_workload(w)
    xq = torch.as_tensor(w["xq"], device="cuda")
    t = torch.as_tensor(w["t"], device="cuda")
    for kw, code in ((dict(formulation="hopf"), 2), (dict(scheme="trap"), 2), (dict(), 1)):
        opts = binding.make_opts(sigma=1.0, tau=0.24, value_tol=1e-6 if kw else -1.0, **kw)
        with pytest.raises(binding.HJError) as e:
            binding.solve_batch(prob, xq, t, int(w["N"]), opts)
        assert e.value.code == code
    wt = _custom("tanh_drift", 8, 8, B=3)                # shared-memory kernel: no value test
    pt = binding.Problem.from_workload(wt)
    with pytest.raises(binding.HJError) as e:
        binding.solve_batch(pt, torch.as_tensor(wt["xq"], device="cuda"),
                            torch.as_tensor(wt["t"], device="cuda"), 8,
                            binding.make_opts(sigma=1.0, tau=0.24, value_tol=1e-6))
    assert e.value.code == 2
