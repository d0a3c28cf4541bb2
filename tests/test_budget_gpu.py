"""The launch budget of the persistent kernels (hj_solver_opts.time_budget_ms and
iter_budget, the failure-detection budget of the design): once it is used up the
kernel drains its batch, marking every point drawn afterwards HJ_POINT_TIMEOUT
(not iterated, iters = 0, V = NaN), and ends by itself.

A budget is made to run out on purpose: an iteration budget of 1 (exhausted as
soon as the first point finishes) and a time budget of 1 ns.  Every point the
kernel did solve must equal the unbudgeted solve of that point exactly (the
budget only decides which points are drawn for solving).  The batches are
larger than one wave of the persistent grid, so that points are still drawn
after the first ones finish; every kernel family takes part: the register-resident kernel, the tiled and the
shared-memory tanh-drift kernels, the coordinate-parallel eikonal kernel (one
CTA, and a cluster of two CTAs per point), and a ragged plan.  Nothing here waits on the device beyond an ordinary
synchronisation; no kernel spins.
"""
import numpy as np
import pytest

from gpu_common import gpu
from paper_1803_01215_gb300 import workloads as W
from test_parity_gpu import _custom

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TIMEOUT = 5


def _check(g, ref, expect_some_timeout=True):
    st = g["status"]
    timed = st == TIMEOUT
    solved = ~timed
    if expect_some_timeout:
        assert timed.any(), "the budget never ran out"
    assert np.all(g["iters"][timed] == 0) and np.all(np.isnan(g["V"][timed]))
    assert np.array_equal(st[solved], ref["status"][solved])
    assert np.array_equal(g["iters"][solved], ref["iters"][solved])
    assert np.array_equal(g["V"][solved], ref["V"][solved])
    return int(timed.sum()), int(solved.sum())


CASES = [
    ("quadcopter", lambda: W.quadcopter(B=4096, seed=81, N=32, t=0.5), "fp32"),
    ("tanh_d32_tiled", lambda: W.tanh_drift(32, B=2048, seed=82), "fp32"),
    ("tanh_d32_shared", lambda: W.tanh_drift(32, B=1024, seed=83), "fp64"),
    ("eikonal_d37", lambda: W.eikonal(d=37, sign=1, t=0.2, B=8192, seed=84), "fp32"),
    ("eikonal_d1500_cluster", lambda: W.eikonal(d=1500, sign=1, t=0.2, B=400, seed=87), "fp32"),
]


@pytest.mark.parametrize("name,make,precision", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("budget", ["iter", "time"])
def test_budget_drains_the_batch(name, make, precision, budget):
    w = make()
    ref = gpu(w, precision)
    kw = dict(iter_budget=1) if budget == "iter" else dict(time_budget_ms=1e-6)
    g = gpu(w, precision, **kw)
    n_out, n_in = _check(g, ref)
    print(f"{name} {precision} {budget} budget: {n_in} solved, {n_out} drained")
    assert n_in >= 1


def test_generous_budget_changes_nothing():
    w = W.quadcopter(B=512, seed=85, N=32, t=0.5)
    ref = gpu(w, "fp32")
    g = gpu(w, "fp32", time_budget_ms=6.0e4, iter_budget=10 ** 15)
    _check(g, ref, expect_some_timeout=False)
    assert not np.any(g["status"] == TIMEOUT)


def test_ragged_plan_budget():
    from test_ragged_gpu import _plan
    rw = W.ragged_mix(B=3000, seed=86)
    plan, xq, t = _plan(rw, "fp32")
    ref = {k: v.cpu().numpy() for k, v in plan.solve(xq, t).items()}
    # each bucket's launch has its own budget: 1 ns runs out after its first draws
    plan_b, xq_b, t_b = _plan(rw, "fp32", time_budget_ms=1e-6)
    g = {k: v.cpu().numpy() for k, v in plan_b.solve(xq_b, t_b).items()}
    n_out, n_in = _check(g, ref)
    print(f"ragged: {n_in} solved, {n_out} drained")


def test_budget_argument_errors():
    from paper_1803_01215_gb300 import binding
    w = _custom("quadratic", 2, 8, B=3)
    prob = binding.Problem.from_workload(w)
    xq = torch.as_tensor(w["xq"], device="cuda")
    t = torch.as_tensor(w["t"], device="cuda")
    for bad in (dict(time_budget_ms=-1.0), dict(time_budget_ms=float("nan")),
                dict(time_budget_ms=float("inf")), dict(iter_budget=-1)):
        with pytest.raises(binding.HJError) as e:
            binding.solve_batch(prob, xq, t, 8, binding.make_opts(sigma=1.0, tau=0.24, **bad))
        assert e.value.code == binding.HJ_ERR_INVALID_ARG
