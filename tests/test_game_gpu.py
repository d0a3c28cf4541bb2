"""The difference-of-norms game (Section 6.2, Algorithm 3) on the CUDA path,
through the C ABI, against the FP64 game oracle (pinned by
tests/test_oracle_game_pins.py).

Bars: element-wise after a fixed number of iterations (FP64 1e-10; FP32 1e-4
for z, and for (p, q) 1e-4 sigma / 25, since sigma = 50 multiplies FP32 rounding
of z 50-fold in every dual step), FP64 with the workload's stopping rule (value
1e-9, same iteration counts for most points), FP32 value within 1e-4 of the
converged oracle, and the exact constant-speed value.
"""
import numpy as np
import pytest

from gpu_common import gpu, value_err
from oracle import game_pdhg as GO
from oracle import lax_pdhg as O
from paper_1803_01215_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _w(d, N, B, seed=61):
    w = W.game_norms(d=d, B=B, seed=seed)
    w["N"] = N
    w["t"] = np.full(B, N * W.EIK_DELTA)
    return w


@pytest.mark.parametrize("d,N", [(2, 5), (2, 23), (7, 10), (7, 5)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_game_fixed_iterations_elementwise(d, N, precision):
    w = _w(d, N, 21)
    K = 150
    g = gpu(w, precision, tol=0.0, max_iter=K, check_every=K)
    o = GO.solve_game(w, tol=0.0, max_iter=K, check_every=K)
    assert np.all(g["iters"] == K) and np.all(g["status"] == O.MAX_ITER)
    tol = 1e-10 if precision == "fp64" else 1e-4
    tol_p = tol * max(1.0, w["sigma"] / 25.0) if precision == "fp32" else tol
    ex = np.max(np.abs(g["traj_x"] - o["x"]))
    ep = np.max(np.abs(g["traj_p"] - o["p"]))
    ev = np.max(value_err(g["V"], o["V"]))
    print(f"game d={d} N={N} {precision}: |dz| {ex:.2e} |dpq| {ep:.2e} V {ev:.2e}")
    assert ex <= tol and ep <= tol_p
    assert ev <= (1e-9 if precision == "fp64" else 1e-4)


@pytest.mark.parametrize("d", [2, 7])
def test_game_fp64_same_stop_and_fp32_value(d):
    w = _w(d, 5, 24, seed=62)
    o = GO.solve_game(w)
    g = gpu(w, "fp64")
    conv = o["status"] == O.CONVERGED
    assert np.mean(conv) >= 0.8
    same = (g["iters"] == o["iters"]) & conv
    assert np.mean(same) >= 0.7
    assert value_err(g["V"][same], o["V"][same]).max() <= 1e-9
    # FP32 at the paper's stop against the converged oracle (tol 1e-20: with
    # sigma = 50 FP64 rounding keeps the increments near 1e-21), on the points
    # where the paper's stop itself is within 1e-5 of the converged value
    oc = GO.solve_game(w, tol=1e-20, max_iter=200000, check_every=8)
    g32 = gpu(w, "fp32")
    ok = (oc["status"] == O.CONVERGED) & (g["status"] == O.CONVERGED) \
        & (value_err(g["V"], oc["V"]) <= 1e-5) & (g32["status"] == O.CONVERGED)
    assert np.mean(ok) >= 0.6
    assert value_err(g32["V"][ok], oc["V"][ok]).max() <= 1e-4


def test_constant_speed_game_value():
    """a = 0, d1 = d2 = 1: the minimiser's x_0 ranges over [x - R, x + R] and the
    maximiser's y_0 over [y - R, y + R], R = t c0, so
    V = 1/2 W_x^2 max(|x - c_x| - R, 0)^2 + 1/2 W_y^2 (|y - c_y| + R)^2."""
    w = _w(2, 6, 8, seed=63)
    w["dyn"] = np.array(w["dyn"], dtype=float)
    w["dyn"][2] = 0.0
    w["c"] = np.array([0.2, -0.3])
    g = gpu(w, "fp64", tol=1e-20, check_every=8, max_iter=200000)
    assert np.all(g["status"] == O.CONVERGED)
    R = w["t"][0] * w["dyn"][1]
    x, y = w["xq"][:, 0], w["xq"][:, 1]
    ref = 0.5 * w["W"][0] ** 2 * np.maximum(np.abs(x - w["c"][0]) - R, 0.0) ** 2 \
        + 0.5 * w["W"][1] ** 2 * (np.abs(y - w["c"][1]) + R) ** 2
    np.testing.assert_allclose(g["V"], ref, rtol=0, atol=1e-9)


def test_game_argument_errors():
    from paper_1803_01215_gb300 import binding
    w = _w(2, 5, 3)
    prob = binding.Problem.from_workload(w)
    xq = torch.as_tensor(w["xq"], device="cuda")
    t = torch.as_tensor(w["t"], device="cuda")
    ok = binding.make_opts(sigma=50.0, tau=0.0048, precision="fp64")
    out = binding.solve_batch(prob, xq, t, 5, ok, return_traj=True)
    cases = [
        (binding.make_opts(sigma=50.0, tau=0.0048, formulation="hopf"), 2),   # Lax form only
        (binding.make_opts(sigma=50.0, tau=0.0048, inner_steps=2), 2),         # one gradient step
    ]
    for opts, code in cases:
        with pytest.raises(binding.HJError) as e:
            binding.solve_batch(prob, xq, t, 5, opts)
        assert e.value.code == code
    # the maximiser's ascent prox needs tau W_y^2 < 1 (W_y = 1)
    wy = dict(w)
    wy["W"] = np.array([0.4, 2.5])
    py = binding.Problem.from_workload(wy)
    with pytest.raises(binding.HJError) as e:
        binding.solve_batch(py, xq, t, 5, binding.make_opts(sigma=1.5, tau=0.165))
    assert e.value.code == 3                                 # HJ_ERR_STEP_SIZE
    with pytest.raises(binding.HJError):
        binding.solve_grad(prob, t, 5, "fp64", out["traj_x"], out["traj_p"],
                           torch.ones(3, dtype=torch.float64, device="cuda"))
    w3 = _w(2, 5, 3)
    w3["d"] = 3
    w3["xq"] = np.zeros((3, 3))
    w3["W"] = np.ones(3)
    w3["c"] = np.zeros(3)
    w3["dyn"] = np.concatenate([[1.0, 1.0, 3.0, 4.0], np.zeros(3)])
    p3 = binding.Problem.from_workload(w3)                   # valid, but no kernel for d = 3
    with pytest.raises(binding.HJError) as e:
        binding.solve_batch(p3, torch.zeros(3, 3, dtype=torch.float64, device="cuda"), t, 5, ok)
    assert e.value.code == 2
    bad = dict(w)
    bad["dyn"] = np.array(w["dyn"], dtype=float)
    bad["dyn"][0] = 2.0                                      # d1 must be 1..d-1
    with pytest.raises(binding.HJError):
        binding.Problem.from_workload(bad)
