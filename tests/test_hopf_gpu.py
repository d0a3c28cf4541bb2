"""The Hopf form (Algorithm 2, Eq. dischopf) on the CUDA path, through the C ABI,
against the FP64 Hopf oracle (tests/test_oracle_hopf_pins.py pins it).

Bars, as for the Lax form:
  * element-wise after a fixed number of iterations (tol = 0): FP64 within
    1e-10, FP32 within 1e-4; node 0 of the trajectory is grad g*(p_1);
  * FP64 with the workload's stopping rule: value within 1e-9 * max(1, |V|) and
    the same iteration counts for most points;
  * FP32 against the converged oracle: value within 1e-4 * max(1, |V|),
    trajectory within 1e-3 at the tighter stop.
"""
import numpy as np
import pytest

from gpu_common import CONVERGED_TOL, gpu, value_err
from oracle import hopf_pdhg as HO
from oracle import lax_pdhg as O
from paper_1803_01215_gb300 import workloads as W
from test_parity_gpu import TRAJ_TOL, _custom
from test_ragged_gpu import _groups, _plan, _small_mix

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# every kernel: the register kernel (quadratic, quadcopter, tanh drift d <= 4,
# NPL 1/2 with ragged N), the register-tiled FP32 tanh kernel (d = 13 with a
# partial coordinate tile, N = 21 and 7 with partial node tiles), the
# shared-memory kernel (FP64 tanh drift; H = |p|^2/2 at d = 9)
SHAPES = [
    ("quadratic", 2, 20), ("quadratic", 4, 100), ("quadratic", 9, 12),
    ("quadcopter", 12, 64), ("quadcopter", 12, 23),
    ("tanh_drift", 4, 50), ("tanh_drift", 2, 128),
    ("tanh_drift", 32, 32), ("tanh_drift", 13, 21), ("tanh_drift", 100, 32), ("tanh_drift", 64, 7),
]


def hopf_converged(w, **kw):
    kw.setdefault("tol", CONVERGED_TOL)
    kw.setdefault("check_every", 1)
    kw.setdefault("max_iter", 200000)
    return HO.solve_hopf(w, **kw)


@pytest.mark.parametrize("family,d,N", SHAPES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_hopf_fixed_iterations_elementwise(family, d, N, precision):
    w = _custom(family, d, N, B=37)
    K = 150
    g = gpu(w, precision, tol=0.0, max_iter=K, check_every=K, formulation="hopf")
    o = HO.solve_hopf(w, tol=0.0, max_iter=K, check_every=K)
    assert np.all(g["iters"] == K) and np.all(g["status"] == O.MAX_ITER)
    tol = 1e-10 if precision == "fp64" else 1e-4
    ex = np.max(np.abs(g["traj_x"] - o["x"]))
    ep = np.max(np.abs(g["traj_p"] - o["p"]))
    ev = np.max(value_err(g["V"], o["V"]))
    print(f"hopf {family} d={d} N={N} {precision}: max|dx|={ex:.2e} max|dp|={ep:.2e} V rel={ev:.2e}")
    assert ex <= tol and ep <= tol
    assert ev <= (1e-9 if precision == "fp64" else 1e-4)


@pytest.mark.parametrize("family,d,N,B", [
    ("quadratic", 2, 20, 64), ("quadcopter", 12, 64, 24), ("tanh_drift", 4, 32, 40),
    ("tanh_drift", 32, 32, 12)])
def test_hopf_fp64_same_stop(family, d, N, B):
    w = _custom(family, d, N, B)
    g = gpu(w, "fp64", formulation="hopf")
    o = HO.solve_hopf(w)
    assert np.all(g["status"] == O.CONVERGED)
    same = g["iters"] == o["iters"]
    assert np.mean(same) >= 0.8
    assert value_err(g["V"], o["V"])[same].max() <= 1e-9
    assert np.max(np.abs(g["traj_x"][same] - o["x"][same])) <= 1e-9


@pytest.mark.parametrize("family,d,N,B", [
    ("quadcopter", 12, 64, 24), ("tanh_drift", 32, 32, 12), ("tanh_drift", 100, 32, 5)])
def test_hopf_fp32_against_converged_oracle(family, d, N, B):
    w = _custom(family, d, N, B)
    o = hopf_converged(w)
    assert np.all(o["status"] == O.CONVERGED)
    g = gpu(w, "fp32", formulation="hopf")
    assert np.all(g["status"] == O.CONVERGED)
    assert value_err(g["V"], o["V"]).max() <= 1e-4
    gt = gpu(w, "fp32", tol=TRAJ_TOL(d), formulation="hopf")
    assert value_err(gt["V"], o["V"]).max() <= 1e-4
    ett = max(np.max(np.abs(gt["traj_x"] - o["x"])), np.max(np.abs(gt["traj_p"] - o["p"])))
    assert ett <= 1e-3


def test_hopf_closed_form_on_gpu():
    """H = |p|^2/2, g = |x|^2/2: V = |x|^2 / (2 (1 + t)) and x_0 = x / (1 + t)."""
    w = W.quadratic_closed_form()
    g = gpu(w, "fp64", tol=1e-24, check_every=1, max_iter=20000, formulation="hopf")
    assert np.all(g["status"] == O.CONVERGED)
    exact = np.sum(w["xq"] ** 2, axis=1) / (2.0 * (1.0 + w["t"]))
    np.testing.assert_allclose(g["V"], exact, rtol=0, atol=1e-11)
    np.testing.assert_allclose(g["traj_x"][:, 0], w["xq"] / (1.0 + w["t"][:, None]), atol=1e-9)


def test_hopf_and_lax_reach_the_same_value_on_gpu():
    """Same discrete saddle for convex g: the 12-D workload's values agree between
    the two formulations to the stopping accuracy."""
    w = W.subset(W.quadcopter(), np.arange(256))
    gl = gpu(w, "fp32")
    gh = gpu(w, "fp32", formulation="hopf")
    ok = (gl["status"] == O.CONVERGED) & (gh["status"] == O.CONVERGED)
    assert np.mean(ok) >= 0.99
    assert value_err(gh["V"][ok], gl["V"][ok]).max() <= 1e-4


def test_hopf_envelope_gradient_equals_lax_envelope_gradient():
    """hj_solve_grad on Hopf trajectories (node 0 = grad g*(p_1)) gives the
    derivatives of the same converged value as on Lax trajectories."""
    from paper_1803_01215_gb300 import binding
    w = _custom("quadcopter", 12, 16, B=8, t=0.5)
    prob = binding.Problem.from_workload(w)
    xq = torch.as_tensor(w["xq"], device="cuda")
    t = torch.as_tensor(w["t"], device="cuda")
    wts = torch.full((8,), 1.0 / 8, dtype=torch.float64, device="cuda")
    grads = {}
    for form in ("lax", "hopf"):
        opts = binding.make_opts(sigma=w["sigma"], tau=w["tau"], tol=1e-26, max_iter=200000,
                                 check_every=16, precision="fp64", seed=w["seed"],
                                 formulation=form)
        out = binding.solve_batch(prob, xq, t, 16, opts, return_traj=True)
        assert np.all(out["status"].cpu().numpy() == O.CONVERGED)
        grads[form] = {k: v.cpu().numpy() for k, v in
                       binding.solve_grad(prob, t, 16, "fp64", out["traj_x"], out["traj_p"],
                                          wts).items()}
    for k in ("dW", "dc", "ddyn", "dxq"):
        np.testing.assert_allclose(grads["hopf"][k], grads["lax"][k], rtol=1e-7, atol=1e-9)


def test_hopf_argument_errors():
    from paper_1803_01215_gb300 import binding
    w = _custom("tanh_drift", 4, 8, B=3)
    w["W"] = np.array([1.0, 0.0, 1.0, 1.0])          # g* infinite: the Hopf form is undefined
    prob = binding.Problem.from_workload(w)
    xq = torch.as_tensor(w["xq"], device="cuda")
    t = torch.as_tensor(w["t"], device="cuda")
    lax = binding.make_opts(sigma=1.0, tau=0.24, precision="fp64")
    binding.solve_batch(prob, xq, t, 8, lax)
    with pytest.raises(binding.HJError):
        binding.solve_batch(prob, xq, t, 8, binding.make_opts(sigma=1.0, tau=0.24,
                                                              formulation="hopf"))
    bad = binding.make_opts(sigma=1.0, tau=0.24)
    bad.formulation = 7
    with pytest.raises(binding.HJError):
        binding.solve_batch(prob, xq, t, 8, bad)
    # the reverse sweep differentiates the Lax iteration only
    wq = _custom("quadcopter", 12, 8, B=2)
    pq = binding.Problem.from_workload(wq)
    oq = binding.make_opts(sigma=1.0, tau=0.24, formulation="hopf", precision="fp64")
    xqq = torch.as_tensor(wq["xq"], device="cuda")
    tq = torch.as_tensor(wq["t"], device="cuda")
    out = binding.solve_batch(pq, xqq, tq, 8, oq)
    with pytest.raises(binding.HJError):
        binding.solve_grad_unrolled(pq, xqq, tq, 8, oq, out["iters"],
                                    torch.ones(2, dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_hopf_ragged_fixed_iterations_elementwise(precision):
    rw = _small_mix(B=60, seed=31, fp64=precision == "fp64")
    K = 40
    plan, xq, t = _plan(rw, precision, tol=0.0, max_iter=K, check_every=K, formulation="hopf")
    out = {k: v.cpu().numpy() for k, v in plan.solve(xq, t, return_traj=True).items()}
    assert np.all(out["iters"] == K)
    tol = 1e-10 if precision == "fp64" else 1e-4
    for k, N in _groups(rw):
        g = W.ragged_group(rw, k, N)
        o = HO.solve_hopf(g, tol=0.0, max_iter=K, check_every=K)
        for i, b in enumerate(g["point_index"]):
            assert np.max(np.abs(plan.point_traj(out["traj_x"], b) - o["x"][i])) <= tol, (k, N, b)
            assert np.max(np.abs(plan.point_traj(out["traj_p"], b) - o["p"][i])) <= tol, (k, N, b)
        assert np.max(value_err(out["V"][g["point_index"]], o["V"])) <= \
            (1e-9 if precision == "fp64" else 1e-4)
