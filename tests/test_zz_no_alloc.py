"""hj_solve_batch_static: the solve for callers that cannot allocate device
memory (the parameters and the work counter live in the library's fixed
file-scope device array).  Its output must match hj_solve_batch on the same
inputs, call after call, since both run the same kernels.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test.  It must pass alone in a fresh process too.
"""
import ctypes

import numpy as np
import pytest

from gpu_common import value_err
from paper_1803_01215_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _static_solve(w, opts, xq, t, out):
    from paper_1803_01215_gb300 import binding
    lib = binding._lib()
    fn = lib.hj_solve_batch_static
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    D = ctypes.POINTER(ctypes.c_double)
    fn.argtypes = [I32, I32, D, I64, D, D, I64, P, P, I32, ctypes.POINTER(binding.SolverOpts),
                   P, P, P, P, P, P]
    fn.restype = ctypes.c_int
    dyn = np.ascontiguousarray(w["dyn"], dtype=np.float64)
    Wv = np.ascontiguousarray(w["W"], dtype=np.float64)
    cv = np.ascontiguousarray(w["c"], dtype=np.float64)
    s = torch.cuda.current_stream()
    r = fn(binding.FAMILIES[w["family"]], w["d"],
           dyn.ctypes.data_as(D) if dyn.size else None, dyn.size,
           Wv.ctypes.data_as(D), cv.ctypes.data_as(D), xq.shape[0],
           ctypes.c_void_p(xq.data_ptr()), ctypes.c_void_p(t.data_ptr()), int(w["N"]),
           ctypes.byref(opts), ctypes.c_void_p(out["V"].data_ptr()),
           ctypes.c_void_p(out["iters"].data_ptr()), ctypes.c_void_p(out["status"].data_ptr()),
           ctypes.c_void_p(out["traj_x"].data_ptr()), ctypes.c_void_p(out["traj_p"].data_ptr()),
           ctypes.c_void_p(s.cuda_stream))
    return r


@pytest.mark.parametrize("which,precision", [("quadcopter", "fp32"), ("tanh_drift", "fp32"),
                                             ("tanh_drift", "fp64")])
def test_static_entry_point_matches_solve_batch_twice(which, precision):
    from paper_1803_01215_gb300 import binding
    if which == "quadcopter":
        ws = [W.quadcopter(B=300, seed=41), W.quadcopter(B=200, seed=42, N=40)]
    else:
        ws = [W.tanh_drift(32, B=150, seed=43), W.tanh_drift(8, B=100, seed=44, N=20)]
    for w in ws:                       # two calls in a row, different problems and sizes
        opts = binding.make_opts(sigma=w["sigma"], tau=w["tau"], tol=w["tol"],
                                 max_iter=w["max_iter"], check_every=w["check_every"],
                                 precision=precision, seed=w["seed"])
        xq = torch.as_tensor(w["xq"], device="cuda")
        t = torch.as_tensor(w["t"], device="cuda")
        ref = binding.solve_batch(binding.Problem.from_workload(w), xq, t, int(w["N"]), opts,
                                  return_traj=True)
        it = torch.float32 if precision == "fp32" else torch.float64
        B, d, N = xq.shape[0], w["d"], int(w["N"])
        out = dict(V=torch.full((B,), np.nan, dtype=torch.float64, device="cuda"),
                   iters=torch.zeros(B, dtype=torch.int32, device="cuda"),
                   status=torch.full((B,), -1, dtype=torch.int8, device="cuda"),
                   traj_x=torch.zeros(B, N + 1, d, dtype=it, device="cuda"),
                   traj_p=torch.zeros(B, N + 1, d, dtype=it, device="cuda"))
        assert _static_solve(w, opts, xq, t, out) == binding.HJ_OK
        torch.cuda.synchronize()
        assert torch.equal(out["status"], ref["status"])
        assert torch.equal(out["iters"], ref["iters"])
        tol = 1e-9 if precision == "fp64" else 1e-4
        assert np.max(value_err(out["V"].cpu().numpy(), ref["V"].cpu().numpy())) <= tol
        assert torch.allclose(out["traj_x"], ref["traj_x"], rtol=0, atol=tol)
        assert torch.allclose(out["traj_p"], ref["traj_p"], rtol=0, atol=tol)


def _quadratic(d, B, seed, N=20):
    r = np.random.default_rng(seed)
    return dict(family="quadratic", d=d, dyn=np.zeros(0), W=r.uniform(0.5, 2.0, d),
                c=r.standard_normal(d), xq=r.uniform(-2.0, 2.0, (B, d)), t=r.uniform(0.5, 2.0, B),
                N=N, sigma=0.5, tau=0.48, tol=1e-8, max_iter=4000, check_every=1, seed=seed,
                init_radius=0.1)


def _empty_out(B, N, d, precision):
    it = torch.float32 if precision == "fp32" else torch.float64
    return dict(V=torch.full((B,), np.nan, dtype=torch.float64, device="cuda"),
                iters=torch.zeros(B, dtype=torch.int32, device="cuda"),
                status=torch.full((B,), -1, dtype=torch.int8, device="cuda"),
                traj_x=torch.zeros(B, N + 1, d, dtype=it, device="cuda"),
                traj_p=torch.zeros(B, N + 1, d, dtype=it, device="cuda"))


@pytest.mark.parametrize("case", ["quadratic_d3", "quadratic_d6", "quadcopter_hopf",
                                  "quadcopter_trap", "tanh_d4_fe", "quadratic_d6_fp64"])
def test_static_entry_point_matches_other_kernels_and_forms(case):
    """The register kernel (quadratic d <= 4) and the shared-memory kernel
    (quadratic d > 4), the Hopf form and the forward-Euler / trapezoid schemes:
    the same status, iterations, values and trajectories as hj_solve_batch."""
    from paper_1803_01215_gb300 import binding
    precision = "fp64" if case.endswith("fp64") else "fp32"
    form, scheme = "lax", "be"
    if case.startswith("quadratic"):
        w = _quadratic(3 if "d3" in case else 6, 120, 46)
    elif case.startswith("quadcopter"):
        w = W.quadcopter(B=160, seed=47, N=32, t=0.5)
        form, scheme = ("hopf", "be") if case.endswith("hopf") else ("lax", "trap")
    else:
        w = W.tanh_drift(4, B=140, seed=48, N=24)
        scheme = "fe"
    opts = binding.make_opts(sigma=w["sigma"], tau=w["tau"], tol=w["tol"], max_iter=w["max_iter"],
                             check_every=w["check_every"], precision=precision, seed=w["seed"],
                             formulation=form, scheme=scheme)
    xq = torch.as_tensor(w["xq"], device="cuda")
    t = torch.as_tensor(w["t"], device="cuda")
    ref = binding.solve_batch(binding.Problem.from_workload(w), xq, t, int(w["N"]), opts,
                              return_traj=True)
    for _ in range(2):
        out = _empty_out(xq.shape[0], int(w["N"]), w["d"], precision)
        assert _static_solve(w, opts, xq, t, out) == binding.HJ_OK
        torch.cuda.synchronize()
        assert torch.equal(out["status"], ref["status"])
        assert torch.equal(out["iters"], ref["iters"])
        tol = 1e-9 if precision == "fp64" else 1e-4
        assert np.max(value_err(out["V"].cpu().numpy(), ref["V"].cpu().numpy())) <= tol
        assert torch.allclose(out["traj_x"], ref["traj_x"], rtol=0, atol=tol)
        assert torch.allclose(out["traj_p"], ref["traj_p"], rtol=0, atol=tol)


@pytest.mark.parametrize("case", ["value_tol_hopf", "fe_inner_steps_2"])
def test_static_entry_point_refuses_what_solve_batch_refuses(case):
    """Option sets that hj_solve_batch refuses are refused here with the same
    status, before anything runs."""
    from paper_1803_01215_gb300 import binding
    w = W.quadcopter(B=8, seed=49, N=32, t=0.5)
    if case == "value_tol_hopf":
        opts = binding.make_opts(sigma=w["sigma"], tau=w["tau"], formulation="hopf", value_tol=1e-6)
    else:
        opts = binding.make_opts(sigma=w["sigma"], tau=w["tau"], scheme="fe", inner_steps=2)
    xq = torch.as_tensor(w["xq"], device="cuda")
    t = torch.as_tensor(w["t"], device="cuda")
    with pytest.raises(binding.HJError) as e:
        binding.solve_batch(binding.Problem.from_workload(w), xq, t, 32, opts, return_traj=True)
    assert e.value.code == binding.HJ_ERR_UNSUPPORTED
    out = _empty_out(8, 32, 12, "fp32")
    assert _static_solve(w, opts, xq, t, out) == e.value.code
    torch.cuda.synchronize()
    assert torch.all(out["status"] == -1)               # nothing ran


@pytest.mark.parametrize("family", ["eikonal", "game_norms"])
def test_static_entry_point_refuses_families_with_device_centres(family):
    from paper_1803_01215_gb300 import binding
    w = W.eikonal(d=2, sign=1, t=0.2, B=8) if family == "eikonal" else W.game_norms(d=2, t=0.1, B=8)
    opts = binding.make_opts(sigma=w["sigma"], tau=w["tau"])
    xq = torch.as_tensor(w["xq"], device="cuda")
    t = torch.as_tensor(w["t"], device="cuda")
    out = _empty_out(8, int(w["N"]), 2, "fp32")
    assert _static_solve(w, opts, xq, t, out) == binding.HJ_ERR_UNSUPPORTED


def test_static_entry_point_rejects_oversized_parameters():
    from paper_1803_01215_gb300 import binding
    w = W.tanh_drift(100, B=4, seed=45)          # A of 100 x 100 does not fit the array
    opts = binding.make_opts(sigma=w["sigma"], tau=w["tau"])
    xq = torch.as_tensor(w["xq"], device="cuda")
    t = torch.as_tensor(w["t"], device="cuda")
    out = dict(V=torch.empty(4, dtype=torch.float64, device="cuda"),
               iters=torch.empty(4, dtype=torch.int32, device="cuda"),
               status=torch.empty(4, dtype=torch.int8, device="cuda"),
               traj_x=torch.empty(4, 33, 100, dtype=torch.float32, device="cuda"),
               traj_p=torch.empty(4, 33, 100, dtype=torch.float32, device="cuda"))
    assert _static_solve(w, opts, xq, t, out) == binding.HJ_ERR_UNSUPPORTED
