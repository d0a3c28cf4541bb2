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
