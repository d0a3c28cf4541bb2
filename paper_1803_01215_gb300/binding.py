"""ctypes binding of libhjpdhg.so (include/hjpdhg.h): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels; this module turns
torch tensors into pointers and status codes into exceptions.  If the library
is not built, loading fails loudly: there is no CPU fallback.
"""
import ctypes
import os

import numpy as np
import torch

from . import build_lib
from .workloads import FAMILIES

HJ_OK, HJ_ERR_INVALID_ARG, HJ_ERR_UNSUPPORTED, HJ_ERR_STEP_SIZE, HJ_ERR_CUDA, HJ_ERR_OOM = range(6)
PREC = {"fp32": 0, "fp64": 1}
POINT_CONVERGED, POINT_MAX_ITER, POINT_NONFINITE = 0, 1, 2
POINT_TIMEOUT = 5


class HJError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {_lib().hj_status_str(code).decode()} (status {code})")
        self.code = code


class SolverOpts(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("tau", ctypes.c_double),
                ("theta", ctypes.c_double), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("inner_steps", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("init_radius", ctypes.c_double),
                ("point_offset", ctypes.c_int64), ("formulation", ctypes.c_int32),
                ("scheme", ctypes.c_int32), ("value_tol", ctypes.c_double),
                ("time_budget_ms", ctypes.c_double), ("iter_budget", ctypes.c_int64)]


_LIB = None
EXPORTED = ("hj_problem_create", "hj_problem_destroy", "hj_solve_batch",
            "hj_set_launch_shape", "hj_get_launch_shape", "hj_autotune",
            "hj_ragged_plan_create", "hj_ragged_plan_layout", "hj_ragged_plan_bucket",
            "hj_ragged_solve", "hj_ragged_autotune", "hj_ragged_plan_destroy",
            "hj_solve_grad", "hj_solve_grad_unrolled", "hj_solve_batch_static",
            "hj_static_scratch_bytes", "hj_probe_fp32_fma", "hj_solve_batch_retry",
            "hj_kkt_residual", "hj_shapes_save", "hj_shapes_load", "hj_status_str", "hj_version")


def _lib():
    global _LIB
    if _LIB is None:
        path = build_lib.lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with "
                               "`python -m paper_1803_01215_gb300.build_lib` (no CPU fallback)")
        lib = ctypes.CDLL(path)
        P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
        lib.hj_problem_create.argtypes = [ctypes.POINTER(P), I32, I32, D, I64, D, D]
        lib.hj_problem_destroy.argtypes = [P]
        lib.hj_solve_batch.argtypes = [P, I64, P, P, I32, ctypes.POINTER(SolverOpts),
                                       P, P, P, P, P, P, P, P, P]
        lib.hj_kkt_residual.argtypes = [P, I64, P, I32, I32, P, P, P, P]
        lib.hj_kkt_residual.restype = ctypes.c_int
        lib.hj_shapes_save.argtypes = [P, ctypes.c_char_p]
        lib.hj_shapes_save.restype = ctypes.c_int
        lib.hj_shapes_load.argtypes = [P, ctypes.c_char_p, ctypes.POINTER(I32)]
        lib.hj_shapes_load.restype = ctypes.c_int
        lib.hj_set_launch_shape.argtypes = [P, I32, I32, I32, I32]
        lib.hj_get_launch_shape.argtypes = [P, I32, I32, ctypes.POINTER(I32), ctypes.POINTER(I32)]
        lib.hj_autotune.argtypes = [P, I64, P, P, I32, ctypes.POINTER(SolverOpts), I32,
                                    ctypes.POINTER(I32), ctypes.POINTER(I32),
                                    ctypes.POINTER(ctypes.c_float), P]
        for name in ("hj_set_launch_shape", "hj_get_launch_shape", "hj_autotune"):
            getattr(lib, name).restype = ctypes.c_int
        PI32, PI64 = ctypes.POINTER(I32), ctypes.POINTER(I64)
        lib.hj_ragged_plan_create.argtypes = [ctypes.POINTER(P), I32, ctypes.POINTER(P), I64,
                                              PI32, PI32, ctypes.POINTER(SolverOpts)]
        lib.hj_ragged_plan_layout.argtypes = [P, PI64, PI64, PI32]
        lib.hj_ragged_plan_bucket.argtypes = [P, I32, PI32, PI32, PI64, PI32, PI32, PI32]
        lib.hj_ragged_solve.argtypes = [P, P, P, P, P, P, P, P, P]
        lib.hj_ragged_autotune.argtypes = [P, P, P, I32, I32, P]
        lib.hj_ragged_plan_destroy.argtypes = [P]
        for name in ("hj_ragged_plan_create", "hj_ragged_plan_layout", "hj_ragged_plan_bucket",
                     "hj_ragged_solve", "hj_ragged_autotune", "hj_ragged_plan_destroy"):
            getattr(lib, name).restype = ctypes.c_int
        lib.hj_solve_grad.argtypes = [P, I64, P, I32, I32, P, P, P, P, P, P, P, P]
        lib.hj_solve_grad.restype = ctypes.c_int
        lib.hj_solve_grad_unrolled.argtypes = [P, I64, P, P, I32, ctypes.POINTER(SolverOpts), P,
                                               I32, I32, P, P, P, P, P, P]
        lib.hj_solve_grad_unrolled.restype = ctypes.c_int
        lib.hj_solve_batch_retry.argtypes = [P, I64, P, P, I32, ctypes.POINTER(SolverOpts),
                                             ctypes.POINTER(RetryPolicy), P, P, P, P, P, P, P]
        lib.hj_solve_batch_retry.restype = ctypes.c_int
        lib.hj_probe_fp32_fma.argtypes = [I64, I32, ctypes.POINTER(ctypes.c_double), P]
        lib.hj_probe_fp32_fma.restype = ctypes.c_int
        lib.hj_status_str.restype = ctypes.c_char_p
        lib.hj_status_str.argtypes = [ctypes.c_int]
        lib.hj_version.restype = ctypes.c_int32
        for name in ("hj_problem_create", "hj_problem_destroy", "hj_solve_batch"):
            getattr(lib, name).restype = ctypes.c_int
        _LIB = lib
    return _LIB


def _dptr(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Problem:
    """A Hamiltonian family plus terminal cost g = 1/2 sum W^2 (x - c)^2, on the
    current CUDA device (hj_problem_create)."""

    def __init__(self, family, d, dyn, W, c):
        self.family = FAMILIES[family] if isinstance(family, str) else int(family)
        self.d = int(d)
        dyn_a, dyn_p = _dptr(dyn if dyn is not None else [])
        w_a, w_p = _dptr(W)
        c_a, c_p = _dptr(c)
        h = ctypes.c_void_p()
        r = _lib().hj_problem_create(ctypes.byref(h), self.family, self.d,
                                     dyn_p if dyn_a.size else None, dyn_a.size, w_p, c_p)
        self.n_dyn = int(dyn_a.size)
        if r != HJ_OK:
            raise HJError(r, "hj_problem_create")
        self.handle = h

    @classmethod
    def from_workload(cls, w):
        return cls(w["family"], w["d"], w["dyn"], w["W"], w["c"])

    def close(self):
        if getattr(self, "handle", None):
            _lib().hj_problem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_launch_shape(problem, precision, N, warps_per_point, nodes_per_lane):
    """hj_set_launch_shape: G warps per point, NPL nodes per lane for (precision, N)."""
    r = _lib().hj_set_launch_shape(problem.handle, PREC[precision], int(N), int(warps_per_point),
                                   int(nodes_per_lane))
    if r != HJ_OK:
        raise HJError(r, "hj_set_launch_shape")


def get_launch_shape(problem, precision, N):
    g, n = ctypes.c_int32(), ctypes.c_int32()
    r = _lib().hj_get_launch_shape(problem.handle, PREC[precision], int(N), ctypes.byref(g),
                                   ctypes.byref(n))
    if r != HJ_OK:
        raise HJError(r, "hj_get_launch_shape")
    return g.value, n.value


def save_shapes(problem, path):
    """hj_shapes_save: write the launch shapes stored on `problem` to a text cache."""
    r = _lib().hj_shapes_save(problem.handle, os.fsencode(path))
    if r != HJ_OK:
        raise HJError(r, "hj_shapes_save")


def load_shapes(problem, path):
    """hj_shapes_load: apply the cached shapes for this GPU and problem; returns how many."""
    n = ctypes.c_int32(0)
    r = _lib().hj_shapes_load(problem.handle, os.fsencode(path), ctypes.byref(n))
    if r != HJ_OK:
        raise HJError(r, "hj_shapes_load")
    return n.value


def probe_fp32_fma(iters=50000, packed=False, stream=None):
    """hj_probe_fp32_fma: measured FP32 FMA throughput of the current device, TFLOP/s."""
    out = ctypes.c_double(0.0)
    s = stream if stream is not None else torch.cuda.current_stream()
    r = _lib().hj_probe_fp32_fma(int(iters), int(bool(packed)), ctypes.byref(out),
                                 ctypes.c_void_p(s.cuda_stream))
    if r != HJ_OK:
        raise HJError(r, "hj_probe_fp32_fma")
    return out.value


def autotune(problem, xq, t, N, opts, repeats=2, stream=None):
    """hj_autotune on a device sample; returns (warps_per_point, nodes_per_lane, ms)."""
    g, n, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    s = stream if stream is not None else torch.cuda.current_stream(xq.device)
    r = _lib().hj_autotune(problem.handle, xq.shape[0], _ptr(xq.contiguous()), _ptr(t.contiguous()),
                           int(N), ctypes.byref(opts), int(repeats), ctypes.byref(g),
                           ctypes.byref(n), ctypes.byref(ms), ctypes.c_void_p(s.cuda_stream))
    if r != HJ_OK:
        raise HJError(r, "hj_autotune")
    return g.value, n.value, ms.value


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def n_dyn(problem):
    """Length of the problem's dyn array (the layout hj_solve_grad's ddyn follows)."""
    return problem.n_dyn


def solve_grad(problem, t, N, precision, traj_x, traj_p, dL_dV, want_dxq=True, stream=None):
    """hj_solve_grad: gradient of sum_b dL_dV[b] V_b at solved trajectories.
    Returns dict(dW [d], dc [d], ddyn [n_dyn], dxq [B, d] or None), FP64 device tensors."""
    dev = t.device
    d = problem.d
    B = t.shape[0]
    out = dict(dW=torch.empty(d, dtype=torch.float64, device=dev),
               dc=torch.empty(d, dtype=torch.float64, device=dev),
               ddyn=torch.empty(max(n_dyn(problem), 1), dtype=torch.float64, device=dev),
               dxq=torch.empty(B, d, dtype=torch.float64, device=dev) if want_dxq else None)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    r = _lib().hj_solve_grad(problem.handle, B, _ptr(t.contiguous()), int(N), PREC[precision],
                             _ptr(traj_x.contiguous()), _ptr(traj_p.contiguous()),
                             _ptr(dL_dV.contiguous()), _ptr(out["dW"]), _ptr(out["dc"]),
                             _ptr(out["ddyn"]), _ptr(out["dxq"]), ctypes.c_void_p(s.cuda_stream))
    if r != HJ_OK:
        raise HJError(r, "hj_solve_grad")
    out["ddyn"] = out["ddyn"][:n_dyn(problem)]
    return out


def solve_grad_unrolled(problem, xq, t, N, opts, iters, dL_dV, checkpoint_every=32,
                        max_iters=None, stream=None):
    """hj_solve_grad_unrolled: reverse sweep through the iterations each point ran
    (iters from the forward solve), checkpoints every `checkpoint_every` iterations.
    Returns dict(dW, dc, ddyn, dxq) of FP64 device tensors."""
    dev = xq.device
    d = problem.d
    B = xq.shape[0]
    if max_iters is None:
        max_iters = int(iters.max().item()) if B else 0
    out = dict(dW=torch.empty(d, dtype=torch.float64, device=dev),
               dc=torch.empty(d, dtype=torch.float64, device=dev),
               ddyn=torch.empty(max(n_dyn(problem), 1), dtype=torch.float64, device=dev),
               dxq=torch.empty(B, d, dtype=torch.float64, device=dev))
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    r = _lib().hj_solve_grad_unrolled(problem.handle, B, _ptr(xq.contiguous()), _ptr(t.contiguous()),
                                      int(N), ctypes.byref(opts), _ptr(iters.contiguous()),
                                      int(max_iters), int(checkpoint_every), _ptr(dL_dV.contiguous()),
                                      _ptr(out["dW"]), _ptr(out["dc"]), _ptr(out["ddyn"]),
                                      _ptr(out["dxq"]), ctypes.c_void_p(s.cuda_stream))
    if r != HJ_OK:
        raise HJError(r, "hj_solve_grad_unrolled")
    out["ddyn"] = out["ddyn"][:n_dyn(problem)]
    return out


FORM = {"lax": 0, "hopf": 1}
SCHEME = {"be": 0, "fe": 1, "trap": 2}


def make_opts(*, sigma, tau, theta=1.0, tol=1e-8, max_iter=20000, check_every=16,
              inner_steps=1, precision="fp32", seed=0, init_radius=0.1, point_offset=0,
              formulation="lax", scheme="be", value_tol=0.0, time_budget_ms=0.0, iter_budget=0):
    return SolverOpts(float(sigma), float(tau), float(theta), float(tol), int(max_iter),
                      int(check_every), int(inner_steps), PREC[precision], int(seed),
                      float(init_radius), int(point_offset), FORM[formulation], SCHEME[scheme],
                      float(value_tol), float(time_budget_ms), int(iter_budget))


def solve_batch(problem, xq, t, N, opts, *, return_traj=False, warm_x=None, warm_p=None,
                out=None, stream=None, kkt=False):
    """hj_solve_batch on device tensors.  xq [B, d] float64 cuda, t [B] float64 cuda.
    Returns dict(V, iters, status[, traj_x, traj_p][, kkt]) of device tensors; kkt
    (FP64, [B]) is the residual of the discrete characteristic equations at the
    returned iterates.  With `out` given, its "kkt" entry (if any) is filled."""
    if not (xq.is_cuda and t.is_cuda):
        raise ValueError("xq and t must be CUDA tensors")
    xq = xq.contiguous()
    t = t.contiguous()
    if xq.dtype != torch.float64 or t.dtype != torch.float64:
        raise ValueError("xq and t must be float64")
    B, d = xq.shape
    dev = xq.device
    it_dtype = torch.float32 if opts.precision == 0 else torch.float64
    if out is None:
        out = dict(V=torch.empty(B, dtype=torch.float64, device=dev),
                   iters=torch.empty(B, dtype=torch.int32, device=dev),
                   status=torch.empty(B, dtype=torch.int8, device=dev))
        if return_traj:
            out["traj_x"] = torch.empty(B, N + 1, d, dtype=it_dtype, device=dev)
            out["traj_p"] = torch.empty(B, N + 1, d, dtype=it_dtype, device=dev)
        if kkt:
            out["kkt"] = torch.empty(B, dtype=torch.float64, device=dev)
    for key in ("warm_x", "warm_p"):
        w = warm_x if key == "warm_x" else warm_p
        if w is not None and (w.dtype != it_dtype or tuple(w.shape) != (B, N + 1, d)
                              or not w.is_contiguous()):
            raise ValueError(f"{key} must be a contiguous [B, N+1, d] {it_dtype} tensor")
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    r = _lib().hj_solve_batch(problem.handle, B, _ptr(xq), _ptr(t), int(N), ctypes.byref(opts),
                              _ptr(out["V"]), _ptr(out["iters"]), _ptr(out["status"]),
                              _ptr(out.get("kkt")), _ptr(out.get("traj_x")),
                              _ptr(out.get("traj_p")), _ptr(warm_x), _ptr(warm_p),
                              ctypes.c_void_p(s.cuda_stream))
    if r != HJ_OK:
        raise HJError(r, "hj_solve_batch")
    return out


def kkt_residual(problem, t, N, precision, traj_x, traj_p, stream=None):
    """hj_kkt_residual: residual of the discrete characteristic equations at the
    given trajectories ([B, N+1, d] in the precision's type; FP64 evaluation, FP32
    for the quadcopter's FP32 trajectories), [B] float64 device tensor."""
    B = t.shape[0]
    out = torch.empty(B, dtype=torch.float64, device=t.device)
    s = stream if stream is not None else torch.cuda.current_stream(t.device)
    r = _lib().hj_kkt_residual(problem.handle, B, _ptr(t.contiguous()), int(N), PREC[precision],
                               _ptr(traj_x.contiguous()), _ptr(traj_p.contiguous()), _ptr(out),
                               ctypes.c_void_p(s.cuda_stream))
    if r != HJ_OK:
        raise HJError(r, "hj_kkt_residual")
    return out


class RetryPolicy(ctypes.Structure):
    """hj_retry_policy: extra rounds for points that reach the iteration cap."""
    _fields_ = [("rounds", ctypes.c_int32), ("sigma_step", ctypes.c_double),
                ("step_product", ctypes.c_double), ("warm", ctypes.c_int32),
                ("value_tol", ctypes.c_double)]


def solve_batch_retry(problem, xq, t, N, opts, policy, *, return_traj=False, stream=None):
    """hj_solve_batch_retry on device tensors (as solve_batch); the result also
    holds `rounds` [B] int8, the last round each point ran in."""
    if not (xq.is_cuda and t.is_cuda) or xq.dtype != torch.float64 or t.dtype != torch.float64:
        raise ValueError("xq and t must be float64 CUDA tensors")
    xq = xq.contiguous()
    t = t.contiguous()
    B, d = xq.shape
    dev = xq.device
    it_dtype = torch.float32 if opts.precision == 0 else torch.float64
    out = dict(V=torch.empty(B, dtype=torch.float64, device=dev),
               iters=torch.empty(B, dtype=torch.int32, device=dev),
               status=torch.empty(B, dtype=torch.int8, device=dev),
               rounds=torch.empty(B, dtype=torch.int8, device=dev))
    if return_traj:
        out["traj_x"] = torch.empty(B, N + 1, d, dtype=it_dtype, device=dev)
        out["traj_p"] = torch.empty(B, N + 1, d, dtype=it_dtype, device=dev)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    r = _lib().hj_solve_batch_retry(problem.handle, B, _ptr(xq), _ptr(t), int(N),
                                    ctypes.byref(opts), ctypes.byref(policy), _ptr(out["V"]),
                                    _ptr(out["iters"]), _ptr(out["status"]), _ptr(out["rounds"]),
                                    _ptr(out.get("traj_x")), _ptr(out.get("traj_p")),
                                    ctypes.c_void_p(s.cuda_stream))
    if r != HJ_OK:
        raise HJError(r, "hj_solve_batch_retry")
    return out


def solve_workload(w, *, precision="fp32", return_traj=False, problem=None, device="cuda",
                   **overrides):
    """Convenience: run a workload dict (workloads.py) end to end on the GPU."""
    prob = problem if problem is not None else Problem.from_workload(w)
    kkt = bool(overrides.pop("kkt", False))
    o = dict(sigma=w["sigma"], tau=w["tau"], tol=w["tol"], max_iter=w["max_iter"],
             check_every=w["check_every"], seed=w["seed"], init_radius=w["init_radius"])
    o.update(overrides)
    opts = make_opts(precision=precision, **o)
    xq = torch.as_tensor(np.asarray(w["xq"], dtype=np.float64), device=device)
    t = torch.as_tensor(np.asarray(w["t"], dtype=np.float64), device=device)
    return solve_batch(prob, xq, t, int(w["N"]), opts, return_traj=return_traj, kkt=kkt)


class RaggedPlan:
    """hj_ragged_plan_*: a batch mixing problems and per-point N, solved by one
    CUDA-graph launch.  `problems` are Problem objects (kept alive here)."""

    def __init__(self, problems, prob_of, N_of, opts):
        self.problems = list(problems)
        self.prob_of = np.ascontiguousarray(prob_of, dtype=np.int32)
        self.N_of = np.ascontiguousarray(N_of, dtype=np.int32)
        self.B = len(self.prob_of)
        self.opts = opts
        hs = (ctypes.c_void_p * len(self.problems))(*[p.handle.value for p in self.problems])
        h = ctypes.c_void_p()
        I32P = ctypes.POINTER(ctypes.c_int32)
        r = _lib().hj_ragged_plan_create(ctypes.byref(h), len(self.problems), hs, self.B,
                                         self.prob_of.ctypes.data_as(I32P),
                                         self.N_of.ctypes.data_as(I32P), ctypes.byref(opts))
        if r != HJ_OK:
            raise HJError(r, "hj_ragged_plan_create")
        self.handle = h
        self.xq_off = np.zeros(self.B + 1, dtype=np.int64)
        self.traj_off = np.zeros(self.B + 1, dtype=np.int64)
        nb = ctypes.c_int32()
        I64P = ctypes.POINTER(ctypes.c_int64)
        _lib().hj_ragged_plan_layout(h, self.xq_off.ctypes.data_as(I64P),
                                     self.traj_off.ctypes.data_as(I64P), ctypes.byref(nb))
        self.n_buckets = nb.value

    def buckets(self):
        out = []
        for i in range(self.n_buckets):
            v = [ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32(),
                 ctypes.c_int32(), ctypes.c_int32()]
            _lib().hj_ragged_plan_bucket(self.handle, i, *[ctypes.byref(x) for x in v])
            out.append(dict(problem=v[0].value, n_max=v[1].value, n_points=v[2].value,
                            warps_per_point=v[3].value, nodes_per_lane=v[4].value,
                            inner_steps=v[5].value))
        return out

    def pack_xq(self, xq_list):
        """Host list of per-point query arrays -> packed float64 numpy array."""
        out = np.empty(self.xq_off[-1])
        for b, x in enumerate(xq_list):
            out[self.xq_off[b]:self.xq_off[b + 1]] = x
        return out

    def autotune(self, xq, t, repeats=1, max_inner_steps=1, stream=None):
        s = stream if stream is not None else torch.cuda.current_stream(xq.device)
        r = _lib().hj_ragged_autotune(self.handle, _ptr(xq), _ptr(t), int(repeats),
                                      int(max_inner_steps), ctypes.c_void_p(s.cuda_stream))
        if r != HJ_OK:
            raise HJError(r, "hj_ragged_autotune")

    def solve(self, xq, t, *, return_traj=False, out=None, stream=None):
        """xq packed float64 cuda tensor, t [B] float64 cuda tensor."""
        dev = xq.device
        it_dtype = torch.float32 if self.opts.precision == 0 else torch.float64
        if out is None:
            out = dict(V=torch.empty(self.B, dtype=torch.float64, device=dev),
                       iters=torch.empty(self.B, dtype=torch.int32, device=dev),
                       status=torch.empty(self.B, dtype=torch.int8, device=dev))
            if return_traj:
                n = int(self.traj_off[-1])
                out["traj_x"] = torch.empty(n, dtype=it_dtype, device=dev)
                out["traj_p"] = torch.empty(n, dtype=it_dtype, device=dev)
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        r = _lib().hj_ragged_solve(self.handle, _ptr(xq), _ptr(t), _ptr(out["V"]),
                                   _ptr(out["iters"]), _ptr(out["status"]),
                                   _ptr(out.get("traj_x")), _ptr(out.get("traj_p")),
                                   ctypes.c_void_p(s.cuda_stream))
        if r != HJ_OK:
            raise HJError(r, "hj_ragged_solve")
        return out

    def point_traj(self, flat, b):
        """Trajectory block [N_b+1][d_b] of point b in a packed array."""
        d = int((self.xq_off[b + 1] - self.xq_off[b]))
        return flat[self.traj_off[b]:self.traj_off[b + 1]].reshape(-1, d)

    def close(self):
        if getattr(self, "handle", None):
            _lib().hj_ragged_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
