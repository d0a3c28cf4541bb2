"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and the FP64 oracle on the same seeded inputs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lax_pdhg as O  # noqa: E402
from paper_1803_01215_gb300 import binding  # noqa: E402

CONVERGED_TOL = 1e-24


def gpu(w, precision, **kw):
    out = binding.solve_workload(w, precision=precision, return_traj=True, **kw)
    return {k: v.cpu().numpy() for k, v in out.items()}


def oracle_same_stop(w, **kw):
    return O.solve(w, **kw)


def oracle_converged(w, **kw):
    kw.setdefault("tol", CONVERGED_TOL)
    kw.setdefault("check_every", 1)
    kw.setdefault("max_iter", 200000)
    return O.solve(w, **kw)


def value_err(Vg, Vo):
    return np.abs(Vg - Vo) / np.maximum(1.0, np.abs(Vo))
