"""The NEXT rows at the sizes and launch configurations bench.py times, on
sampled points: the trapezoid scheme on the 4096-point 12-D batch, the
difference-of-norms game on the paper's 5329-point grid, and the moving-bump
eikonal on its 3721-point grid.  Every sampled point's FP32 value is compared
with the converged FP64 oracle (1e-4 * max(1, |V|)); where the paper's stop
(tol 1e-8) leaves slow points short of the saddle in both precisions, at a
tighter stop where the FP64 path itself meets 1e-5."""
import numpy as np
import pytest

from gpu_common import gpu, value_err
from oracle import game_pdhg as GO
from oracle import lax_pdhg as O
from oracle import lax_schemes as S
from paper_1803_01215_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _sample(g, n, seed):
    conv = np.where(g["status"] == O.CONVERGED)[0]
    return np.sort(np.random.default_rng(seed).choice(conv, size=n, replace=False))


def test_trapezoid_full_size_sampled():
    w = W.quadcopter()
    g = gpu(w, "fp32", scheme="trap")
    assert np.all(g["status"] == O.CONVERGED)
    idx = _sample(g, 6, 101)
    o = S.solve_scheme(W.subset(w, idx), "trap", tol=1e-24, max_iter=200000, check_every=8)
    assert np.all(o["status"] == O.CONVERGED)
    assert value_err(g["V"][idx], o["V"]).max() <= 1e-4


def _by_sigma(run, sigmas, n):
    """Run `run(sigma)` for each sigma in turn and keep, per point, the first run
    that converged (the fixed point does not depend on sigma; the paper takes a
    larger sigma for the points that reach the cap), else the last run's.
    Returns V and status."""
    V = np.full(n, np.nan)
    st = np.full(n, O.MAX_ITER)
    for sig in sigmas:
        todo = st != O.CONVERGED
        if not np.any(todo):
            break
        r = run(sig, np.where(todo)[0])
        V[todo] = r["V"]               # the last run's value where none converged
        st[todo] = r["status"]
    return V, st


def _tight_bars(w, solve_oracle, idx, sigmas):
    """Every sampled point against the converged oracle, at a stop where the FP64
    path is within 1e-5 of it: FP64 tol 1e-14, FP32 tol 1e-11 (its rounding floor
    is near 1e-10 at these step sizes), the whole grid rerun on the GPU so that
    each point keeps its own initial guess."""
    sub = W.subset(w, idx)
    Vo, so = _by_sigma(lambda sig, ids: solve_oracle(W.subset(sub, ids), sigma=sig, tau=0.24 / sig,
                                                      tol=1e-20, max_iter=400000, check_every=8),
                       sigmas, len(idx))
    assert np.all(so == O.CONVERGED)
    out = {}
    for prec, tol in (("fp64", 1e-14), ("fp32", 1e-11)):
        V, st = _by_sigma(lambda sig, ids: {k: v[idx][ids] for k, v in gpu(
            w, prec, sigma=sig, tau=0.24 / sig, tol=tol, max_iter=400000, check_every=16).items()},
            sigmas, len(idx))
        out[prec] = (value_err(V, Vo), st)
    return out


def test_game_full_grid_sampled():
    """The game's points converge slowly (sigma = 50): at the paper's stop some
    values are still 1e-3 from the saddle, in either precision.  So the value
    bars are taken at a tighter stop, where the FP64 path itself is within 1e-5
    of the converged oracle on every sampled point: there every sampled point's
    FP32 value must be within 1e-4 of it.  Points that reach the cap at sigma = 50
    are rerun with sigma raised by 20 (Section 6.2), on both sides.  At the paper's
    stop the FP64 path stops where the oracle does, with the same value (1e-9)."""
    w = W.game_norms(d=2, t=0.2)
    g = gpu(w, "fp32")
    g64 = gpu(w, "fp64")
    assert np.mean(g["status"] == O.CONVERGED) >= 0.9
    idx = np.sort(np.random.default_rng(102).choice(len(w["xq"]), 10, replace=False))
    o = GO.solve_game(W.subset(w, idx))
    same = o["status"] == O.CONVERGED
    assert np.all(g64["iters"][idx][same] == o["iters"][same])
    assert value_err(g64["V"][idx][same], o["V"][same]).max() <= 1e-9
    bars = _tight_bars(w, GO.solve_game, idx, (50.0, 70.0, 90.0))
    print("game tight stop: FP64 max {:.2e}, FP32 max {:.2e}".format(
        bars["fp64"][0].max(), bars["fp32"][0].max()))
    assert bars["fp64"][0].max() <= 1e-5
    assert bars["fp32"][0].max() <= 1e-4


def test_moving_bump_full_grid_sampled():
    """Every sampled point (converged or not at the paper's stop) against the
    converged oracle, at a stop where the FP64 path is within 1e-5 of it; points
    that reach the cap at sigma = 0.5 are rerun at sigma = 50, the paper's choice
    near the bump (Section 6.1), on both sides."""
    w = W.eikonal_moving(t=0.3)
    g = gpu(w, "fp32")
    assert np.mean(g["status"] == O.CONVERGED) >= 0.9
    idx = np.sort(np.random.default_rng(103).choice(len(w["xq"]), 10, replace=False))
    bars = _tight_bars(w, O.solve, idx, (0.5, 50.0))
    print("moving bump tight stop: FP64 max {:.2e}, FP32 max {:.2e}".format(
        bars["fp64"][0].max(), bars["fp32"][0].max()))
    assert bars["fp64"][0].max() <= 1e-5
    assert bars["fp32"][0].max() <= 1e-4
