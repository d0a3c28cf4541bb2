"""Retry rounds for the points that reach the iteration cap: the paper's
handling of slow points in Section 6.2 (raise sigma by a fixed step and set tau
from the step-size bound) and Section 6.1 (rerun the point with the same steps),
on top of the FP64 solvers.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Round 0 is the plain solve.  Round r = 1..R takes the points whose status is
MAX_ITER after round r - 1 and solves them again with
  sigma_r = sigma + r * sigma_step,
  tau_r   = step_product / sigma_r   (step_product = 0: sigma * tau of the options),
either from a fresh random guess drawn with seed + r (warm = False: the point is
rerun) or from its last iterate (warm = True: the iteration continues with the
new steps, z restarting at x).  A point's iterations add up over its rounds and
`rounds` records the last round it ran in.  value_tol > 0: the last round also
stops a point whose value moved by less than value_tol between two tests (the
paper's switch to a value criterion after a maximum count).
"""
import numpy as np

from . import game_pdhg, lax_pdhg

MAX_ITER = lax_pdhg.MAX_ITER


def _solver(w):
    return game_pdhg.solve_game if w["family"] == "game_norms" else lax_pdhg.solve


def solve_retry(w, *, rounds, sigma_step, step_product=0.0, warm=False, value_tol=0.0, **kw):
    solve = _solver(w)
    out = solve(w, **kw)
    out = {k: np.array(v) for k, v in out.items()}
    out["rounds"] = np.zeros(len(out["V"]), dtype=np.int64)
    sigma0 = float(kw.get("sigma", w["sigma"]))
    tau0 = float(kw.get("tau", w["tau"]))
    seed0 = int(kw.get("seed", w["seed"]))
    prod = step_product if step_product > 0 else sigma0 * tau0
    pidx = np.asarray(w.get("point_index", np.arange(len(out["V"]))))
    for r in range(1, rounds + 1):
        ids = np.where(out["status"] == MAX_ITER)[0]
        if ids.size == 0:
            break
        sub = dict(w)
        sub["xq"] = np.asarray(w["xq"])[ids]
        sub["t"] = np.asarray(w["t"])[ids]
        sub["point_index"] = pidx[ids]
        sig = sigma0 + r * sigma_step
        args = dict(kw, sigma=sig, tau=prod / sig)
        if r == rounds and value_tol > 0:
            args.update(value_tol=value_tol)      # the last round may also stop on the value
        if warm:
            args.update(x_init=out["x"][ids], p_init=out["p"][ids])
        else:
            args.update(seed=seed0 + r)
        o = solve(sub, **args)
        for k in ("V", "status", "x", "p", "rx", "rp"):
            out[k][ids] = o[k]
        out["iters"][ids] += o["iters"]
        out["rounds"][ids] = r
    return out
