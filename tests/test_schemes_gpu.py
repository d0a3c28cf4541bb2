"""The forward-Euler (Eq. disclaxFE) and trapezoid schemes on the CUDA path,
through the C ABI, against the FP64 oracle of those forms (oracle/lax_schemes.py,
pinned by tests/test_oracle_schemes_pins.py).  The CUDA path stores the costate
of interval [s_{j-1}, s_j] at node j: traj_p[:, j] is the oracle's p[:, j - 1].

Bars, as for the backward-Euler form: element-wise after a fixed number of
iterations (FP64 1e-10; FP32 1e-4, and for p of the negative eikonal equation,
whose sigma = 100 multiplies FP32 rounding of x 100-fold in every dual step,
1e-4 sigma / 25), FP64 with the workload's stopping rule (value 1e-9, same
iteration counts for most points), the FP32 value within 1e-4 * max(1, |V|) of
the converged oracle, and the convergence order in delta of the GPU values.
"""
import numpy as np
import pytest

from gpu_common import CONVERGED_TOL, gpu, value_err
from oracle import lax_pdhg as O
from oracle import game_schemes as GS
from oracle import lax_schemes as S
from paper_1803_01215_gb300 import workloads as W
from test_parity_gpu import _custom

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _eik(d, sign, N, B, seed=71):
    w = W.eikonal(d=d, sign=sign, B=B, seed=seed)
    w["N"] = N
    w["t"] = np.full(B, N * W.EIK_DELTA)
    return w


# the default launch shapes (one node per lane, G = 1, 2, 4 for N = 23, 64, 100,
# 128) with ragged tails, the four families; every other shape is checked by
# test_scheme_every_launch_shape_gives_the_same_iterates.  tanh drift at d >= 8
# (and d = 4 with N = 200, beyond the mixed FP64 register kernel) runs the
# shared-memory kernel, the eikonal family at d not in {2, 10} the
# coordinate-parallel one, d not a multiple of 4 included
CASES = [
    ("quadcopter", 12, 23), ("quadcopter", 12, 64), ("quadcopter", 12, 100),
    ("tanh_drift", 4, 50), ("tanh_drift", 2, 128),
    ("eikonal+", 2, 5), ("eikonal+", 10, 30), ("eikonal-", 2, 10),
    ("game", 2, 5), ("game", 2, 23), ("game", 7, 10),
    ("tanh_drift", 8, 16), ("tanh_drift", 13, 21), ("tanh_drift", 32, 32),
    ("tanh_drift", 4, 200), ("eikonal+", 5, 10), ("eikonal-", 37, 10), ("eikonal+", 3, 40),
]


def _case(family, d, N, B, seed=21):
    if family == "game":
        w = W.game_norms(d=d, B=B, seed=seed)
        w["N"] = N
        w["t"] = np.full(B, N * W.EIK_DELTA)
        return w
    if family.startswith("eikonal"):
        return _eik(d, 1 if family.endswith("+") else -1, N, B, seed=seed)
    return _custom(family, d, N, B, seed=seed)


def _cmp(g, o):
    ex = np.max(np.abs(g["traj_x"] - o["x"]))
    ep = np.max(np.abs(g["traj_p"][:, 1:] - o["p"]))
    assert np.all(g["traj_p"][:, 0] == 0.0)
    return ex, ep, np.max(value_err(g["V"], o["V"]))


@pytest.mark.parametrize("family,d,N", CASES)
@pytest.mark.parametrize("scheme", ["fe", "trap"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_scheme_fixed_iterations_elementwise(family, d, N, scheme, precision):
    w = _case(family, d, N, B=37)
    K = 150
    g = gpu(w, precision, tol=0.0, max_iter=K, check_every=K, scheme=scheme)
    solve = GS.solve_game_scheme if family == "game" else S.solve_scheme
    o = solve(w, scheme, tol=0.0, max_iter=K, check_every=K)
    assert np.all(g["iters"] == K) and np.all(g["status"] == O.MAX_ITER)
    ex, ep, ev = _cmp(g, o)
    print(f"{scheme} {family} d={d} N={N} {precision}: |dx| {ex:.2e} |dp| {ep:.2e} V {ev:.2e}")
    tol = 1e-10 if precision == "fp64" else 1e-4
    tol_p = tol * max(1.0, w["sigma"] / 25.0) if precision == "fp32" else tol
    assert ex <= tol and ep <= tol_p
    assert ev <= (1e-9 if precision == "fp64" else 1e-4)


@pytest.mark.parametrize("family,d,N,B", [
    ("quadcopter", 12, 32, 24), ("tanh_drift", 4, 40, 40), ("eikonal+", 2, 10, 24),
    ("tanh_drift", 32, 32, 12), ("eikonal+", 5, 10, 24)])
@pytest.mark.parametrize("scheme", ["fe", "trap"])
def test_scheme_fp64_same_stop_and_fp32_value(family, d, N, B, scheme):
    w = _case(family, d, N, B, seed=22)
    o = S.solve_scheme(w, scheme)
    g = gpu(w, "fp64", scheme=scheme)
    conv = o["status"] == O.CONVERGED
    assert np.mean(conv) >= 0.9 and np.all(g["status"][conv] == O.CONVERGED)
    same = (g["iters"] == o["iters"]) & conv
    assert np.mean(same) >= 0.8
    assert value_err(g["V"][same], o["V"][same]).max() <= 1e-9
    assert np.max(np.abs(g["traj_x"][same] - o["x"][same])) <= 1e-9
    oc = S.solve_scheme(w, scheme, tol=CONVERGED_TOL, max_iter=200000, check_every=8)
    g32 = gpu(w, "fp32", scheme=scheme)
    ok = (oc["status"] == O.CONVERGED) & (g32["status"] == O.CONVERGED)
    assert np.mean(ok) >= 0.9
    assert value_err(g32["V"][ok], oc["V"][ok]).max() <= 1e-4


@pytest.mark.parametrize("d", [2, 7])
@pytest.mark.parametrize("scheme", ["fe", "trap"])
def test_game_scheme_fp64_same_stop(d, scheme):
    w = _case("game", d, 5, 24, seed=62)
    o = GS.solve_game_scheme(w, scheme)
    g = gpu(w, "fp64", scheme=scheme)
    conv = o["status"] == O.CONVERGED
    assert np.mean(conv) >= 0.8
    same = (g["iters"] == o["iters"]) & conv
    assert np.mean(same) >= 0.7
    assert value_err(g["V"][same], o["V"][same]).max() <= 1e-9


@pytest.mark.parametrize("family,d,N", [("quadcopter", 12, 64), ("eikonal+", 2, 64),
                                        ("game", 2, 40), ("tanh_drift", 4, 64)])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_scheme_every_launch_shape_gives_the_same_iterates(family, d, N, precision):
    """Every (warps per point, nodes per lane) instantiation of the mixed kernel
    computes the same node formulas: the first shape against the oracle, the
    others against the first to the rounding level."""
    from paper_1803_01215_gb300 import binding
    w = _case(family, d, N, B=21)
    prob = binding.Problem.from_workload(w)
    xq = torch.as_tensor(w["xq"], device="cuda")
    t = torch.as_tensor(w["t"], device="cuda")
    opts = binding.make_opts(sigma=w["sigma"], tau=w["tau"], tol=0.0, max_iter=60, check_every=60,
                             precision=precision, seed=w["seed"], scheme="trap")
    outs = []
    for G in (1, 2, 4, 8):
        for npl in ((1, 2) if precision == "fp32" else (1,)):
            if N > 32 * G * npl or (precision == "fp64" and G == 8):
                continue
            binding.set_launch_shape(prob, precision, N, G, npl)
            o = binding.solve_batch(prob, xq, t, N, opts, return_traj=True)
            outs.append(((G, npl), {k: v.cpu().numpy() for k, v in o.items()}))
    assert len(outs) >= 2
    ref = outs[0][1]
    solve = GS.solve_game_scheme if family == "game" else S.solve_scheme
    o = solve(w, "trap", tol=0.0, max_iter=60, check_every=60)
    ex, ep, _ = _cmp(ref, o)
    tol = 1e-10 if precision == "fp64" else 1e-4
    assert ex <= tol and ep <= (tol * max(1.0, w["sigma"] / 25.0) if precision == "fp32" else tol)
    rt = 1e-13 if precision == "fp64" else 1e-5
    rp = rt * (max(1.0, w["sigma"] / 25.0) if precision == "fp32" else 1.0)
    for shape, out in outs[1:]:
        np.testing.assert_allclose(out["traj_x"], ref["traj_x"], rtol=rt, atol=rt, err_msg=str(shape))
        np.testing.assert_allclose(out["traj_p"], ref["traj_p"], rtol=rp, atol=rp, err_msg=str(shape))
        assert np.max(value_err(out["V"], ref["V"])) <= (1e-12 if precision == "fp64" else 1e-6)


def test_quadratic_family_is_scheme_independent():
    """H = |p|^2/2 does not see x: every scheme is the same problem, and the
    library runs it as backward Euler (identical outputs)."""
    w = _custom("quadratic", 3, 37, B=20)
    ref = gpu(w, "fp32")
    for scheme in ("fe", "trap"):
        g = gpu(w, "fp32", scheme=scheme)
        for k in ("V", "iters", "traj_x", "traj_p"):
            assert np.array_equal(g[k], ref[k]), (scheme, k)


def test_gpu_values_show_the_orders_in_delta():
    """Quadcopter, FP64 converged: successive differences of V over N = 16, 32,
    64, 128 shrink by 2 per halving of delta for both Euler forms and by 4 for
    the trapezoid form (a property of the discretisations that holds at any
    size)."""
    base = _custom("quadcopter", 12, 16, B=6, t=0.5, seed=23)
    V = {}
    for scheme in ("be", "fe", "trap"):
        vals = []
        for N in (16, 32, 64, 128):
            w = dict(base, N=N)
            g = gpu(w, "fp64", tol=1e-24, max_iter=400000, check_every=64, scheme=scheme)
            assert np.all(g["status"] == O.CONVERGED), (scheme, N)
            vals.append(g["V"])
        V[scheme] = np.array(vals)
    for scheme, (lo, hi) in (("be", (1.6, 2.4)), ("fe", (1.6, 2.4)), ("trap", (3.4, 4.6))):
        d = np.diff(V[scheme], axis=0)
        ratio = np.abs(d[1] / d[2])
        print(scheme, ratio)
        assert np.all((ratio > lo) & (ratio < hi)), (scheme, ratio)
    # the trapezoid values sit between the two Euler values at the finest N
    lo = np.minimum(V["be"][-1], V["fe"][-1])
    hi = np.maximum(V["be"][-1], V["fe"][-1])
    assert np.all((V["trap"][-1] > lo) & (V["trap"][-1] < hi))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_scheme_ragged_fixed_iterations_elementwise(precision):
    from test_ragged_gpu import _groups, _plan
    rw = W.ragged_mix(B=60, seed=24)
    rw["problems"] = rw["problems"][:2]                    # tanh drift d = 4, quadcopter
    r = np.random.default_rng(24)
    rw["prob_of"] = r.integers(0, 2, size=60).astype(np.int32)
    rw["N_of"] = r.choice(np.array([3, 17, 40, 64, 100], dtype=np.int32), size=60)
    rw["xq"] = [0.5 * r.standard_normal(12) if k == 1 else r.standard_normal(4)
                for k in rw["prob_of"]]
    # delta = 0.03 for every point: with N = 3 and t ~ 1.7 (delta ~ 0.6) the
    # quadcopter iteration is chaotic before it settles (the oracle itself turns a
    # 1e-13 change of the initial guess into O(1) after 40 iterations)
    rw["t"] = 0.03 * rw["N_of"].astype(np.float64)
    K = 40
    plan, xq, t = _plan(rw, precision, tol=0.0, max_iter=K, check_every=K, scheme="trap")
    out = {k: v.cpu().numpy() for k, v in plan.solve(xq, t, return_traj=True).items()}
    assert np.all(out["iters"] == K)
    tol = 1e-10 if precision == "fp64" else 1e-4
    for k, N in _groups(rw):
        g = W.ragged_group(rw, k, N)
        o = S.solve_scheme(g, "trap", tol=0.0, max_iter=K, check_every=K)
        for i, b in enumerate(g["point_index"]):
            assert np.max(np.abs(plan.point_traj(out["traj_x"], b) - o["x"][i])) <= tol, (k, N, b)
            assert np.max(np.abs(plan.point_traj(out["traj_p"], b)[1:] - o["p"][i])) <= tol, (k, N, b)
        assert np.max(value_err(out["V"][g["point_index"]], o["V"])) <= \
            (1e-9 if precision == "fp64" else 1e-4)


def test_scheme_argument_errors():
    from paper_1803_01215_gb300 import binding
    w = _custom("quadcopter", 12, 8, B=3)
    prob = binding.Problem.from_workload(w)
    xq = torch.as_tensor(w["xq"], device="cuda")
    t = torch.as_tensor(w["t"], device="cuda")
    binding.solve_batch(prob, xq, t, 8, binding.make_opts(sigma=1.0, tau=0.24, scheme="fe"))
    unsupported = [
        binding.make_opts(sigma=1.0, tau=0.24, scheme="fe", formulation="hopf"),
        binding.make_opts(sigma=1.0, tau=0.24, scheme="trap", inner_steps=2),
    ]
    for opts in unsupported:
        with pytest.raises(binding.HJError) as e:
            binding.solve_batch(prob, xq, t, 8, opts)
        assert e.value.code == 2                                   # HJ_ERR_UNSUPPORTED
    # FP64 with N > 128 needs the 8-warp group, which the mixed kernels do not have
    with pytest.raises(binding.HJError) as e:
        binding.solve_batch(prob, xq, t, 200, binding.make_opts(sigma=1.0, tau=0.24, scheme="fe",
                                                                precision="fp64"))
    assert e.value.code == 2
    bad = binding.make_opts(sigma=1.0, tau=0.24)
    bad.scheme = 5
    with pytest.raises(binding.HJError) as e:
        binding.solve_batch(prob, xq, t, 8, bad)
    assert e.value.code == 1                                       # HJ_ERR_INVALID_ARG
    # the shared-memory tanh-drift kernel runs the mixed schemes, but not the Hopf form
    wt = _custom("tanh_drift", 8, 8, B=3)
    pt = binding.Problem.from_workload(wt)
    xt = torch.as_tensor(wt["xq"], device="cuda")
    binding.solve_batch(pt, xt, t, 8, binding.make_opts(sigma=1.0, tau=0.24, scheme="trap"))
    with pytest.raises(binding.HJError) as e:
        binding.solve_batch(pt, xt, t, 8, binding.make_opts(sigma=1.0, tau=0.24, scheme="trap",
                                                            formulation="hopf"))
    assert e.value.code == 2
    # the reverse sweep differentiates the backward-Euler iteration only
    fe = binding.make_opts(sigma=1.0, tau=0.24, scheme="fe", precision="fp64")
    out = binding.solve_batch(prob, xq, t, 8, fe)
    with pytest.raises(binding.HJError) as e:
        binding.solve_grad_unrolled(prob, xq, t, 8, fe, out["iters"],
                                    torch.ones(3, dtype=torch.float64, device="cuda"))
    assert e.value.code == 2
