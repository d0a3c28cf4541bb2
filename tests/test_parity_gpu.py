"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars (tolerances written in each test):
  * FP64 GPU vs oracle, same stopping rule: value within 1e-9 * max(1, |V|),
    same iteration counts, iterates within 1e-9.
  * FP32 GPU vs the converged oracle: value within 1e-4 * max(1, |V|) at the
    paper's stopping rule (tol 1e-8 on the squared increments); trajectory max
    error within 1e-3 when the GPU stops at tol 1e-10 (1e-9 for d >= 32, where
    FP32 rounding of (N+1)*d entries puts the squared-increment floor near
    1e-10).  At tol 1e-8 the last iterate is still ~1e-3 from the fixed point
    in both precisions, so the trajectory bar needs the tighter stop.
  * Element-wise after a fixed number of iterations (tol = 0): FP64 within
    1e-10, FP32 within 1e-4.
"""
import numpy as np
import pytest

from gpu_common import gpu, oracle_converged, oracle_same_stop, value_err
from oracle import lax_pdhg as O
from paper_1803_01215_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _custom(family, d, N, B, seed=21, t=None, sigma=1.0):
    r = np.random.default_rng(seed)
    if family == "quadratic":
        dyn = np.zeros(0)
    elif family == "quadcopter":
        dyn = np.array([W.QC_MASS, W.QC_HOVER, W.QC_GRAVITY, W.QC_EPS])
    else:
        dyn = (r.standard_normal((d, d)) / np.sqrt(d)).reshape(-1)
    scale = 0.5 if family == "quadcopter" else 1.0
    return dict(family=family, d=d, dyn=dyn, W=r.uniform(0.5, 2.0, d),
                c=(np.zeros(d) if family == "quadcopter" else 0.3 * r.standard_normal(d)),
                xq=scale * r.standard_normal((B, d)),
                t=(r.uniform(0.5, 2.0, B) if t is None else np.full(B, t)), N=N,
                sigma=sigma, tau=0.24 / sigma, tol=1e-8, max_iter=20000, check_every=16,
                seed=seed, init_radius=0.1)


def TRAJ_TOL(d):
    return 1e-10 if d <= 12 else 1e-9


# shapes that cover every kernel variant: warp kernel NPL 1/2/4 with ragged N,
# the shared-memory kernel with d not a multiple of 4, and B not a multiple of
# the warps per CTA; the FP32 tiled tanh-drift kernel with four-node tiles
# (d = 8, 13, 32, 64 at N = 7, 24 at N = 70, 64 at N = 64, 32 at N = 200: one,
# two, four, eight and sixteen warps per point) and eight-node tiles (d = 100 at
# N = 32, 80 at N = 40: four and eight warps)
SHAPES = [
    ("quadratic", 2, 20), ("quadratic", 3, 37), ("quadratic", 4, 100), ("quadratic", 1, 5),
    ("quadcopter", 12, 64), ("quadcopter", 12, 23),
    ("tanh_drift", 4, 50), ("tanh_drift", 8, 16), ("tanh_drift", 2, 128),
    ("tanh_drift", 32, 32), ("tanh_drift", 13, 21), ("tanh_drift", 100, 32), ("tanh_drift", 64, 7),
    ("tanh_drift", 24, 70), ("tanh_drift", 32, 200), ("tanh_drift", 80, 40),
    ("tanh_drift", 64, 64),
]


@pytest.mark.parametrize("family,d,N", SHAPES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fixed_iterations_elementwise(family, d, N, precision):
    w = _custom(family, d, N, B=37)
    K = 150
    g = gpu(w, precision, tol=0.0, max_iter=K, check_every=K)
    o = oracle_same_stop(w, tol=0.0, max_iter=K, check_every=K)
    assert np.all(g["iters"] == K) and np.all(g["status"] == O.MAX_ITER)
    tol = 1e-10 if precision == "fp64" else 1e-4
    ex = np.max(np.abs(g["traj_x"] - o["x"]))
    ep = np.max(np.abs(g["traj_p"] - o["p"]))
    ev = np.max(value_err(g["V"], o["V"]))
    print(f"{family} d={d} N={N} {precision}: max|dx|={ex:.2e} max|dp|={ep:.2e} V rel={ev:.2e}")
    assert ex <= tol and ep <= tol
    assert ev <= (1e-9 if precision == "fp64" else 1e-4)


@pytest.mark.parametrize("family,d,N,B", [
    ("quadratic", 2, 20, 64), ("quadcopter", 12, 64, 24), ("tanh_drift", 4, 32, 40),
    ("tanh_drift", 32, 32, 12), ("tanh_drift", 100, 32, 5)])
def test_fp64_same_stop(family, d, N, B):
    w = _custom(family, d, N, B)
    g = gpu(w, "fp64")
    o = oracle_same_stop(w)
    assert np.all(g["status"] == O.CONVERGED)
    assert np.mean(g["iters"] == o["iters"]) >= 0.8
    same = g["iters"] == o["iters"]
    ev = value_err(g["V"], o["V"])[same]
    print(f"{family} d={d}: iters {np.median(g['iters'])}, max V rel {ev.max():.2e}")
    assert ev.max() <= 1e-9
    assert np.max(np.abs(g["traj_x"][same] - o["x"][same])) <= 1e-9


@pytest.mark.parametrize("family,d,N,B", [
    ("quadratic", 2, 20, 64), ("quadcopter", 12, 64, 24), ("tanh_drift", 4, 32, 40),
    ("tanh_drift", 32, 32, 12), ("tanh_drift", 100, 32, 5)])
def test_fp32_against_converged_oracle(family, d, N, B):
    w = _custom(family, d, N, B)
    g = gpu(w, "fp32")
    o = oracle_converged(w)
    assert np.all(o["status"] == O.CONVERGED)
    assert np.all(g["status"] == O.CONVERGED)
    ev = value_err(g["V"], o["V"])
    et = np.max(np.abs(g["traj_x"] - o["x"]))
    gt = gpu(w, "fp32", tol=TRAJ_TOL(d))
    evt = value_err(gt["V"], o["V"])
    ett = max(np.max(np.abs(gt["traj_x"] - o["x"])), np.max(np.abs(gt["traj_p"] - o["p"])))
    print(f"{family} d={d}: fp32 iters {np.median(g['iters'])}, max V rel {ev.max():.2e}, "
          f"traj at tol 1e-8 {et:.2e}; at tol {TRAJ_TOL(d):.0e}: iters {np.median(gt['iters'])} "
          f"V rel {evt.max():.2e} traj {ett:.2e}")
    assert ev.max() <= 1e-4
    assert evt.max() <= 1e-4
    assert ett <= 1e-3


def test_quadratic_closed_form_on_gpu():
    """H = |p|^2/2, g = |x|^2/2: V = |x|^2 / (2 (1 + t)) (the 64-point d = 2 workload)."""
    w = W.quadratic_closed_form()
    g = gpu(w, "fp64", tol=1e-24, check_every=1, max_iter=20000)
    exact = np.sum(w["xq"] ** 2, axis=1) / (2.0 * (1.0 + w["t"]))
    assert np.all(g["status"] == O.CONVERGED)
    np.testing.assert_allclose(g["V"], exact, rtol=0, atol=1e-11)
    g = gpu(w, "fp64")            # the workload's own stop (tol 1e-8, max 2000)
    o = oracle_same_stop(w)
    assert np.array_equal(g["iters"], o["iters"])
    assert np.max(value_err(g["V"], o["V"])) <= 1e-9


def test_full_size_quadcopter_sampled():
    """The 4096-point quadcopter workload in the configuration the benchmark times:
    sampled points against the converged oracle, and every point's trajectory
    against the discrete characteristic equations."""
    w = W.quadcopter()
    g = gpu(w, "fp32")
    conv = g["status"] == O.CONVERGED
    assert np.mean(conv) >= 0.995
    assert np.all(g["status"][~conv] == O.MAX_ITER) and np.all(g["iters"][~conv] == w["max_iter"])
    assert np.all(np.isfinite(g["V"]))
    idx = np.random.default_rng(0).choice(np.where(conv)[0], 8, replace=False)
    o = oracle_converged(W.subset(w, idx))
    ev = value_err(g["V"][idx], o["V"])
    print(f"quadcopter 4096: converged {conv.sum()}, median iters {np.median(g['iters'])}, "
          f"sampled V rel {ev.max():.2e}")
    assert ev.max() <= 1e-4
    # trajectories of the sampled points at the tighter stop of the trajectory bar
    # (the whole batch rerun, so each point keeps its own initial guess)
    gt = gpu(w, "fp32", tol=1e-10, kkt=True)
    et = np.max(np.abs(gt["traj_x"][idx] - o["x"]))
    ep = np.max(np.abs(gt["traj_p"][idx] - o["p"]))
    print(f"quadcopter 4096 at tol 1e-10: sampled |dx| {et:.2e} |dp| {ep:.2e}")
    assert et <= 1e-3 and ep <= 1e-3
    # every point of the batch: the oracle's residual of the discrete
    # characteristic equations (Section 4) on the GPU's own trajectory, and the
    # GPU's certificate of it (evaluated in FP32 for FP32 iterates)
    xt, pt = gt["traj_x"].astype(np.float64), gt["traj_p"].astype(np.float64)
    r = O.kkt_residual(w, xt, pt)
    ok = gt["status"] == O.CONVERGED
    print(f"quadcopter 4096 at tol 1e-10: oracle KKT of the GPU trajectories, converged "
          f"points: median {np.median(r[ok]):.2e}, max {r[ok].max():.2e}")
    assert np.mean(ok) >= 0.995 and r[ok].max() <= 2e-4
    from test_kkt_gpu import _qc_fp32_scale     # the FP32 evaluation's derived bar
    assert np.all(np.abs(gt["kkt"] - r) <= 2.0 ** -19 * _qc_fp32_scale(w, xt, pt))
    # the points the GPU reports as not converged are slow for the oracle too
    bad = np.where(~conv)[0][:2]
    if bad.size:
        ob = O.solve(W.subset(w, bad))
        assert np.all(ob["iters"] >= 0.5 * w["max_iter"])


@pytest.mark.parametrize("d", [32, 64, 100])
def test_full_size_tanh_drift_sampled(d):
    w = W.tanh_drift(d, seed={32: 3, 64: 4, 100: 5}[d])
    g = gpu(w, "fp32")
    assert np.all(g["status"] == O.CONVERGED)
    idx = np.random.default_rng(1).choice(len(w["xq"]), 4, replace=False)
    o = oracle_converged(W.subset(w, idx))
    ev = value_err(g["V"][idx], o["V"])
    et = np.max(np.abs(g["traj_x"][idx] - o["x"]))
    print(f"tanh d={d}: median iters {np.median(g['iters'])}, V rel {ev.max():.2e}, traj {et:.2e}")
    assert ev.max() <= 1e-4 and et <= 1e-3


# ---------------------------------------------------------------- edge cases
def test_empty_batch_is_a_no_op():
    from paper_1803_01215_gb300 import binding
    w = _custom("quadratic", 2, 8, B=3)
    prob = binding.Problem.from_workload(w)
    xq = torch.zeros(0, 2, dtype=torch.float64, device="cuda")
    t = torch.zeros(0, dtype=torch.float64, device="cuda")
    out = binding.solve_batch(prob, xq, t, 8, binding.make_opts(sigma=1.0, tau=0.24))
    assert out["V"].numel() == 0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_single_step_and_single_iteration(precision):
    w = _custom("tanh_drift", 4, 1, B=9)
    g = gpu(w, precision, tol=1e-20, check_every=1, max_iter=5000)
    o = oracle_same_stop(w, tol=1e-20, check_every=1, max_iter=5000)
    assert np.max(value_err(g["V"], o["V"])) <= (1e-9 if precision == "fp64" else 1e-4)
    g = gpu(w, precision, max_iter=1, check_every=7)
    o = oracle_same_stop(w, max_iter=1, check_every=7)
    assert np.all(g["iters"] == 1)
    np.testing.assert_allclose(g["traj_x"], o["x"], atol=1e-12 if precision == "fp64" else 1e-6)


def test_zero_radius_and_warm_start_from_oracle_iterate():
    w = _custom("quadcopter", 12, 30, B=11)
    g = gpu(w, "fp64", init_radius=0.0, tol=0.0, max_iter=40, check_every=40)
    o = oracle_same_stop(w, init_radius=0.0, tol=0.0, max_iter=40, check_every=40)
    assert np.max(np.abs(g["traj_x"] - o["x"])) <= 1e-10
    # resume both sides from the same (oracle-produced) iterate
    from paper_1803_01215_gb300 import binding
    prob = binding.Problem.from_workload(w)
    wx = torch.as_tensor(o["x"], device="cuda").contiguous()
    wp = torch.as_tensor(o["p"], device="cuda").contiguous()
    opts = binding.make_opts(sigma=w["sigma"], tau=w["tau"], tol=0.0, max_iter=60,
                             check_every=60, precision="fp64", seed=w["seed"])
    out = binding.solve_batch(prob, torch.as_tensor(w["xq"], device="cuda"),
                              torch.as_tensor(w["t"], device="cuda"), 30, opts,
                              return_traj=True, warm_x=wx, warm_p=wp)
    o2 = O.solve(w, tol=0.0, max_iter=60, check_every=60, x_init=o["x"], p_init=o["p"])
    assert np.max(np.abs(out["traj_x"].cpu().numpy() - o2["x"])) <= 1e-10


def test_point_offset_reproduces_slices_bit_exactly():
    from paper_1803_01215_gb300 import binding
    w = _custom("tanh_drift", 4, 24, B=50)
    full = gpu(w, "fp32")
    prob = binding.Problem.from_workload(w)
    xq = torch.as_tensor(w["xq"][20:35], device="cuda")
    t = torch.as_tensor(w["t"][20:35], device="cuda")
    opts = binding.make_opts(sigma=w["sigma"], tau=w["tau"], tol=w["tol"], max_iter=w["max_iter"],
                             check_every=w["check_every"], seed=w["seed"], point_offset=20)
    part = binding.solve_batch(prob, xq, t, 24, opts, return_traj=True)
    assert np.array_equal(part["V"].cpu().numpy(), full["V"][20:35])
    assert np.array_equal(part["traj_x"].cpu().numpy(), full["traj_x"][20:35])


def test_deterministic():
    w = _custom("quadcopter", 12, 64, B=20)
    a, b = gpu(w, "fp32"), gpu(w, "fp32")
    assert np.array_equal(a["V"], b["V"]) and np.array_equal(a["traj_p"], b["traj_p"])


def test_nonfinite_query_flags_only_that_point():
    w = _custom("tanh_drift", 32, 16, B=6)
    w["xq"][2, 5] = np.nan
    g = gpu(w, "fp32")
    assert g["status"][2] == O.NONFINITE
    assert np.all(g["status"][[0, 1, 3, 4, 5]] == O.CONVERGED)


def test_error_codes():
    from paper_1803_01215_gb300 import binding
    w = _custom("quadratic", 2, 8, B=3)
    prob = binding.Problem.from_workload(w)
    xq = torch.as_tensor(w["xq"], device="cuda")
    t = torch.as_tensor(w["t"], device="cuda")
    with pytest.raises(binding.HJError) as e:
        binding.solve_batch(prob, xq, t, 8, binding.make_opts(sigma=1.0, tau=0.25))
    assert e.value.code == binding.HJ_ERR_STEP_SIZE
    with pytest.raises(binding.HJError) as e:
        binding.solve_batch(prob, xq, t, 0, binding.make_opts(sigma=1.0, tau=0.2))
    assert e.value.code == binding.HJ_ERR_INVALID_ARG
    with pytest.raises(binding.HJError) as e:
        binding.solve_batch(prob, xq, t, 300, binding.make_opts(sigma=1.0, tau=0.2))
    assert e.value.code == binding.HJ_ERR_INVALID_ARG


# ---------------------------------------------------------------- launch shapes and autotuner
@pytest.mark.parametrize("family,d,N", [("quadcopter", 12, 64), ("tanh_drift", 4, 100),
                                        ("quadratic", 3, 120)])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_every_launch_shape_gives_identical_iterates(family, d, N, precision):
    """The lane/warp mapping (G warps per point, NPL nodes per lane) changes no
    formula of a node: after K iterations the iterates agree across shapes to the
    rounding level (instantiations may contract a*b+c into an FMA differently),
    and the values agree to FP64 summation order."""
    from paper_1803_01215_gb300 import binding
    w = _custom(family, d, N, B=21)
    prob = binding.Problem.from_workload(w)
    xq = torch.as_tensor(w["xq"], device="cuda")
    t = torch.as_tensor(w["t"], device="cuda")
    opts = binding.make_opts(sigma=w["sigma"], tau=w["tau"], tol=0.0, max_iter=60,
                             check_every=60, precision=precision, seed=w["seed"])
    outs = []
    for G in (1, 2, 4, 8):
        for npl in ((1, 2) if precision == "fp32" else (1,)):
            if N > 32 * G * npl:
                continue
            binding.set_launch_shape(prob, precision, N, G, npl)
            assert binding.get_launch_shape(prob, precision, N) == (G, npl)
            o = binding.solve_batch(prob, xq, t, N, opts, return_traj=True)
            outs.append(((G, npl), {k: v.cpu().numpy() for k, v in o.items()}))
    assert len(outs) >= 2
    ref = outs[0][1]
    o = oracle_same_stop(w, tol=0.0, max_iter=60, check_every=60)
    assert np.max(np.abs(ref["traj_x"] - o["x"])) <= (1e-10 if precision == "fp64" else 1e-4)
    rt = 1e-13 if precision == "fp64" else 1e-5
    for shape, out in outs[1:]:
        np.testing.assert_allclose(out["traj_x"], ref["traj_x"], rtol=rt, atol=rt, err_msg=str(shape))
        np.testing.assert_allclose(out["traj_p"], ref["traj_p"], rtol=rt, atol=rt, err_msg=str(shape))
        assert np.max(value_err(out["V"], ref["V"])) <= (1e-12 if precision == "fp64" else 1e-6)


def test_autotune_picks_an_instantiated_shape():
    from paper_1803_01215_gb300 import binding
    w = W.quadcopter(B=512)
    prob = binding.Problem.from_workload(w)
    xq = torch.as_tensor(w["xq"], device="cuda")
    t = torch.as_tensor(w["t"], device="cuda")
    opts = binding.make_opts(sigma=w["sigma"], tau=w["tau"], tol=w["tol"], max_iter=w["max_iter"],
                             check_every=w["check_every"], seed=w["seed"])
    G, npl, ms = binding.autotune(prob, xq, t, 64, opts, repeats=1)
    assert G in (1, 2, 4, 8) and npl in (1, 2) and 64 <= 32 * G * npl and ms > 0
    assert binding.get_launch_shape(prob, "fp32", 64) == (G, npl)
    with pytest.raises(binding.HJError) as e:
        binding.set_launch_shape(prob, "fp64", 64, 1, 2)       # no FP64 instantiation with NPL 2
    assert e.value.code == binding.HJ_ERR_UNSUPPORTED


# ---------------------------------------------------------------- large batches, shared-memory kernel
@pytest.mark.parametrize("d,B,precision", [(32, 700, "fp32"), (13, 700, "fp64"), (64, 330, "fp32")])
def test_shared_memory_kernel_large_batches(d, B, precision):
    """Batches larger than the persistent grid (CTAs take several points from the
    work counter, points finish at different iterations): every point
    element-wise against the oracle after a fixed number of iterations, and
    values at the same stop."""
    w = _custom("tanh_drift", d, 24, B=B, seed=51)
    K = 60
    g = gpu(w, precision, tol=0.0, max_iter=K, check_every=K)
    o = oracle_same_stop(w, tol=0.0, max_iter=K, check_every=K)
    tol = 1e-10 if precision == "fp64" else 1e-4
    assert np.all(g["iters"] == K)
    assert np.max(np.abs(g["traj_x"] - o["x"])) <= tol
    assert np.max(np.abs(g["traj_p"] - o["p"])) <= tol
    # the same stop, with points finishing at different iterations and slots refilled
    g = gpu(w, precision, max_iter=3000)
    idx = np.arange(0, B, 37)
    o = oracle_same_stop(W.subset(w, idx), max_iter=3000)
    same = g["iters"][idx] == o["iters"]
    assert np.mean(same) >= 0.8
    bar = 1e-9 if precision == "fp64" else 1e-4
    assert np.max(value_err(g["V"][idx][same], o["V"][same])) <= bar


@pytest.mark.parametrize("family,d,N", [("quadcopter", 12, 16), ("tanh_drift", 4, 9),
                                        ("quadratic", 2, 16), ("eikonal", 10, 10),
                                        ("game_norms", 7, 13)])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_half_warp_groups_match_the_oracle(family, d, N, precision):
    """Half a warp per point (two points per warp, N <= 16): element-wise
    against the oracle after K iterations, for a batch whose size is not a
    multiple of the points per CTA."""
    from oracle import game_pdhg as GO
    from paper_1803_01215_gb300 import binding
    if family == "eikonal":
        w = dict(W.eikonal(d=d, sign=1, B=21, seed=81), N=N)
        w["t"] = np.full(21, N * W.EIK_DELTA)
    elif family == "game_norms":
        w = dict(W.game_norms(d=d, B=21, seed=82), N=N)
        w["t"] = np.full(21, N * W.EIK_DELTA)
    else:
        w = _custom(family, d, N, B=21)
    prob = binding.Problem.from_workload(w)
    binding.set_launch_shape(prob, precision, N, 0, 1)
    assert binding.get_launch_shape(prob, precision, N) == (0, 1)
    xq = torch.as_tensor(w["xq"], device="cuda")
    t = torch.as_tensor(w["t"], device="cuda")
    K = 90
    opts = binding.make_opts(sigma=w["sigma"], tau=w["tau"], tol=0.0, max_iter=K, check_every=K,
                             precision=precision, seed=w["seed"])
    g = {k: v.cpu().numpy() for k, v in
         binding.solve_batch(prob, xq, t, N, opts, return_traj=True).items()}
    solve = GO.solve_game if family == "game_norms" else oracle_same_stop
    o = solve(w, tol=0.0, max_iter=K, check_every=K)
    assert np.all(g["iters"] == K)
    tol = 1e-10 if precision == "fp64" else 1e-4
    tol_p = tol * max(1.0, w["sigma"] / 25.0) if precision == "fp32" else tol
    assert np.max(np.abs(g["traj_x"] - o["x"])) <= tol
    assert np.max(np.abs(g["traj_p"] - o["p"])) <= tol_p
    assert np.max(value_err(g["V"], o["V"])) <= (1e-9 if precision == "fp64" else 1e-4)
    with pytest.raises(binding.HJError):
        binding.set_launch_shape(prob, precision, 17, 0, 1)        # 16 lanes hold N <= 16


def test_gpu_trajectories_certified_by_the_kkt_residual():
    """Any trajectory, GPU or CPU, is certified by the discrete characteristic
    equations evaluated in FP64 (the oracle's kkt_residual): the FP64 path's
    converged iterates satisfy them to 1e-9, the FP32 path's to its rounding,
    and the two precisions land on the same saddle (same value to 1e-4)."""
    w = W.quadcopter(B=16, seed=41, N=32, t=0.5)
    g64 = gpu(w, "fp64", tol=1e-24, check_every=16, max_iter=100000)
    g32 = gpu(w, "fp32", tol=1e-11, check_every=16, max_iter=100000)
    r64 = O.kkt_residual(w, g64["traj_x"], g64["traj_p"])
    r32 = O.kkt_residual(w, g32["traj_x"].astype(np.float64), g32["traj_p"].astype(np.float64))
    print(f"KKT residual: FP64 max {r64.max():.2e}, FP32 max {r32.max():.2e}")
    assert r64.max() <= 1e-9
    assert r32.max() <= 1e-4
    assert value_err(g32["V"], g64["V"]).max() <= 1e-4
