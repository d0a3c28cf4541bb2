"""The per-point residual of the discrete characteristic equations (Section 4)
that the CUDA path returns (hj_solve_batch's kkt output, hj_kkt_residual),
against the oracle's kkt_residual (pinned by tests/test_oracle_kkt_pins.py)
evaluated on the very trajectories the GPU returned.

Both sides evaluate the same formula from the same iterates.  The GPU does so
in FP64, so the two agree to FP64 rounding (1e-12 absolute and relative),
except for the quadcopter's FP32 iterates, which it evaluates in FP32 (sines
and cosines from the accurate sincosf): there the bar is 32 units of 2^-24
times the magnitudes that enter the residual (_qc_fp32_scale).  The iterates are taken after a fixed number of iterations, far
from the saddle, so every part of the residual is large and exercised; at
convergence the FP64 path certifies its points below 1e-9 and the FP32 path at
its rounding level.
"""
import numpy as np
import pytest

from gpu_common import gpu
from oracle import lax_pdhg as O
from paper_1803_01215_gb300 import workloads as W
from test_parity_gpu import _custom

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _eik(d, sign, t=0.2, B=29, moving=False):
    w = W.eikonal(d=d, sign=sign, t=t, B=B, seed=5)
    if moving:
        w = W.eikonal_moving(t=t, B=B, seed=5, d=d)
    return w


# (case, workload factory, which kernel serves it)
CASES = [
    ("quadcopter_N64", lambda: _custom("quadcopter", 12, 64, B=37), "register"),
    ("quadcopter_N23", lambda: _custom("quadcopter", 12, 23, B=37), "register"),
    ("quadratic_d3", lambda: _custom("quadratic", 3, 37, B=37), "register"),
    ("quadratic_d6", lambda: _custom("quadratic", 6, 20, B=37), "shared-memory"),
    ("tanh_d4", lambda: _custom("tanh_drift", 4, 50, B=37), "register"),
    ("tanh_d13", lambda: _custom("tanh_drift", 13, 21, B=37), "tiled / shared-memory"),
    ("tanh_d32", lambda: _custom("tanh_drift", 32, 32, B=21), "tiled / shared-memory"),
    ("eik_d2_pos", lambda: _eik(2, 1), "register"),
    ("eik_d10_neg", lambda: _eik(10, -1), "register"),
    ("eik_d5_neg", lambda: _eik(5, -1), "coordinate-parallel"),
    ("eik_d37_pos", lambda: _eik(37, 1), "coordinate-parallel"),
    ("eik_moving_d2", lambda: _eik(2, 1, moving=True), "register"),
]


def _qc_fp32_scale(w, x, p):
    """Per point: the largest magnitude entering the quadcopter's r1 and r3 at one
    node (infinity norms): |x_j| + |x_{j-1}| + |p_j| + |p_{j+1}| plus delta times
    the terms of grad_p H (a_h |a| + g_z + |a| |u0| / m + eps |p_j|, |a| = 1,
    |u0| <= sqrt(3) |p_j| / m) and of grad_x H ((a_h + |u0| / m) 3 |p_j|)."""
    m, a_h, g_z, eps = (float(v) for v in w["dyn"][:4])
    N = x.shape[1] - 1
    out = np.zeros(x.shape[0])
    for b in range(x.shape[0]):
        delta = float(w["t"][b]) / N
        s = 0.0
        for j in range(1, N + 1):
            pj = np.max(np.abs(p[b, j]))
            pr = np.max(np.abs(p[b, j + 1])) if j < N else 0.0
            u0 = np.sqrt(3.0) * pj / m
            s = max(s, np.max(np.abs(x[b, j])) + np.max(np.abs(x[b, j - 1])) + pj + pr
                    + delta * (a_h + g_z + u0 / m + eps * pj + (a_h + u0 / m) * 3.0 * pj))
        out[b] = s
    return out


def _kkt_case(name, make, precision, K=120, **kw):
    w = make()
    g = gpu(w, precision, tol=0.0, max_iter=K, check_every=K, kkt=True, **kw)
    x = g["traj_x"].astype(np.float64)
    p = g["traj_p"].astype(np.float64)
    ref = O.kkt_residual(w, x, p)
    return w, g, ref


@pytest.mark.parametrize("name,make,kernel", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_kkt_output_matches_the_oracle_residual(name, make, kernel, precision):
    w, g, ref = _kkt_case(name, make, precision)
    err = np.abs(g["kkt"] - ref)
    print(f"{name} ({kernel}) {precision}: kkt in [{ref.min():.2e}, {ref.max():.2e}], "
          f"max |gpu - oracle| = {err.max():.2e}")
    assert np.all(np.isfinite(g["kkt"]))
    assert ref.max() > 1e-4                     # far from the saddle: the terms are live
    if precision == "fp32" and name.startswith("quadcopter"):
        # FP32 evaluation: each term of r1 and r3 carries a few roundings of 2^-24
        # relative to the magnitudes that enter it (sincosf within 2 ulp)
        bar = 2.0 ** -19 * _qc_fp32_scale(w, g["traj_x"].astype(np.float64),
                                          g["traj_p"].astype(np.float64))
        print(f"  FP32 evaluation bar: {bar.min():.2e} .. {bar.max():.2e}")
        assert np.all(err <= bar)
    else:
        assert np.all(err <= 1e-12 + 1e-12 * ref)


SOME = [c for c in CASES if c[0] in ("tanh_d13", "tanh_d32", "eik_d5_neg", "quadcopter_N64")]


@pytest.mark.parametrize("name,make,kernel", SOME, ids=[c[0] for c in SOME])
def test_kkt_without_trajectories_and_the_standalone_entry_point(name, make, kernel):
    """The kkt output needs no trajectory arguments (a workspace holds them), and
    hj_kkt_residual on the returned trajectories gives the same numbers."""
    from paper_1803_01215_gb300 import binding
    w = make()
    prob = binding.Problem.from_workload(w)
    opts = binding.make_opts(sigma=w["sigma"], tau=w["tau"], tol=0.0, max_iter=90, check_every=90,
                             precision="fp32", seed=w["seed"], init_radius=w["init_radius"])
    xq = torch.as_tensor(w["xq"], device="cuda")
    t = torch.as_tensor(w["t"], device="cuda")
    N = int(w["N"])
    with_traj = binding.solve_batch(prob, xq, t, N, opts, return_traj=True, kkt=True)
    bare = binding.solve_batch(prob, xq, t, N, opts, kkt=True)
    alone = binding.kkt_residual(prob, t, N, "fp32", with_traj["traj_x"], with_traj["traj_p"])
    torch.cuda.synchronize()
    assert torch.equal(bare["kkt"], with_traj["kkt"])
    assert torch.allclose(alone, with_traj["kkt"], rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("family,d,N", [("quadcopter", 12, 32), ("tanh_drift", 4, 32),
                                        ("tanh_drift", 32, 32), ("quadratic", 6, 16)])
def test_converged_points_are_certified(family, d, N):
    """At convergence the residual certifies each point: FP64 below 1e-9, FP32 at
    its rounding level (below 1e-4)."""
    if family == "quadcopter":                  # the workload's step sizes (sigma = 1.4)
        w = W.quadcopter(B=24, seed=43, N=N, t=0.5)
    else:
        w = _custom(family, d, N, B=24, t=0.5)
    g64 = gpu(w, "fp64", tol=1e-24, check_every=16, max_iter=100000, kkt=True)
    g32 = gpu(w, "fp32", tol=1e-11, check_every=16, max_iter=100000, kkt=True)
    print(f"{family} d={d}: kkt FP64 max {g64['kkt'].max():.2e}, FP32 max {g32['kkt'].max():.2e}")
    assert np.all(g64["status"] == 0) and g64["kkt"].max() <= 1e-9
    assert g32["kkt"].max() <= 1e-4
    x32, p32 = g32["traj_x"].astype(np.float64), g32["traj_p"].astype(np.float64)
    r32 = O.kkt_residual(w, x32, p32)
    if family == "quadcopter":                  # evaluated in FP32 (see the module docstring)
        assert np.all(np.abs(g32["kkt"] - r32) <= 2.0 ** -19 * _qc_fp32_scale(w, x32, p32))
    else:
        np.testing.assert_allclose(g32["kkt"], r32, rtol=1e-12, atol=1e-13)


def test_hopf_form_kkt():
    """The Hopf form returns x_0 = grad g*(p_1), so the same equations hold at its
    saddle (Algorithm 2); the residual matches the oracle's on the returned arrays."""
    w = W.quadcopter(B=16, seed=44, N=32, t=0.5)
    g = gpu(w, "fp64", tol=0.0, max_iter=100, check_every=100, kkt=True, formulation="hopf")
    ref = O.kkt_residual(w, g["traj_x"], g["traj_p"])
    assert np.all(np.abs(g["kkt"] - ref) <= 1e-12 + 1e-12 * ref)
    gc = gpu(w, "fp64", tol=1e-24, check_every=16, max_iter=100000, kkt=True, formulation="hopf")
    assert np.all(gc["status"] == 0) and gc["kkt"].max() <= 1e-9


def test_kkt_refused_where_undefined():
    from paper_1803_01215_gb300 import binding
    wg = W.game_norms(d=2, t=0.1, B=8)
    with pytest.raises(binding.HJError) as e:
        gpu(wg, "fp32", kkt=True)
    assert e.value.code == binding.HJ_ERR_UNSUPPORTED
    wq = _custom("quadcopter", 12, 16, B=4)
    with pytest.raises(binding.HJError) as e:
        gpu(wq, "fp32", kkt=True, scheme="trap")
    assert e.value.code == binding.HJ_ERR_UNSUPPORTED
