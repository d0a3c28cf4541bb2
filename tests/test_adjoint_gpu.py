"""Adjoint of the value (hj_solve_grad behind torch.autograd) against central
finite differences (h = 1e-4) of the FP64 oracle's converged value, the closed
form, and the costate p_N."""
import numpy as np
import pytest

from oracle import lax_pdhg as O
from paper_1803_01215_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TIGHT = dict(tol=1e-24, check_every=1, max_iter=200000)


def _mean_V(w):
    return float(np.mean(O.solve(w, **TIGHT)["V"]))


def _fd(w, field, i, h=1e-4):
    wp, wm = dict(w), dict(w)
    vp = np.array(w[field], dtype=float).copy(); vp.reshape(-1)[i] += h
    vm = np.array(w[field], dtype=float).copy(); vm.reshape(-1)[i] -= h
    wp[field], wm[field] = vp, vm
    return (_mean_V(wp) - _mean_V(wm)) / (2 * h)


def _gpu_grads(w, precision):
    from paper_1803_01215_gb300.autograd import hj_value
    xq = torch.as_tensor(w["xq"], device="cuda").requires_grad_(True)
    t = torch.as_tensor(w["t"], device="cuda")
    Wt = torch.as_tensor(w["W"]).requires_grad_(True)
    ct = torch.as_tensor(w["c"]).requires_grad_(True)
    dyn = torch.as_tensor(w["dyn"]).requires_grad_(w["dyn"].size > 0)
    tol = 1e-24 if precision == "fp64" else 1e-11
    V, it, st = hj_value(xq, t, Wt, ct, dyn, family=w["family"], N=w["N"], sigma=w["sigma"],
                         tau=w["tau"], tol=tol, check_every=1, max_iter=100000,
                         precision=precision, seed=w["seed"], init_radius=w["init_radius"])
    V.mean().backward()
    return dict(V=V.detach().cpu().numpy(), st=st.cpu().numpy(), dxq=xq.grad.cpu().numpy(),
                dW=Wt.grad.cpu().numpy(), dc=ct.grad.cpu().numpy(),
                ddyn=(dyn.grad.cpu().numpy() if dyn.grad is not None else None))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_quadcopter_gradient_vs_finite_differences(precision):
    w = W.quadcopter(B=3, seed=31, N=10, t=0.4)
    g = _gpu_grads(w, precision)
    rt = 1e-6 if precision == "fp64" else 2e-3
    def close(a, b):
        return abs(a - b) <= rt * max(1.0, abs(b))
    for i in range(12):
        fd = _fd(w, "W", i)
        assert close(g["dW"][i], fd), ("W", i, g["dW"][i], fd)
    for i, name in enumerate(["m", "a_h", "g_z", "eps"]):
        fd = _fd(w, "dyn", i)
        assert close(g["ddyn"][i], fd), (name, g["ddyn"][i], fd)
    for k in (0, 4, 7, 11):
        fd = _fd(w, "xq", np.ravel_multi_index((1, k), w["xq"].shape))
        assert close(g["dxq"][1, k], fd), ("xq", k, g["dxq"][1, k], fd)


def test_tanh_drift_gradient_vs_finite_differences():
    w = W.tanh_drift(3, B=3, seed=32, N=8)
    w["sigma"], w["tau"] = 1.0, 0.24
    g = _gpu_grads(w, "fp64")
    for i in range(9):
        fd = _fd(w, "dyn", i)
        assert abs(g["ddyn"][i] - fd) <= 1e-6 * max(1.0, abs(fd)), ("A", i, g["ddyn"][i], fd)
    for i in range(3):
        fd = _fd(w, "c", i)
        assert abs(g["dc"][i] - fd) <= 1e-6 * max(1.0, abs(fd)), ("c", i)
    fd = _fd(w, "xq", 4)
    assert abs(g["dxq"][1, 1] - fd) <= 1e-6 * max(1.0, abs(fd))


def test_quadratic_gradient_is_the_costate_and_the_closed_form():
    """H = |p|^2/2: dV/dx_q = p_N exactly, and for g = |x|^2/2, V = |x|^2/(2(1+t))
    gives dV/dx = x/(1+t)."""
    w = W.quadratic_closed_form(B=8)
    g = _gpu_grads(w, "fp64")
    B = len(w["xq"])
    np.testing.assert_allclose(g["dxq"] * B, w["xq"] / (1.0 + w["t"][:, None]), atol=1e-10)
    o = O.solve(w, **TIGHT)
    np.testing.assert_allclose(g["dxq"] * B, o["p"][:, -1, :], atol=1e-10)


def test_full_size_adjoint_sampled():
    """The 4096-point quadcopter batch: FP32 gradient of mean V; sampled per-point
    gradients dV_b/dx_q against finite differences of the oracle, and the
    O(delta) gap to the costate p_N reported."""
    from paper_1803_01215_gb300 import binding
    w = W.quadcopter()
    prob = binding.Problem.from_workload(w)
    xq = torch.as_tensor(w["xq"], device="cuda")
    t = torch.as_tensor(w["t"], device="cuda")
    opts = binding.make_opts(sigma=w["sigma"], tau=w["tau"], tol=1e-10, max_iter=20000,
                             check_every=16, seed=w["seed"])
    out = binding.solve_batch(prob, xq, t, 64, opts, return_traj=True)
    B = len(w["xq"])
    wts = torch.full((B,), 1.0 / B, dtype=torch.float64, device="cuda")
    g = binding.solve_grad(prob, t, 64, "fp32", out["traj_x"], out["traj_p"], wts)
    dxq = g["dxq"].cpu().numpy() * B
    assert np.all(np.isfinite(dxq)) and np.all(np.isfinite(g["dW"].cpu().numpy()))
    pN = out["traj_p"].cpu().numpy()[:, -1, :]
    print(f"max |dV/dx - p_N| = {np.max(np.abs(dxq - pN)):.3e} (O(delta), delta = 1/64)")
    for b in (7, 1234):
        sub = W.subset(w, [b])
        for k in (2, 5, 8):
            h = 1e-4
            sp, sm = dict(sub), dict(sub)
            sp["xq"] = sub["xq"].copy(); sp["xq"][0, k] += h
            sm["xq"] = sub["xq"].copy(); sm["xq"][0, k] -= h
            fd = (O.solve(sp, **TIGHT)["V"][0] - O.solve(sm, **TIGHT)["V"][0]) / (2 * h)
            assert abs(dxq[b, k] - fd) <= 2e-3 * max(1.0, abs(fd)), (b, k, dxq[b, k], fd)


# ---------------------------------------------------------------- reverse sweep through the iterations
def _fd_fixed(w, field, i, K, h=1e-5):
    """Central difference of the oracle's mean value after exactly K iterations."""
    def meanV(ww):
        return float(np.mean(O.solve(ww, tol=0.0, max_iter=K, check_every=K)["V"]))
    wp, wm = dict(w), dict(w)
    vp = np.array(w[field], dtype=float).copy(); vp.reshape(-1)[i] += h
    vm = np.array(w[field], dtype=float).copy(); vm.reshape(-1)[i] -= h
    wp[field], wm[field] = vp, vm
    return (meanV(wp) - meanV(wm)) / (2 * h)


def _unrolled(w, precision, K, ckpt):
    from paper_1803_01215_gb300 import binding
    prob = binding.Problem.from_workload(w)
    xq = torch.as_tensor(w["xq"], device="cuda")
    t = torch.as_tensor(w["t"], device="cuda")
    opts = binding.make_opts(sigma=w["sigma"], tau=w["tau"], tol=0.0, max_iter=K, check_every=K,
                             precision=precision, seed=w["seed"], init_radius=w["init_radius"])
    out = binding.solve_batch(prob, xq, t, int(w["N"]), opts)
    B = xq.shape[0]
    wts = torch.full((B,), 1.0 / B, dtype=torch.float64, device="cuda")
    g = binding.solve_grad_unrolled(prob, xq, t, int(w["N"]), opts, out["iters"], wts,
                                    checkpoint_every=ckpt)
    return {k: v.cpu().numpy() for k, v in g.items()}


@pytest.mark.parametrize("ckpt", [7, 32])
def test_unrolled_adjoint_quadcopter_vs_finite_differences(ckpt):
    """Exact gradient of the value after K = 40 iterations (not converged):
    W, (m, a_h, g_z, eps) and x_q against central differences of the oracle
    run for the same 40 iterations; checkpoint spacings that do and do not
    divide K."""
    w = W.quadcopter(B=3, seed=33, N=10, t=0.4)
    K = 40
    g = _unrolled(w, "fp64", K, ckpt)
    def close(a, b):
        return abs(a - b) <= 1e-6 * max(1.0, abs(b))
    for i in (0, 3, 6, 11):
        fd = _fd_fixed(w, "W", i, K)
        assert close(g["dW"][i], fd), ("W", i, g["dW"][i], fd)
    for i, name in enumerate(["m", "a_h", "g_z", "eps"]):
        fd = _fd_fixed(w, "dyn", i, K)
        assert close(g["ddyn"][i], fd), (name, g["ddyn"][i], fd)
    for k in (0, 4, 7, 11):
        fd = _fd_fixed(w, "xq", np.ravel_multi_index((2, k), w["xq"].shape), K)
        assert close(g["dxq"][2, k], fd), ("xq", k, g["dxq"][2, k], fd)


def test_unrolled_adjoint_quadratic_and_converged_agreement():
    """H = |p|^2/2, d = 2: the unrolled gradient after K iterations matches finite
    differences; run to convergence it matches the closed form x/(1+t)."""
    w = W.quadratic_closed_form(B=6)
    K = 25
    g = _unrolled(w, "fp64", K, 8)
    for k in range(2):
        fd = _fd_fixed(w, "xq", np.ravel_multi_index((1, k), w["xq"].shape), K)
        assert abs(g["dxq"][1, k] - fd) <= 1e-7 * max(1.0, abs(fd))
    fd = _fd_fixed(w, "c", 0, K)
    assert abs(g["dc"][0] - fd) <= 1e-7 * max(1.0, abs(fd))
    gk = _unrolled(w, "fp64", 2000, 32)
    np.testing.assert_allclose(gk["dxq"] * 6, w["xq"] / (1.0 + w["t"][:, None]), atol=1e-6)


def test_unrolled_matches_envelope_at_convergence_fp32():
    """The 12-D problem run to a tight stop: the reverse sweep and the envelope
    gradient agree (both are the gradient of the converged value)."""
    from paper_1803_01215_gb300 import binding
    w = W.quadcopter(B=64, seed=34, N=16, t=0.5)
    prob = binding.Problem.from_workload(w)
    xq = torch.as_tensor(w["xq"], device="cuda")
    t = torch.as_tensor(w["t"], device="cuda")
    opts = binding.make_opts(sigma=w["sigma"], tau=w["tau"], tol=1e-10, max_iter=20000,
                             check_every=16, seed=w["seed"])
    out = binding.solve_batch(prob, xq, t, 16, opts, return_traj=True)
    wts = torch.full((64,), 1.0 / 64, dtype=torch.float64, device="cuda")
    ge = binding.solve_grad(prob, t, 16, "fp32", out["traj_x"], out["traj_p"], wts)
    gu = binding.solve_grad_unrolled(prob, xq, t, 16, opts, out["iters"], wts, checkpoint_every=32)
    for key in ("dW", "ddyn", "dxq"):
        a, b = gu[key].cpu().numpy(), ge[key].cpu().numpy()
        assert np.max(np.abs(a - b)) <= 2e-3 * max(1.0, np.max(np.abs(b))), key


def _fd_tol(w, field, i, tol, h=1e-4):
    wp, wm = dict(w), dict(w)
    vp = np.array(w[field], dtype=float).copy(); vp.reshape(-1)[i] += h
    vm = np.array(w[field], dtype=float).copy(); vm.reshape(-1)[i] -= h
    wp[field], wm[field] = vp, vm
    kw = dict(tol=tol, check_every=1, max_iter=200000)
    return (np.mean(O.solve(wp, **kw)["V"]) - np.mean(O.solve(wm, **kw)["V"])) / (2 * h)


@pytest.mark.parametrize("sign,moving", [(1, False), (-1, False), (1, True)])
def test_eikonal_gradient_vs_finite_differences(sign, moving):
    """Envelope gradient of the eikonal value (Section 6.1's bump, the negative
    equation through phi = -psi, the moving bump) against central differences
    of the FP64 oracle's converged value: cost weights and centre, the speed's
    c0, c1, c2, the bump centre and velocity, and the query point."""
    w = (W.eikonal_moving(d=2, B=3, seed=57) if moving else
         W.eikonal(d=2, sign=sign, B=3, seed=56))
    w["N"] = 6
    w["t"] = np.full(3, 6 * W.EIK_DELTA)
    tol = 1e-20 if sign < 0 else 1e-24
    g = _gpu_grads(w, "fp64")
    def close(a, b):
        return abs(a - b) <= 2e-5 * max(1.0, abs(b))
    for field, i, got in [("W", 0, g["dW"][0]), ("c", 1, g["dc"][1]),
                          ("dyn", 1, g["ddyn"][1]), ("dyn", 2, g["ddyn"][2]),
                          ("dyn", 3, g["ddyn"][3]), ("dyn", 4, g["ddyn"][4]),
                          ("dyn", 5, g["ddyn"][5])] + \
                         ([("dyn", 6, g["ddyn"][6]), ("dyn", 7, g["ddyn"][7])] if moving else []):
        fd = _fd_tol(w, field, i, tol)
        assert close(got, fd), (field, i, got, fd)
    for k in (0, 1):
        fd = _fd_tol(w, "xq", np.ravel_multi_index((1, k), w["xq"].shape), tol)
        assert close(g["dxq"][1, k], fd), ("xq", k, g["dxq"][1, k], fd)
    assert g["ddyn"][0] == 0.0
