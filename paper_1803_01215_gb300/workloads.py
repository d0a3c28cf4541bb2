"""Seeded synthetic workloads for the batched Lax/PDHG Hamilton-Jacobi solver.

This module only draws numbers: problem parameters and query points shaped
like the paper's examples (Section 6: quadcopter-class 12-D control, Eq. for
the eikonal dimension-scaling study, the quadratic closed-form case).  It
holds none of the method's arithmetic, so both the CUDA path and the FP64
oracle may take their inputs from here.  It imports nothing else from this
package.

Every workload is a plain dict:

    family      "quadratic" | "quadcopter" | "tanh_drift"
    d           state dimension
    dyn         dynamics parameters (float64 ndarray)
                  quadratic : empty
                  quadcopter: [m, a_h, g_z, eps]  (mass, hover thrust gain,
                              gravity, weight of the full-state disturbance input)
                  tanh_drift: A, d*d row-major
    W, c        terminal cost g(x) = 1/2 sum_i W_i^2 (x_i - c_i)^2
    xq          [B, d] float64 query points
    t           [B] float64 horizons
    N           int (uniform) or [B] int32 (ragged) number of time steps
    sigma, tau  PDHG step sizes (tau * sigma * 4 < 1, the bound ||D||^2 < 4)
    tol, max_iter, check_every, seed, init_radius
"""
import numpy as np

FAMILIES = {"quadratic": 0, "quadcopter": 1, "tanh_drift": 2, "eikonal": 3, "game_norms": 4}

# Quadcopter constants: unit mass, hover thrust gain equal to gravity so that
# the level-attitude state is an equilibrium of the drift.
QC_MASS = 1.0
QC_GRAVITY = 9.81
QC_HOVER = 9.81
# H gains eps |p|^2 / 2 (disturbance input with cost |w|^2 / (2 eps)); with the
# rank-4 thrust/torque input alone the Lax saddle problem does not converge.
QC_EPS = 1.0


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def quadratic_closed_form(B=64, seed=1):
    """H = |p|^2/2, g = |x|^2/2, d = 2, x ~ U[-2,2]^2, t = 1, N = 20."""
    r = _rng(seed)
    d = 2
    return dict(family="quadratic", d=d, dyn=np.zeros(0),
                W=np.ones(d), c=np.zeros(d),
                xq=r.uniform(-2.0, 2.0, size=(B, d)), t=np.ones(B), N=20,
                sigma=0.5, tau=0.48, tol=1e-8, max_iter=2000, check_every=1,
                seed=seed, init_radius=0.1)


def quadcopter(B=4096, seed=2, N=64, t=1.0):
    """12-D quadcopter-class control, x ~ N(0, 0.5^2 I), W = diag U[0.5, 2], x* = 0."""
    r = _rng(seed)
    d = 12
    W = r.uniform(0.5, 2.0, size=d)
    xq = 0.5 * r.standard_normal((B, d))
    return dict(family="quadcopter", d=d,
                dyn=np.array([QC_MASS, QC_HOVER, QC_GRAVITY, QC_EPS]),
                W=W, c=np.zeros(d), xq=xq, t=np.full(B, float(t)), N=N,
                sigma=QC_SIGMA, tau=0.24 / QC_SIGMA, tol=1e-8, max_iter=20000,
                check_every=16, seed=seed, init_radius=0.1)


def tanh_drift(d, B=16384, seed=3, N=32):
    """H = <p, tanh(Ax)> + |p|^2/2, A ~ N(0,1)/sqrt(d), g = |x - c|^2/2, c ~ N(0, I),
    x ~ N(0, I), t ~ U[0.5, 2]."""
    r = _rng(seed)
    A = r.standard_normal((d, d)) / np.sqrt(d)
    c = r.standard_normal(d)
    xq = r.standard_normal((B, d))
    t = r.uniform(0.5, 2.0, size=B)
    return dict(family="tanh_drift", d=d, dyn=A.reshape(-1).copy(),
                W=np.ones(d), c=c, xq=xq, t=t, N=N,
                sigma=TD_SIGMA, tau=0.24 / TD_SIGMA, tol=1e-8, max_iter=20000,
                check_every=16, seed=seed, init_radius=0.1)


# Step sizes chosen on the oracle (sigma sweep at tau = 0.24 / sigma); the fixed
# point does not depend on them, only the iteration count does.
QC_SIGMA = 1.4
TD_SIGMA = 1.0


EIK_DELTA = 0.02            # time step of Section 6.1's eikonal runs
EIK_G_CONST = -0.5          # g(x) = -1/2 + 1/2 <A^-1 x, x>: the constant shifts V


def eikonal(d=2, sign=1, t=0.2, B=None, grid_step=0.1, seed=8):
    """Section 6.1's eikonal problems: phi_t + sign c(x)|grad phi| = 0 with
    c(x) = 1 + 3 exp(-4 |x - (1, 1, 0, ..., 0)|^2) and
    g(x) = -1/2 + 1/2 <A^-1 x, x>, A = diag(2.5^2, 1, 0.5^2, ..., 0.5^2)
    (W = (1/2.5, 1, 2, ..., 2), c = 0; the constant -1/2 is EIK_G_CONST, added
    to V by the caller).  Query points on the 2-D slice [-3, 3]^2 x {0}^(d-2):
    the grid of mesh grid_step (B None) or B uniform draws.  delta = 0.02
    (N = t / 0.02); sigma = 0.5 for sign +1 (the paper's choice away from the
    bump) and 100 for sign -1, tau = 0.24 / sigma."""
    r = _rng(seed)
    if B is None:
        ax = np.arange(-3.0, 3.0 + 1e-9, grid_step)
        a, b = np.meshgrid(ax, ax, indexing="ij")
        pts = np.stack([a.ravel(), b.ravel()], axis=1)
    else:
        pts = r.uniform(-3.0, 3.0, size=(B, 2))
    xq = np.zeros((len(pts), d))
    xq[:, :2] = pts
    W = np.full(d, 2.0)
    W[0], W[1] = 1.0 / 2.5, 1.0
    xb = np.zeros(d)
    xb[:2] = 1.0
    N = int(round(t / EIK_DELTA))
    sigma = 0.5 if sign > 0 else 100.0
    return dict(family="eikonal", d=d, dyn=np.concatenate([[float(sign), 1.0, 3.0, 4.0], xb]),
                W=W, c=np.zeros(d), xq=xq, t=np.full(len(pts), float(t)), N=N,
                sigma=sigma, tau=0.24 / sigma, tol=1e-8, max_iter=20000, check_every=16,
                seed=seed, init_radius=0.1, g_const=EIK_G_CONST)


def eikonal_moving(t=0.2, B=None, grid_step=0.1, seed=8, d=2):
    """Section 6.1's state-and-time-dependent eikonal: H(x, p, s) = c(x - s v_b)|p|
    with the bump of eikonal() moving with velocity v_b = (-1, 1, 0, ...), the
    positive equation, the same g, delta = 0.02 and sigma = 0.5 (tau = 0.24 / sigma)."""
    w = eikonal(d=d, sign=1, t=t, B=B, grid_step=grid_step, seed=seed)
    vb = np.zeros(d)
    vb[0], vb[1] = -1.0, 1.0
    w["dyn"] = np.concatenate([w["dyn"], vb])
    return w


def game_norms(d=2, t=0.1, B=None, grid_step=1.0 / 12.0, seed=9):
    """Section 6.2's difference-of-norms game: z = (x, y) with x = z[0] (d1 = 1)
    and y = z[1..d), H = c1(z)|p| - c2(z)|q|, c1(z) = 1 + 3 exp(-4 |z - (1, 1, 0, ...)|^2),
    c2(z) = c1(-z), and the eikonal example's data g(z) = -1/2 + 1/2 <A^-1 z, z>
    (W = (1/2.5, 1, 2, ..., 2), c = 0; the -1/2 is EIK_G_CONST).  Query points on
    the 2-D slice [-3, 3]^2 x {0}^(d-2): the grid of mesh grid_step (1/12, the
    paper's; B None) or B uniform draws.  delta = 0.02, sigma = 50, tau = 0.24 / sigma."""
    r = _rng(seed)
    if B is None:
        ax = np.linspace(-3.0, 3.0, int(round(6.0 / grid_step)) + 1)
        a, b = np.meshgrid(ax, ax, indexing="ij")
        pts = np.stack([a.ravel(), b.ravel()], axis=1)
    else:
        pts = r.uniform(-3.0, 3.0, size=(B, 2))
    zq = np.zeros((len(pts), d))
    zq[:, :2] = pts
    W = np.full(d, 2.0)
    W[0], W[1] = 1.0 / 2.5, 1.0
    zb = np.zeros(d)
    zb[:2] = 1.0
    sigma = 50.0
    return dict(family="game_norms", d=d, dyn=np.concatenate([[1.0, 1.0, 3.0, 4.0], zb]),
                W=W, c=np.zeros(d), xq=zq, t=np.full(len(pts), float(t)),
                N=int(round(t / EIK_DELTA)), sigma=sigma, tau=0.24 / sigma, tol=1e-8,
                max_iter=20000, check_every=16, seed=seed, init_radius=0.1,
                g_const=EIK_G_CONST)


def subset(w, idx):
    """The same workload restricted to the points `idx` (global point indices
    are kept in 'point_index' so the counter-based initial guess is unchanged)."""
    idx = np.asarray(idx)
    out = dict(w)
    out["xq"] = w["xq"][idx]
    out["t"] = w["t"][idx]
    if not np.isscalar(w["N"]):
        out["N"] = np.asarray(w["N"])[idx]
    base = w.get("point_index")
    out["point_index"] = (np.asarray(base)[idx] if base is not None
                          else idx.astype(np.int64))
    return out


def ragged_mix(B=100000, seed=6, sigma=1.4):
    """Ragged batch: thirds of tanh drift d = 4, the 12-D quadcopter and tanh drift
    d = 32 (problem parameters from the generators above), each point with its own
    N ~ U{16..256} and the horizon its generator draws.  Returns
        problems  list of three problem dicts (family, d, dyn, W, c)
        prob_of   [B] int32 problem index,  N_of [B] int32,
        xq        list of B arrays (d_b,),  t [B]
    plus the shared solver options."""
    r = _rng(seed)
    gens = [tanh_drift(4, B=1, seed=seed + 100), quadcopter(B=1, seed=seed + 200),
            tanh_drift(32, B=1, seed=seed + 300)]
    problems = [{k: g[k] for k in ("family", "d", "dyn", "W", "c")} for g in gens]
    prob_of = r.integers(0, 3, size=B).astype(np.int32)
    N_of = r.integers(16, 257, size=B).astype(np.int32)
    xq, t = [], np.empty(B)
    for b in range(B):
        k = prob_of[b]
        if k == 1:
            xq.append(0.5 * r.standard_normal(12))
            t[b] = 1.0
        else:
            xq.append(r.standard_normal(problems[k]["d"]))
            t[b] = r.uniform(0.5, 2.0)
    return dict(problems=problems, prob_of=prob_of, N_of=N_of, xq=xq, t=t,
                sigma=sigma, tau=0.24 / sigma, tol=1e-8, max_iter=20000, check_every=16,
                seed=seed, init_radius=0.1)


def ragged_group(rw, k, N, idx=None):
    """The points of ragged workload `rw` with problem k and time steps N (or the
    given global indices) as a uniform workload dict for the oracle; global point
    indices are kept so the counter-based initial guess matches."""
    if idx is None:
        idx = np.where((rw["prob_of"] == k) & (rw["N_of"] == N))[0]
    out = dict(rw["problems"][k])
    out.update(xq=np.stack([rw["xq"][i] for i in idx]), t=rw["t"][idx], N=int(N),
               point_index=np.asarray(idx, dtype=np.int64),
               **{key: rw[key] for key in ("sigma", "tau", "tol", "max_iter", "check_every",
                                           "seed", "init_radius")})
    return out
