"""Arithmetic of one PDHG iteration per time node, counted on the oracle's code.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

`Flop` is a float that counts the additions, multiplications and divisions done
with it (and, apart, the sines, cosines and other transcendentals).  An
operation with an exact constant 0 (an addend, or a factor that makes the
result 0) or a constant factor 1 is free: the oracle's dense arrays (np.eye,
np.zeros, the 12 x 4 input matrix B) then cost only their nonzero structure.
Constants of a point (sigma, tau, delta, sigma delta) are plain floats, so the
count is per node and iteration, as the roofline of the iteration kernels
needs it.

node_step_counts(w) runs, on Flop inputs, the oracle's own Hamiltonian
functions in the order of one iteration of Algorithm 1 at an interior node j
(Section 5.3 updates, Appendix Algorithm A.1 loop):
    v     = p_j + sigma (z_j - z_{j-1})
    p_j'  = prox_{sigma delta H(x_j, .)}(v)                   (family prox_p)
    x_j'  = x_j - tau (p_j' - p_{j+1}') + tau delta grad_x H(x_j, p_j')
    z_j'  = x_j' + theta (x_j' - x_j)
The prox of the quadcopter is the oracle's linear solve, run here as Gaussian
elimination on the Flop entries, so only the entries its structure makes
nonzero are worked on.  H's state quantities at x_j (the thrust direction and
its Jacobian; tanh(A x) and its derivative; the eikonal speed and its
gradient) enter the prox and the gradient;
Algorithm A.1 evaluates H at x^k for both, so they are counted once (one
evaluation shared by both calls).
"""
import contextlib
import numbers

import numpy as np

from . import families
from .families import make_family

KINDS = ("add", "mul", "div", "sin", "cos", "exp", "tanh", "sqrt")


def _const(o):
    return isinstance(o, (numbers.Real, np.floating, np.integer)) and not isinstance(o, Flop)


class Flop:
    """A float that counts the arithmetic done with it (class-level tally)."""
    counts = dict.fromkeys(KINDS, 0)
    __slots__ = ("v",)

    def __init__(self, v):
        self.v = float(v)

    @classmethod
    def reset(cls):
        cls.counts = dict.fromkeys(KINDS, 0)

    @staticmethod
    def _val(o):
        return o.v if isinstance(o, Flop) else float(o)

    def _add(self, o, sign):
        if _const(o) and o == 0:
            return self if sign > 0 else self
        Flop.counts["add"] += 1
        return Flop(self.v + sign * Flop._val(o))

    def __add__(self, o):
        return self._add(o, 1.0)

    __radd__ = __add__

    def __sub__(self, o):
        return self._add(o, -1.0)

    def __rsub__(self, o):
        if _const(o) and o == 0:
            return -self
        Flop.counts["add"] += 1
        return Flop(float(o) - self.v)

    def __mul__(self, o):
        if _const(o):
            if o == 0:
                return 0.0
            if o == 1:
                return self
            if o == -1:
                return -self
        Flop.counts["mul"] += 1
        return Flop(self.v * Flop._val(o))

    __rmul__ = __mul__

    def __truediv__(self, o):
        if _const(o) and o == 1:
            return self
        Flop.counts["div"] += 1
        return Flop(self.v / Flop._val(o))

    def __rtruediv__(self, o):
        if _const(o) and o == 0:
            return 0.0
        Flop.counts["div"] += 1
        return Flop(float(o) / self.v)

    def __neg__(self):
        return Flop(-self.v)              # a sign flip is not a flop

    def __pos__(self):
        return self

    # comparisons (shrink_2's max and the p = 0 case) are not counted
    def __gt__(self, o):
        return self.v > Flop._val(o)

    def __ge__(self, o):
        return self.v >= Flop._val(o)

    def __lt__(self, o):
        return self.v < Flop._val(o)

    def __le__(self, o):
        return self.v <= Flop._val(o)

    def _f(self, kind, fn):
        Flop.counts[kind] += 1
        return Flop(fn(self.v))

    def sin(self):
        return self._f("sin", np.sin)

    def cos(self):
        return self._f("cos", np.cos)

    def exp(self):
        return self._f("exp", np.exp)

    def tanh(self):
        return self._f("tanh", np.tanh)

    def sqrt(self):
        return self._f("sqrt", np.sqrt)


def _solve_counted(M, b):
    """Gaussian elimination without pivoting on object arrays [..., n, n], [..., n, 1]
    (the oracle's systems are diagonally dominant: 1 + lam eps on the diagonal)."""
    M = np.array(M, dtype=object)
    b = np.array(b, dtype=object)
    n = M.shape[-1]
    for k in range(n):
        for i in range(k + 1, n):
            if _const(M[..., i, k].item()) and M[..., i, k].item() == 0:
                continue
            f = M[..., i, k] / M[..., k, k]
            for j in range(k + 1, n):
                M[..., i, j] = M[..., i, j] - f * M[..., k, j]
            b[..., i, 0] = b[..., i, 0] - f * b[..., k, 0]
    x = np.empty_like(b)
    for i in range(n - 1, -1, -1):
        acc = b[..., i, 0]
        for j in range(i + 1, n):
            acc = acc - M[..., i, j] * x[..., j, 0]
        x[..., i, 0] = acc / M[..., i, i]
    return x


@contextlib.contextmanager
def _counting_patches():
    """Route the oracle's dense solve to the counting elimination, and share one
    evaluation of H's state quantities per node (the quadcopter's thrust
    direction, tanh(A x) and its derivative for the tanh drift, the eikonal
    speed and its gradient)."""
    solve0 = np.linalg.solve
    thrust0 = families.Quadcopter.thrust_dir
    memo = {}

    def thrust(x):
        key = tuple(id(v) for v in np.ravel(x[..., 3:6]))
        if key not in memo:
            memo[key] = thrust0(x)
        return memo[key]

    act0 = families.TanhDrift._act

    def act(self, x):
        key = ("act",) + tuple(id(v) for v in np.ravel(x))
        if key not in memo:
            memo[key] = act0(self, x)
        return memo[key]

    speed0 = families.Eikonal.speed

    def speed(self, x, s=None):
        key = ("speed",) + tuple(id(v) for v in np.ravel(x))
        if key not in memo:
            memo[key] = speed0(self, x, s)
        return memo[key]

    np.linalg.solve = _solve_counted
    families.Quadcopter.thrust_dir = staticmethod(thrust)
    families.TanhDrift._act = act
    families.Eikonal.speed = speed
    try:
        yield
    finally:
        np.linalg.solve = solve0
        families.Quadcopter.thrust_dir = staticmethod(thrust0)
        families.TanhDrift._act = act0
        families.Eikonal.speed = speed0


def node_step_counts(w, sigma=1.4, tau=0.24 / 1.4, delta=1.0 / 64, theta=1.0, seed=0):
    """Operation counts of one iteration at one interior node (see the module
    docstring) for workload `w`'s family; returns dict(kind -> count) and the
    flop total add + mul + div."""
    fam = make_family(w)
    d = int(w["d"])
    r = np.random.default_rng(seed)
    mk = lambda: np.array([Flop(v) for v in r.standard_normal(d)], dtype=object)[None]  # noqa: E731
    x, p, z, zl, pn_next = mk(), mk(), mk(), mk(), mk()
    lam = np.array([sigma * delta])
    Flop.reset()
    with _counting_patches():
        v = p + sigma * (z - zl)
        pn = fam.prox_p(x, v, lam)
        xn = x - tau * (pn - pn_next) + (tau * delta) * fam.grad_x(x, pn)
        zn = xn + theta * (xn - x)
    assert zn.shape == (1, d)
    c = dict(Flop.counts)
    c["flops"] = c["add"] + c["mul"] + c["div"]
    return c
