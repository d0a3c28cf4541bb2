"""The roofline numerators of bench.py are the oracle's own step arithmetic:
an op-counting run of one iteration of Algorithm 1 per node (oracle/opcount.py)
must give exactly the flop counts bench.py divides by kernel time.  The
counter itself is checked on expressions whose counts are known by hand."""
import numpy as np

import bench
from oracle import opcount
from oracle.opcount import Flop
from paper_1803_01215_gb300 import workloads as W


def test_counter_on_known_expressions():
    Flop.reset()
    a = np.array([Flop(v) for v in (1.0, 2.0, 3.0)], dtype=object)
    b = np.array([Flop(v) for v in (4.0, 5.0, 6.0)], dtype=object)
    s = np.sum(a * b)                     # 3 mul, 2 add
    assert s.v == 32.0
    assert Flop.counts["mul"] == 3 and Flop.counts["add"] == 2
    Flop.reset()
    r = (a[0] + 0.0) * 1.0 - 0 + a[1] / 1.0     # constants 0 and 1 are free
    assert r.v == 3.0 and Flop.counts["add"] == 1 and Flop.counts["mul"] == 0
    Flop.reset()
    x = opcount._solve_counted(np.array([[[Flop(2.0), 0.0], [0.0, Flop(4.0)]]], dtype=object),
                               np.array([[[Flop(2.0)], [Flop(8.0)]]], dtype=object))
    assert [x[0, 0, 0].v, x[0, 1, 0].v] == [1.0, 2.0]
    assert Flop.counts["div"] == 2 and Flop.counts["mul"] == 0   # a diagonal system: 2 divisions


def test_bench_flop_constants_equal_the_oracle_step_count():
    qc = opcount.node_step_counts(W.quadcopter(B=1))
    assert qc["flops"] == bench.QC_FLOPS_PER_NODE_ITER
    assert qc["sin"] == 3 and qc["cos"] == 3
    for d in (32, 64, 100):
        c = opcount.node_step_counts(W.tanh_drift(d, B=1))
        assert c["flops"] == bench.tanh_flops_per_node_iter(d) and c["tanh"] == d
    for d in (10, 100, 1000):
        c = opcount.node_step_counts(W.eikonal(d=d, sign=-1, t=0.2, B=1))
        assert c["flops"] == bench.eikonal_flops_per_node_iter(d)


def test_counted_step_computes_the_oracle_update():
    """The counted run is the oracle's arithmetic: its result equals a float run."""
    from oracle.families import make_family
    w = W.quadcopter(B=1)
    fam = make_family(w)
    r = np.random.default_rng(0)
    x, v = r.standard_normal((1, 12)), r.standard_normal((1, 12))
    lam = np.array([1.4 / 64])
    ref = fam.prox_p(x, v, lam)
    with opcount._counting_patches():
        got = fam.prox_p(np.array([[Flop(t) for t in x[0]]], dtype=object),
                         np.array([[Flop(t) for t in v[0]]], dtype=object), lam)
    np.testing.assert_allclose([g.v for g in got[0]], ref[0], rtol=1e-12, atol=1e-13)
