"""The persisted launch shapes (hj_shapes_save / hj_shapes_load): a tuned
problem's shapes written to a text cache come back on a fresh handle in the
same process, lines for another GPU, family or dimension are kept but not
applied, a second save replaces its own keys instead of duplicating them, and
a line naming a shape the build lacks is skipped."""
import numpy as np
import pytest

from paper_1803_01215_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_shapes_round_trip_through_the_cache(tmp_path):
    from paper_1803_01215_gb300 import binding
    w = W.quadcopter(B=64, seed=91, N=64)
    prob = binding.Problem.from_workload(w)
    binding.set_launch_shape(prob, "fp32", 64, 2, 1)
    binding.set_launch_shape(prob, "fp32", 16, 0, 1)        # half a warp
    binding.set_launch_shape(prob, "fp64", 64, 2, 1)
    path = tmp_path / "shapes.txt"
    path.write_text("Some Other GPU|1|12|0|64|1|2\nnot a line\n")
    binding.save_shapes(prob, path)
    binding.save_shapes(prob, path)                          # the same keys are replaced
    lines = [l for l in path.read_text().splitlines() if l]
    assert "Some Other GPU|1|12|0|64|1|2" in lines and "not a line" in lines
    assert len(lines) == 2 + 3
    fresh = binding.Problem.from_workload(w)
    n = binding.load_shapes(fresh, path)
    assert n == 3
    assert binding.get_launch_shape(fresh, "fp32", 64) == (2, 1)
    assert binding.get_launch_shape(fresh, "fp32", 16) == (0, 1)
    assert binding.get_launch_shape(fresh, "fp64", 64) == (2, 1)
    # the solve with the loaded shape gives the tuned problem's result
    xq = torch.as_tensor(w["xq"], device="cuda")
    t = torch.as_tensor(w["t"], device="cuda")
    opts = binding.make_opts(sigma=w["sigma"], tau=w["tau"], seed=w["seed"])
    a = binding.solve_batch(prob, xq, t, 64, opts)
    b = binding.solve_batch(fresh, xq, t, 64, opts)
    assert torch.equal(a["V"], b["V"]) and torch.equal(a["iters"], b["iters"])


def test_cache_lines_of_other_problems_are_not_applied(tmp_path):
    from paper_1803_01215_gb300 import binding
    wq = W.quadcopter(B=8, seed=92, N=32)
    pq = binding.Problem.from_workload(wq)
    binding.set_launch_shape(pq, "fp32", 32, 1, 1)
    path = tmp_path / "shapes.txt"
    binding.save_shapes(pq, path)
    wt = W.tanh_drift(4, B=8, seed=93)                        # another family and d
    pt = binding.Problem.from_workload(wt)
    assert binding.load_shapes(pt, path) == 0
    name = path.read_text().split("|")[0]
    # a line for this GPU and problem with a shape the build does not have: skipped
    path.write_text(f"{name}|1|12|0|32|3|1\n{name}|1|12|0|40|1|2\n")
    fresh = binding.Problem.from_workload(wq)
    assert binding.load_shapes(fresh, path) == 1
    assert binding.get_launch_shape(fresh, "fp32", 40) == (1, 2)
    assert binding.load_shapes(fresh, tmp_path / "missing.txt") == 0
