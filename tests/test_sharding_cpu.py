"""The multi-rank path on CPU: two gloo ranks shard a batch by global point
index, solve their slices with the oracle, and reduce timings and counts the
way bench.py does.  No GPU."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1803_01215_gb300 import sharding
from paper_1803_01215_gb300 import workloads as W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import lax_pdhg as O
    w = W.tanh_drift(4, B=10, seed=9, N=8)
    lo, hi = sharding.strong_slice(rank, world, len(w["xq"]))
    res = O.solve(W.subset(w, np.arange(lo, hi)), max_iter=200)
    np.save(os.path.join(outdir, f"V{rank}.npy"), res["V"])
    times, counts = sharding.reduce_step_stats([10.0 + rank, 5.0 * (rank + 1)],
                                               [hi - lo, int(res["iters"].sum())])
    np.save(os.path.join(outdir, f"stats{rank}.npy"), np.array(times + counts))
    dist.barrier()
    dist.destroy_process_group()


def test_slices_cover_and_are_disjoint():
    for B, world in [(10, 2), (4096, 4), (7, 3), (3, 8)]:
        sl = [sharding.strong_slice(r, world, B) for r in range(world)]
        assert sl[0][0] == 0 and sl[-1][1] == B
        assert all(sl[i][1] == sl[i + 1][0] for i in range(world - 1))
    assert [sharding.weak_offset(r, 4096) for r in range(3)] == [0, 4096, 8192]


def test_two_gloo_ranks_reproduce_the_unsharded_solve(tmp_path):
    from oracle import lax_pdhg as O
    world, port = 2, _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    V = np.concatenate([np.load(tmp_path / f"V{r}.npy") for r in range(world)])
    full = O.solve(W.tanh_drift(4, B=10, seed=9, N=8), max_iter=200)
    np.testing.assert_array_equal(V, full["V"])          # same global indices, same init
    s0, s1 = np.load(tmp_path / "stats0.npy"), np.load(tmp_path / "stats1.npy")
    np.testing.assert_array_equal(s0, s1)                 # every rank sees the reduction
    assert s0[0] == 11.0 and s0[1] == 10.0                # max over ranks
    assert s0[2] == 10 and s0[3] == full["iters"].sum()   # sums over ranks
