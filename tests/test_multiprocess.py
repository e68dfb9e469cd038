"""The multi-GPU bench path without GPUs: two gloo ranks on the CPU. Pairs are independent,
so every rank solves its own seeded batch (weak scaling, no data-path collective); the only
exchange is the max over ranks of the timed region."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench._ARGS = type("A", (), {"workload": "molecule"})()
    w = bench.workload(rank, 30)
    # a stand-in for each rank's timed region: the slowest rank must win
    t = bench.max_over_ranks(10.0 + rank)
    ws, r, _ = bench.dist_env()
    np.save(os.path.join(out_dir, f"r{rank}.npy"),
            np.array([t, ws, r, w.n_pairs, sum(g.n for g in w.graphs)], dtype=np.float64))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = 29500 + (os.getpid() % 2000)
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    assert r0[0] == r1[0] == 11.0            # both ranks see the slowest rank's time
    assert (r0[1], r1[1]) == (2, 2) and (r0[2], r1[2]) == (0, 1)
    assert r0[3] == r1[3] == 30
    assert r0[4] != r1[4]                    # each rank has its own seeded batch


def test_rank_batches_are_deterministic():
    sys.path.insert(0, ROOT)
    import bench
    bench._ARGS = type("A", (), {"workload": "molecule"})()
    a, b = bench.workload(1, 12), bench.workload(1, 12)
    assert all(x.n == y.n and np.array_equal(x.edges, y.edges) for x, y in zip(a.graphs, b.graphs))
