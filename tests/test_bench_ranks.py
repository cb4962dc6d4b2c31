"""The multi-process side of bench.py on CPU: two gloo ranks (one process
per GPU on a GB300 node, NCCL there) combine a timed region into the
whole-job figure -- the slowest rank's time and the units of all ranks --
and each rank draws its own seeded replica of the batch (weak scaling, no
data-path exchange)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        sec, units = bench.combine_ranks(dist, 10.0 + 3.0 * rank, 100 * (rank + 1), device="cpu")
        out[rank] = (sec, units)
    finally:
        dist.destroy_process_group()


def test_combine_ranks_gloo_world2():
    world = 2
    with mp.Manager() as man:
        out = man.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    assert res[0] == res[1] == (13.0, 300)   # max time over ranks, sum of units


def test_combine_ranks_single_process():
    import bench

    assert bench.combine_ranks(None, 2.5, 7) == (2.5, 7)


def test_replicas_differ_per_rank_with_equal_shape():
    import bench

    _, m0 = bench.workload(0, n_mesh=3)
    _, m1 = bench.workload(1, n_mesh=3)
    assert m0.nV == m1.nV and m0.nT == m1.nT
    assert np.array_equal(m0.faces, m1.faces)
    assert not np.array_equal(m0.x, m1.x)    # own seeded perturbation and rotation per rank
