"""The multi-process side of bench.py on CPU: two gloo ranks (one process
per GPU on a GB300 node, NCCL there) combine a timed region into the
whole-job figure -- the slowest rank's time and the units of all ranks --
and split one shell batch between them: contiguous mesh ranges balanced by
vertex count, no data-path exchange, the per-mesh results gathered after
the timed region.  Not measured on more than one GPU."""
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


def test_partition_covers_every_mesh_once_balanced():
    import bench

    _, mesh = bench.workload(0)
    for world in (1, 2, 3, 4, 8):
        ranges = bench.partition_meshes(mesh.v_off, world)
        assert len(ranges) == world and ranges[0][0] == 0 and ranges[-1][1] == mesh.n_mesh
        assert all(a < b for a, b in ranges) and all(ranges[r][1] == ranges[r + 1][0] for r in range(world - 1))
    ranges = bench.partition_meshes(mesh.v_off, 2)
    nv = [int(mesh.v_off[b] - mesh.v_off[a]) for a, b in ranges]
    assert sum(nv) == mesh.nV
    assert max(abs(v - mesh.nV / 2) for v in nv) <= 0.05 * mesh.nV / 2


def test_partition_degenerate_sizes():
    import bench

    v_off = np.array([0, 10, 20, 30])
    assert bench.partition_meshes(v_off, 1) == [(0, 3)]
    r = bench.partition_meshes(v_off, 3)
    assert r == [(0, 1), (1, 2), (2, 3)]
    r = bench.partition_meshes(np.array([0, 5, 100]), 2)     # one big mesh: still one mesh per rank
    assert r == [(0, 1), (1, 2)]


def _slice_energies(mesh):
    """Per-mesh energy and gradient norm of a batch by the oracle, mesh by mesh."""
    import oracle

    import bench

    out = []
    for k in range(mesh.n_mesh):
        v0, v1, f0, f1 = mesh.v_off[k], mesh.v_off[k + 1], mesh.f_off[k], mesh.f_off[k + 1]
        P = oracle.Problem(mesh.rest[v0:v1], mesh.faces[f0:f1] - v0, oracle.SHELL, 3, params=bench.SHELL_PARAMS)
        r = P.assemble(mesh.x[v0:v1].astype(np.float32).astype(np.float64), hessian=False)
        out.append((r["energy"], np.linalg.norm(r["grad"])))
    return np.array(out)


def _gather_main(rank, world, port, n_mesh, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        _, full = bench.workload(0, n_mesh)
        ranges = bench.partition_meshes(full.v_off, world)
        mine = bench.mesh_slice(full, *ranges[rank])
        out[rank] = bench.gather_per_mesh(dist, _slice_energies(mine), ranges)
    finally:
        dist.destroy_process_group()


def test_partitioned_batch_gathers_single_process_result_gloo_world2():
    import bench

    n_mesh = 5
    _, full = bench.workload(0, n_mesh)
    ref = _slice_energies(full)
    world = 2
    with mp.Manager() as man:
        out = man.dict()
        mp.start_processes(_gather_main, args=(world, _free_port(), n_mesh, out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    for r in range(world):
        assert res[r].shape == ref.shape
        assert np.array_equal(res[r], ref)      # same meshes, same order, bit-identical per-mesh results
