"""Multi-rank path on CPU: world_size-2 gloo processes shard independent solves with no
exchange during the solve and gather the fields on rank 0 (no GPU)."""
import os
import socket

import numpy as np
import pytest

from paper_1305_1293_gb300 import meshgen as mg
from paper_1305_1293_gb300.shard import shard_instances, solve_sharded


def test_shard_balanced_and_complete():
    w = [100, 90, 80, 10, 10, 5, 5, 1]
    s = shard_instances(w, 2)
    assert sorted(i for part in s for i in part) == list(range(len(w)))
    loads = [sum(w[i] for i in part) for part in s]
    assert max(loads) - min(loads) <= max(w)
    assert shard_instances(w, 2) == s                       # deterministic
    assert shard_instances([1, 1, 1], 5)[3] == []            # more ranks than instances


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    meshes, srcs = mg.workload("batch", "small")

    def solve(indices):
        return [oracle.geodesic(meshes[i].vertices, meshes[i].faces, int(srcs[i][0]))[0] for i in indices]

    res = solve_sharded(len(meshes), [m.nf for m in meshes], solve, rank, world)
    if rank == 0:
        np.savez(out_path, *res)
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_two_ranks_gather_matches_single(tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "res.npz")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    import oracle
    meshes, srcs = mg.workload("batch", "small")
    for i, m in enumerate(meshes):
        ref = oracle.geodesic(m.vertices, m.faces, int(srcs[i][0]))[0]
        assert np.array_equal(got[f"arr_{i}"], ref)
