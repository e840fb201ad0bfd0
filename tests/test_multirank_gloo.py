"""The benchmark's multi-rank path on the CPU: two ranks over gloo.

The per-step path does not shard (the triangulation and the overlap loop
would need a spatial decomposition with halo flips), so N ranks advance N
independent replicas: each rank its own Philox stream, no collective on the
data path, the job's time the slowest rank's and its throughput the units of
all ranks.  These tests run that host logic with world size 2 on gloo."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import paper_1703_02484_gb300 as bd
    from oracle import noise
    from paper_1703_02484_gb300 import workloads
    ws, r, local = bench.dist_env()
    # the slowest rank's time, on every rank
    t = bench.max_over_ranks(1.5 + rank, ws, "cpu")
    # each rank's replica: same workload, its own noise stream
    cfg = workloads.CONFIGS["c5"]
    p = bench.rank_params(bd, cfg, r, ("periodic",))
    z = np.concatenate([np.ravel(v) for v in noise.normals(np.arange(4), 7, cfg.seed, int(p.replica))])
    got = [None] * world
    dist.all_gather_object(got, (r, int(p.replica), int(p.boundary), t, z.tolist()))
    # the reference arm: ranks other than 0 return at once
    class A:
        pass
    a = A()
    res = bench.run_reference(a) if r != 0 else "skipped"
    dist.destroy_process_group()
    if rank == 0:
        np.save(os.path.join(out_dir, "gathered.npy"), np.array(got, dtype=object), allow_pickle=True)
    else:
        np.save(os.path.join(out_dir, "ref%d.npy" % rank), np.array([res is None]))


def test_two_ranks_over_gloo(tmp_path):
    import sys
    sys.path.insert(0, ROOT)
    from paper_1703_02484_gb300.binding import load
    load()                        # built once here, not by both ranks at once
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    got = np.load(tmp_path / "gathered.npy", allow_pickle=True)
    ranks = [int(g[0]) for g in got]
    assert ranks == [0, 1]
    assert [int(g[1]) for g in got] == [0, 1]            # replica id = rank
    assert all(int(g[2]) == 1 for g in got)              # the workload's mode on every rank
    assert all(float(g[3]) == 2.5 for g in got)          # max over ranks
    z0, z1 = np.array(got[0][4]), np.array(got[1][4])
    assert not np.allclose(z0, z1)                       # independent noise streams
    assert bool(np.load(tmp_path / "ref1.npy")[0])       # rank 1 runs no reference work
