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


def test_replica_shards_cover_and_balance():
    # the batched workload's 256 replicas shared out by cost over 2, 4 and 8 ranks
    import sys
    sys.path.insert(0, ROOT)
    import bench
    from paper_1703_02484_gb300 import workloads
    ns, _, laws = workloads.replica_table(256)
    cost = [float(n) * n if law == 1 else 3000.0 * n for n, law in zip(ns, laws)]
    for world in (1, 2, 4, 8):
        parts = bench.shard_replicas(list(ns), list(laws), world)
        assert len(parts) == world
        flat = sorted(r for p in parts for r in p)
        assert flat == list(range(256))                 # every replica exactly once
        loads = [sum(cost[r] for r in p) for p in parts]
        # greedy largest-first: no rank exceeds the mean by more than the largest single cost
        assert max(loads) <= sum(cost) / world + max(cost) + 1e-6
        if world <= 4:
            assert max(loads) <= 1.05 * sum(cost) / world


class _FakeShard:
    """Stands in for a force-sharded System on the CPU: rank r's partial force
    is the pair sum over the disks j of its share (the oracle's sum), and
    step_end keeps the forces it was given."""

    def __init__(self, F, xy, sp, alpha, rank, world):
        from oracle import forces
        n = len(xy)
        lo, hi = rank * n // world, (rank + 1) * n // world
        d = xy[:, None, :] - xy[None, lo:hi, :]
        r2 = np.einsum("ijk,ijk->ij", d, d)
        A = forces.species_table(alpha)
        with np.errstate(divide="ignore", invalid="ignore"):
            coef = A[sp][:, sp[lo:hi]] / (r2 * np.sqrt(r2))
        coef[~np.isfinite(coef)] = 0.0
        self.partial = np.einsum("ij,ijk->ik", coef, d).reshape(-1)
        self.F = F
        self.seen = None

    def step_begin(self, ptr):
        assert ptr == self.F.data_ptr()
        self.F.copy_(torch.from_numpy(self.partial))

    def step_end(self, ptr):
        assert ptr == self.F.data_ptr()
        self.seen = self.F.clone().numpy()
        return {"steps_done": 1}


def _shard_main(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    rng = np.random.default_rng(5)
    xy = rng.uniform(0, 50, size=(300, 2))
    sp = rng.integers(0, 2, 300).astype(np.int64)
    alpha = (0.05, 0.2, -0.1, 0.05)
    F = torch.zeros(600, dtype=torch.float64)
    fake = _FakeShard(F, xy, sp, alpha, rank, world)
    st = bench.sharded_step(fake, F, world)
    assert st["steps_done"] == 1
    np.save(os.path.join(out_dir, "F%d.npy" % rank), fake.seen)
    dist.destroy_process_group()


def test_force_shards_summed_over_gloo_ranks(tmp_path):
    # each rank's partial force (pairs with its share of the disks) summed by the
    # all-reduce: every rank ends with the whole force, the same bits on both
    port = _free_port()
    mp.start_processes(_shard_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    F0, F1 = np.load(tmp_path / "F0.npy"), np.load(tmp_path / "F1.npy")
    assert np.array_equal(F0, F1)
    import sys
    sys.path.insert(0, ROOT)
    from oracle import forces
    rng = np.random.default_rng(5)
    xy = rng.uniform(0, 50, size=(300, 2))
    sp = rng.integers(0, 2, 300).astype(np.int64)
    ref = forces.long_range_numpy(xy, sp, (0.05, 0.2, -0.1, 0.05)).reshape(-1)
    assert np.allclose(F0, ref, rtol=1e-12, atol=1e-15)
