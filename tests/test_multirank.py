"""The N > 1 path of the benchmark on CPU: two gloo ranks aggregate their step times (max) and
converged counts (sum), and each rank draws its own instance set (weak scaling, no collective
on the data path)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, c = bench.aggregate_ranks(100.0 + 50.0 * rank, 300.0 + rank, world, "cpu")
    out[rank] = (t, c)
    dist.destroy_process_group()


def test_two_ranks_aggregate_and_draw_disjoint_sets():
    mp = torch.multiprocessing.get_context("spawn")
    with mp.Manager() as man:
        out = man.dict()
        port = _free_port()
        procs = [mp.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1] == (150.0, 601.0)
    from synth import batch_grids
    a, b = batch_grids(3, 2, part=0), batch_grids(3, 2, part=1)
    assert not np.allclose(a[0].pd, b[0].pd)
    assert a[3].nb != b[3].nb or not np.allclose(a[3].pd, b[3].pd)


def _split_grids():
    from synth import ring_grid, scale_loads, config_grid
    base = config_grid("ring30")
    return ([scale_loads(base, 50 + k) for k in range(4)] +
            [ring_grid(12, 3, 3, seed=5), ring_grid(20, 5, 4, seed=7)])


def _solve_share(grids, mine):
    """Per-rank solver stand-in on CPU: the oracle IPM on this rank's instances (on the GPU the
    rank runs the batched IPM over the same share)."""
    from oracle.opf import OPFModel
    from oracle import ipm as oipm
    res = [oipm.solve(OPFModel(grids[i]), oipm.Options(kkt="hykkt")) for i in mine]
    return dict(status=[1 if r.status == "converged" else 0 for r in res],
                obj=[r.obj for r in res], iters=[r.iters for r in res])


def _split_worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2405_14236_gb300.shard import partition_by_cost, gather_results
    grids = _split_grids()
    parts = partition_by_cost([g.n for g in grids], world)
    full = gather_results(_solve_share(grids, parts[rank]), parts[rank], len(grids), world)
    out[rank] = (parts, {k: v.tolist() for k, v in full.items()})
    dist.destroy_process_group()


def test_partition_by_cost_is_balanced_and_complete():
    from paper_2405_14236_gb300.shard import partition_by_cost
    rng = np.random.default_rng(3)
    costs = rng.integers(1, 1000, 57)
    for world in (1, 2, 3, 8):
        parts = partition_by_cost(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [costs[p].sum() for p in parts]
        assert max(loads) - min(loads) <= costs.max()


def test_two_ranks_split_one_batch_and_gather():
    """One fixed batch split across two gloo ranks by size, each rank solving its share, the
    results gathered on every rank: identical to a one-rank solve of the whole batch."""
    mp = torch.multiprocessing.get_context("spawn")
    with mp.Manager() as man:
        out = man.dict()
        port = _free_port()
        procs = [mp.Process(target=_split_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
            assert p.exitcode == 0
        res = dict(out)
    parts0, full0 = res[0]
    parts1, full1 = res[1]
    assert parts0 == parts1 and full0 == full1
    assert sorted(parts0[0] + parts0[1]) == list(range(6)) and parts0[0] and parts0[1]
    grids = _split_grids()
    one = _solve_share(grids, list(range(len(grids))))
    assert full0["status"] == one["status"] and all(s == 1 for s in one["status"])
    np.testing.assert_array_equal(full0["obj"], one["obj"])
    np.testing.assert_array_equal(full0["iters"], one["iters"])
