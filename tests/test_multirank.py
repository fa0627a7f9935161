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
