"""The N > 1 path of bench.py is replicas only (no data-path collective):
each rank runs the whole workload on its own GPU, and the job time is the
slowest rank's. This checks that aggregation with two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    t_local = 2.0 + rank          # rank 1 is the slower replica
    value, t = bench.replica_value(t_local, units_per_step=1000, steps=5, dist_mod=dist)
    out.put((rank, value, t))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, value, t in res:
        assert t == 3.0                              # max over ranks
        assert value == ws * 1000 * 5 / 3.0          # units of all ranks / slowest time


def test_replica_value_single_process():
    import bench
    v, t = bench.replica_value(0.5, 200, 4)
    assert (v, t) == (1600.0, 0.5)
