"""bench.py at N > 1: independent replicas, one per rank, combined with the
slowest rank's time and the sum of the ranks' work (weak scaling).  Run here
as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import importlib.util
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    # rank r: 1 + r seconds, 1e9 (r + 1) pairs, e2e 10 (r + 1)
    out = bench.combine_ranks(1.0 + rank, 1e9 * (rank + 1), 10.0 * (rank + 1), "cpu")
    q.put((rank, out))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replicas_combine_max_time_sum_work(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        total_s, pairs, e2e = got[r]
        assert total_s == float(world)                          # the slowest rank
        assert pairs == 1e9 * world * (world + 1) / 2            # all ranks' pairs
        assert e2e == 10.0 * world * (world + 1) / 2
    # the reported whole-job rate: all pairs over the slowest rank's time
    assert got[0][1] / got[0][0] == pytest.approx(1.5e9)
