"""The multi-GPU path of bench.py is N independent replicas (the path shards
with no data-path collective); its only collectives are the barrier and the
max / sum of the timings. These run here as two gloo ranks on the CPU."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    b = _bench()
    assert b.dist_env() == (world, rank, rank)
    b.barrier(world)
    # rank r: 10 + r ms for (r + 1) GFLOP
    max_ms, flop, value = b.aggregate(10.0 + rank, (rank + 1) * 1e9, world)
    # the reference arm prints on rank 0 only; other ranks return at once without work
    b.run_reference(None, world, rank) if rank != 0 else None
    out.put((rank, max_ms, flop, value))
    dist.destroy_process_group()


def test_two_rank_aggregation_over_gloo():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, max_ms, flop, value in res:
        assert max_ms == 11.0                          # the slowest rank's time
        assert flop == 3e9                             # all ranks' work
        assert value == pytest.approx(3e9 / 11e-3 / 1e9)


def test_single_rank_aggregation_is_local():
    b = _bench()
    assert b.aggregate(20.0, 4e9, 1) == (20.0, 4e9, pytest.approx(200.0))
