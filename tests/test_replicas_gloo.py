"""The multi-GPU path is replicas (each rank solves its own system, no
data-path collective); what it adds is host logic: the job's time is the
slowest rank's and its bytes are every rank's.  Two gloo ranks on the CPU
check that aggregation, the function bench.py applies to its timed region."""
import importlib.util
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _rank(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        ms = [100.0, 150.0, 120.0][rank]
        nbytes = [1e9, 2e9, 3e9][rank]
        b.barrier(dist)
        ms_max, value = b.aggregate(dist, ms, nbytes, "cpu")
        out.put((rank, ms_max, value))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_replica_aggregation(world):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = [out.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ms_expect = max([100.0, 150.0, 120.0][:world])
    bytes_expect = sum([1e9, 2e9, 3e9][:world])
    for _, ms_max, value in res:
        assert ms_max == ms_expect
        assert abs(value - bytes_expect / (ms_expect / 1e3) / 1e9) < 1e-9


def test_single_rank_is_identity():
    b = _bench()
    ms_max, value = b.aggregate(None, 200.0, 4e9, "cpu")
    assert ms_max == 200.0 and abs(value - 20.0) < 1e-12
