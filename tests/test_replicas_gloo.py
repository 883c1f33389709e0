"""The benchmark's multi-GPU path is replicas (images are independent; no
data-path collective): the only exchange is the max over ranks of the step
time.  Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [2.0, 3.5][rank]
        ms, units_s = bench.replica_throughput(world, torch.device("cpu"), local_ms, 1000)
        e2e = bench.max_over_ranks(world, torch.device("cpu"), [7.0, 5.0][rank])
        q.put((rank, ms, units_s, e2e))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units_s, e2e in out:
        assert ms == 3.5                      # max over ranks
        assert units_s == pytest.approx(2 * 1000 / 3.5e-3)  # whole job: both ranks' units
        assert e2e == 7.0


def test_single_rank_needs_no_process_group():
    import bench

    ms, units_s = bench.replica_throughput(1, torch.device("cpu"), 4.0, 500)
    assert ms == 4.0 and units_s == pytest.approx(500 / 4e-3)
