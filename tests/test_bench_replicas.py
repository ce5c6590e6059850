"""The bench's multi-GPU path runs independent replicas: a barrier before
and after the timed region, the slowest rank's time, and the whole job's
bytes over that time.  These host-side steps run here on two gloo ranks on
the CPU (the kernels themselves are covered by the GPU tests)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench._barrier(world)
        m = bench._max_over_ranks(times[rank], world, device="cpu")
        bench._barrier(world)
        out.put((rank, m, bench._job_gbs(1e9, world, m)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [3.0, 5.0]  # ms per rank
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, m, gbs in got:
        assert m == 5.0  # both ranks see the maximum
        assert gbs == pytest.approx(2 * 1e9 / 5e-3 / 1e9)  # both ranks' bytes over the slowest time


def test_job_rate_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._job_gbs(8e9, 1, 1000.0) == pytest.approx(8.0)
    assert bench._max_over_ranks(7.5, 1) == 7.5
