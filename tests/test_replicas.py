"""The N > 1 path of bench.py on CPU: two gloo ranks, each timing its own
replica; both must see the max step time and the whole-job throughput."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    ms, value = bench.whole_job(10.0 + 5.0 * rank, 1 << 20, w, "cpu")
    dist.destroy_process_group()
    q.put((r, w, local, ms, value))


def test_two_gloo_ranks_take_the_max_time():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[:3] for o in out] == [(0, 2, 0), (1, 2, 1)]
    for _, _, _, ms, value in out:
        assert ms == 15.0  # the slower rank's step time
        assert value == pytest.approx(2 * (1 << 20) / 15e-3 / 1e9)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.whole_job(4.0, 1 << 28, 1, "cpu")
    assert ms == 4.0 and value == pytest.approx((1 << 28) / 4e-3 / 1e9)
