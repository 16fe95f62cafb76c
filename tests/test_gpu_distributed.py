"""The device steps of the multi-GPU sort of one array, on the GPU through
the C ABI: the top-digit counts against the oracle's digits, and the whole
scheme (counts, all-reduce, plan, partition, exchange, local sort) with one
rank and with two ranks.  The two ranks are two processes on the one GPU of
this machine over gloo (the exchange staged through host memory); neither
launches a kernel that waits on the other."""
import os
import socket
import sys

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import assert_bit_exact, to_device
from test_distributed_model import oracle_digits

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2603_08929_gb300 import build as b
    b.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("desc", [False, True], ids=["asc", "desc"])
@pytest.mark.parametrize("dtype,dist", [("uint8", "uniform"), ("int16", "zipf"), ("float16", "float_edge"),
                                        ("int32", "uniform"), ("float32", "float_edge"), ("uint64", "zipf"),
                                        ("float64", "normal"), ("int64", "distinct8")])
def test_top_digit_counts(dtype, dist, desc):
    import paper_2603_08929_gb300 as bs
    x = W.make(dist, dtype, 100003, seed=9)
    w = x.dtype.itemsize * 8
    for bits in sorted({1, 3, min(8, w), min(12, w)}):
        for off in (0, 1, 3):  # unaligned starts: the kernel finds the aligned middle
            xs = x[off:]
            got = bs.top_digit_counts(to_device(xs), bits, descending=desc).cpu().numpy()
            want = np.bincount(oracle_digits(xs, desc, bits), minlength=1 << bits)
            assert np.array_equal(got, want), (dtype, bits, off)


def test_top_digit_counts_rejects_bad_bits():
    import paper_2603_08929_gb300 as bs
    t = to_device(np.arange(10, dtype=np.int16))
    for bits in (0, 13, 17):
        with pytest.raises(bs.BsortError):
            bs.top_digit_counts(t, bits)
    assert bs.top_digit_counts(to_device(np.zeros(0, np.int32)), 4).sum().item() == 0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


CASES = [("int32", "uniform", 1 << 20, False), ("float32", "float_edge", 700001, True),
         ("int64", "zipf", 300000, False), ("uint16", "uniform", 500000, True)]


def _shard(case, rank):
    dtype, dist, n, _ = case
    return W.make(dist, dtype, n + 1000 * rank, seed=40 + rank)


def _rank(rank, world, port, q):
    sys.path[:0] = [ROOT, os.path.join(ROOT, "tests")]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from paper_2603_08929_gb300 import distributed as D
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out = []
    for case in CASES:
        t = torch.from_numpy(_shard(case, rank)).cuda()
        mine, start = D.sort_distributed(t, descending=case[3], bits=12)
        torch.cuda.synchronize()
        out.append((start, mine.cpu().numpy()))
    dist.destroy_process_group()
    q.put((rank, out))


@pytest.mark.parametrize("world", [1, 2])
def test_sort_distributed(world):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=600) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for i, case in enumerate(CASES):
        allx = np.concatenate([_shard(case, r) for r in range(world)])
        parts = [res[r][1][i] for r in range(world)]
        assert_bit_exact(np.concatenate([p[1] for p in parts]), O.bsort(allx, descending=case[3]), str(case))
        sizes = [p[1].size for p in parts]
        assert [p[0] for p in parts] == list(np.concatenate(([0], np.cumsum(sizes)))[:-1])


def _seg_rank(rank, world, port, q):
    sys.path[:0] = [ROOT, os.path.join(ROOT, "tests")]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from paper_2603_08929_gb300 import distributed as D
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sizes = W.segment_sizes(9, 2000, 16)
    x = W.make("uniform", "int32", int(sizes.sum()), seed=9)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    t = torch.from_numpy(x).cuda()
    a, b = D.sort_segments_distributed(t, off)
    torch.cuda.synchronize()
    dist.destroy_process_group()
    q.put((rank, a, b, t.cpu().numpy()[off[a]:off[b]].copy()))


@pytest.mark.parametrize("world", [1, 2])
def test_sort_segments_distributed(world):
    """The batched form split over ranks by key count: each rank sorts its run
    of segments with the segmented sort; every segment equals the oracle's."""
    import multiprocessing as mp
    from gpu_util import oracle_segments
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_seg_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=600) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sizes = W.segment_sizes(9, 2000, 16)
    x = W.make("uniform", "int32", int(sizes.sum()), seed=9)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    assert res[0][1] == 0 and res[-1][2] == sizes.size
    assert_bit_exact(np.concatenate([r[3] for r in res]), oracle_segments(x, off, False), "segments over ranks")
