"""The multi-GPU sort of one array (``paper_2603_08929_gb300.distributed``) on
CPU ranks: the plan, the digit bookkeeping and the all-to-all-v exchange run
as written, over gloo with 2 and 4 processes; the device steps (digit
counts, partition, local sort) are stood in for by the oracle: a key's digit
is the place of its top-bits pattern in the oracle's order of all such
patterns, which is what the library's encoded top bits are.  The ranks'
outputs, concatenated, must equal the oracle's sort of all shards."""
import os
import socket
import sys

import numpy as np
import pytest

import oracle as O
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


# --- the plan ----------------------------------------------------------------

def _brute_plan_ok(counts, world, b):
    prefix = np.concatenate(([0], np.cumsum(counts)))
    total = prefix[-1]
    assert b[0] == 0 and b[-1] == counts.size and np.all(np.diff(b) >= 0)
    for r in range(1, world):
        goal = total * r / world
        # best boundary not below the previous one
        cands = np.arange(b[r - 1], counts.size + 1)
        best = np.min(np.abs(prefix[cands] - goal))
        assert abs(prefix[b[r]] - goal) == best, (r, b, prefix[b[r]], goal)
    loads = prefix[b[1:]] - prefix[b[:-1]]
    assert loads.max() <= total / world + 2 * counts.max() + 1e-9


def test_plan_is_the_closest_split():
    from paper_2603_08929_gb300.distributed import plan_digit_ranges, send_counts
    rng = np.random.default_rng(0)
    for trial in range(300):
        d = int(rng.integers(1, 300))
        world = int(rng.integers(1, 9))
        kind = trial % 3
        if kind == 0:
            counts = rng.integers(0, 50, d)
        elif kind == 1:
            counts = np.zeros(d, dtype=np.int64)
            counts[rng.integers(0, d, 3)] = rng.integers(1, 10000, 3)  # a few heavy digits
        else:
            counts = (rng.pareto(1.2, d) * 10).astype(np.int64)
        b = plan_digit_ranges(counts, world)
        _brute_plan_ok(counts, world, b)
        # every key is sent exactly once
        local = rng.integers(0, 5, d)
        s = send_counts(local, b)
        assert s.sum() == local.sum() and np.all(s >= 0)


# --- the scheme on gloo ranks --------------------------------------------------

def oracle_digits(x, descending, bits, fmt=None):
    """Digit of each key: the place of its top `bits` bits among all 2^bits
    patterns as the oracle orders them (each pattern's representative, its
    low bits zero, lies inside its group of the sorted output)."""
    fmt = fmt or O.FORMATS[x.dtype]
    ut = {1: np.uint8, 2: np.uint16, 4: np.uint32, 8: np.uint64}[x.dtype.itemsize]
    reps = np.arange(1 << bits, dtype=np.uint64) << np.uint64(fmt.w - bits)
    O.bsort_words(reps, fmt, descending)
    place = np.empty(1 << bits, dtype=np.int64)
    place[(reps >> np.uint64(fmt.w - bits)).astype(np.int64)] = np.arange(1 << bits)
    top = (x.view(ut).astype(np.uint64) >> np.uint64(fmt.w - bits)).astype(np.int64)
    return place[top]


class OracleOps:
    def digit_counts(self, keys, descending, bits):
        return np.bincount(oracle_digits(keys.numpy(), descending, bits), minlength=1 << bits)

    def partition(self, keys, descending, bits):
        import torch
        x = keys.numpy()
        order = np.argsort(oracle_digits(x, descending, bits), kind="stable")
        keys.copy_(torch.from_numpy(x[order]))

    def sort(self, keys, descending):
        import torch
        if keys.numel():
            keys.copy_(torch.from_numpy(O.bsort(keys.numpy(), descending=descending)))


def shard(case, rank, world):
    name, dtype, dist, n, desc, bits = case
    if name == "empty_rank" and rank == 1:
        return np.zeros(0, dtype=dtype)
    if dist == "heavy":
        x = W.make("uniform", dtype, n, seed=100 + rank)
        x[: int(0.7 * n)] = x[0] if rank == 0 else W.make("uniform", dtype, 1, seed=100)[0]
        return x
    return W.make(dist, dtype, n + 17 * rank, seed=100 + rank)


CASES = [
    ("uniform", "int32", "uniform", 20000, False, 8),
    ("zipf", "float32", "zipf", 30000, True, 12),
    ("distinct8", "int64", "distinct8", 25000, False, 6),
    ("heavy", "int32", "heavy", 20000, False, 12),
    ("float_edge", "float64", "float_edge", 20000, True, 12),
    ("empty_rank", "int16", "uniform", 20000, False, 10),
    ("bytes", "uint8", "uniform", 30000, True, 3),
]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, case, q):
    sys.path[:0] = [ROOT, os.path.join(ROOT, "tests")]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from paper_2603_08929_gb300 import distributed as D
    dist.init_process_group("gloo", rank=rank, world_size=world)
    x = shard(case, rank, world)
    out, start = D.sort_distributed(torch.from_numpy(x.copy()), descending=case[4], bits=case[5], ops=OracleOps())
    dist.destroy_process_group()
    q.put((rank, start, out.numpy()))


@pytest.mark.parametrize("world", [2, 4])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_gloo_ranks_sort_one_array(case, world):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, case, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=240) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shards = [shard(case, r, world) for r in range(world)]
    allx = np.concatenate(shards)
    want = O.bsort(allx, descending=case[4])
    got = np.concatenate([r[2] for r in res])
    assert got.dtype == want.dtype and np.array_equal(got.view(np.uint8), want.view(np.uint8))
    sizes = [r[2].size for r in res]
    assert [r[1] for r in res] == list(np.concatenate(([0], np.cumsum(sizes)))[:-1])
    digits = np.bincount(oracle_digits(allx, case[4], case[5]), minlength=1 << case[5])
    assert max(sizes) <= allx.size / world + 2 * digits.max()


# --- batched form: segments spread over gloo ranks -------------------------------

class OracleSegmentOps:
    def sort_segments(self, keys, offsets, descending):
        import torch
        x = keys.numpy()
        for a, b in zip(offsets[:-1], offsets[1:]):
            if b - a > 1:
                x[a:b] = O.bsort(x[a:b].copy(), descending=descending)
        keys.copy_(torch.from_numpy(x))


def _batch(world_seed):
    sizes = W.segment_sizes(world_seed, 300, 14)
    sizes[::37] = 0
    x = W.make("float_edge", "float32", int(sizes.sum()), seed=world_seed)
    return x, np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def _seg_rank(rank, world, port, q):
    sys.path[:0] = [ROOT, os.path.join(ROOT, "tests")]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from paper_2603_08929_gb300 import distributed as D
    dist.init_process_group("gloo", rank=rank, world_size=world)
    x, off = _batch(5)
    t = torch.from_numpy(x.copy())
    a, b = D.sort_segments_distributed(t, off, descending=True, ops=OracleSegmentOps())
    dist.destroy_process_group()
    q.put((rank, a, b, t.numpy()[off[a]:off[b]].copy()))


def test_plan_segments_balances_keys():
    from paper_2603_08929_gb300.distributed import plan_segments
    rng = np.random.default_rng(3)
    for trial in range(200):
        sizes = rng.integers(0, 1000, int(rng.integers(1, 200)))
        world = int(rng.integers(1, 9))
        s = plan_segments(sizes, world)
        _brute_plan_ok(sizes, world, s)


@pytest.mark.parametrize("world", [2, 4])
def test_gloo_ranks_sort_a_batch(world):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_seg_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=240) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    x, off = _batch(5)
    # the runs tile the batch in rank order
    assert res[0][1] == 0 and res[-1][2] == off.size - 1
    assert all(res[i][2] == res[i + 1][1] for i in range(world - 1))
    got = np.concatenate([r[3] for r in res])
    want = x.copy()
    for a, b in zip(off[:-1], off[1:]):
        if b - a > 1:
            want[a:b] = O.bsort(x[a:b].copy(), descending=True)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    sizes = np.diff(off)
    assert max(off[r[2]] - off[r[1]] for r in res) <= sizes.sum() / world + 2 * sizes.max()


@pytest.mark.parametrize("as_tensor", [False, True])
def test_library_segment_ops_hands_the_library_an_int64_tensor(monkeypatch, as_tensor):
    """The device step of the batched form receives the run's boundaries as
    numpy (from the plan) or as a tensor; the segmented sort it calls wants
    an int64 tensor on the keys' device.  The library call is replaced here
    by a recorder (no GPU)."""
    import torch
    import paper_2603_08929_gb300 as pkg
    from paper_2603_08929_gb300 import distributed as D
    seen = []
    monkeypatch.setattr(pkg, "bsort_keys_segmented",
                        lambda keys, off, descending=False: seen.append((keys, off, descending)))
    keys = torch.arange(10, dtype=torch.int32)
    off = np.array([0, 3, 3, 10], dtype=np.int64)
    D.LibrarySegmentOps().sort_segments(keys, torch.from_numpy(off) if as_tensor else off, True)
    (k, o, desc), = seen
    assert k is keys and desc is True
    assert isinstance(o, torch.Tensor) and o.dtype == torch.int64 and o.device == keys.device
    assert o.tolist() == off.tolist()
    seen.clear()
    D.LibrarySegmentOps().sort_segments(keys[:1], np.array([0, 1]), False)  # one key: nothing to sort
    assert not seen
