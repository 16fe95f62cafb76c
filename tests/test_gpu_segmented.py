"""Segmented sorts and captured graphs through the C ABI, against the oracle
segment by segment."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import assert_bit_exact, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2603_08929_gb300 import build as b
    b.build()
    torch.cuda.set_device(0)


def make_segments(sizes, dtype, dist="uniform", seed=0):
    n = int(np.sum(sizes))
    x = W.make(dist, dtype, n, seed=seed)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return x, off


def oracle_segments(x, off, desc):
    out = x.copy()
    for a, b in zip(off[:-1], off[1:]):
        if b - a > 1:
            out[a:b] = O.bsort(x[a:b], descending=desc)
    return out


@pytest.mark.parametrize("desc", [False, True], ids=["asc", "desc"])
@pytest.mark.parametrize("dtype", ["int32", "float32", "uint64", "float64"])
def test_segmented_mixed_sizes(dtype, desc):
    import torch
    import paper_2603_08929_gb300 as bs
    rng = np.random.default_rng(1)
    sizes = np.concatenate([[0, 1, 2, 0, 3], rng.integers(0, 40, 30), rng.integers(1000, 9000, 12),
                            [20000, 70001, 300000], W.segment_sizes(4, 60, 16)])
    rng.shuffle(sizes)
    x, off = make_segments(sizes, dtype, "float_edge" if dtype.startswith("float") else "uniform", seed=3)
    t = to_device(x)
    bs.bsort_keys_segmented(t, torch.from_numpy(off).cuda(), descending=desc)
    assert_bit_exact(t.cpu().numpy(), oracle_segments(x, off, desc), "segmented %s" % dtype)


@pytest.mark.parametrize("dist", ["zipf", "distinct8", "sorted"])
def test_segmented_skewed(dist):
    import torch
    import paper_2603_08929_gb300 as bs
    sizes = np.array([5, 100000, 17, 40000, 6000, 1, 250000, 33])
    x, off = make_segments(sizes, "int32", dist, seed=4)
    t = to_device(x)
    bs.bsort_keys_segmented(t, torch.from_numpy(off).cuda())
    assert_bit_exact(t.cpu().numpy(), oracle_segments(x, off, False), "segmented %s" % dist)


@pytest.mark.parametrize("max_log2", [17, 20], ids=["scaled-2p17", "stated-2p20"])
def test_batched_workload_at_size(max_log2):
    """The batched configuration at size: 10,000 int32 and 10,000 float32
    segments, sizes floor(2^(k*u)) log-uniform in [1, 2^k] (k = 20 as stated,
    about 1.5e9 keys in all; k = 17, about 2.2e8 keys, the stated total),
    uniform bits, ascending, generated as the benchmark generates them and
    sorted by one captured graph per dtype (the benchmark's call); every
    segment byte for byte against the oracle."""
    import torch
    import paper_2603_08929_gb300 as bs
    from gpu_util import oracle_segments
    for k, dt in enumerate(("int32", "float32")):
        sizes = W.segment_sizes(17 * k, 10000, max_log2)
        x, off = make_segments(sizes, dt, seed=k)
        t = to_device(x)
        offs = torch.from_numpy(off).cuda()
        h = bs.Handle()
        ws = torch.empty(bs.segmented_workspace_bytes(t.numel(), len(sizes), dt), dtype=torch.uint8, device="cuda")
        g = bs.Graph(h, t, ws, offsets=offs)
        g.launch()
        assert g.error() == 0
        got = t.cpu().numpy()
        g.close()
        del t, ws, offs
        torch.cuda.empty_cache()
        assert_bit_exact(got, oracle_segments(x, off, False), "batched %s, sizes in [1, 2^%d]" % (dt, max_log2))


def test_segmented_graph_replay_and_ws():
    import torch
    import paper_2603_08929_gb300 as bs
    sizes = W.segment_sizes(7, 300, 14)
    x, off = make_segments(sizes, "int32", seed=5)
    want = oracle_segments(x, off, False)
    t = to_device(x)
    offs = torch.from_numpy(off).cuda()
    h = bs.Handle()
    ws = torch.empty(bs.segmented_workspace_bytes(t.numel(), len(sizes), "int32"), dtype=torch.uint8, device="cuda")
    g = bs.Graph(h, t, ws, offsets=offs)
    for rep in range(3):  # replays on fresh contents
        t.copy_(torch.from_numpy(x).cuda())
        g.launch()
        assert g.error() == 0
        assert_bit_exact(t.cpu().numpy(), want, "graph replay %d" % rep)
    t.copy_(torch.from_numpy(x).cuda())
    bs.bsort_keys_segmented(t, offs, handle=h, workspace=ws)
    assert_bit_exact(t.cpu().numpy(), want, "segmented ws")


def test_plain_graph():
    import torch
    import paper_2603_08929_gb300 as bs
    x = W.make("uniform", "float32", 1 << 20, seed=6)
    t = to_device(x)
    h = bs.Handle()
    ws = torch.empty(bs.workspace_bytes(t.numel(), "float32"), dtype=torch.uint8, device="cuda")
    g = bs.Graph(h, t, ws, descending=True)
    g.launch()
    assert g.error() == 0
    assert_bit_exact(t.cpu().numpy(), O.bsort(x, descending=True), "plain graph")


def test_bad_offsets_set_the_error_word():
    import torch
    import paper_2603_08929_gb300 as bs
    x = W.make("uniform", "int32", 1000, seed=8)
    t = to_device(x)
    off = torch.tensor([0, 500, 400, 1000], dtype=torch.int64, device="cuda")  # decreasing
    h = bs.Handle()
    ws = torch.empty(bs.segmented_workspace_bytes(1000, 3, "int32"), dtype=torch.uint8, device="cuda")
    bs.bsort_keys_segmented(t, off, handle=h, workspace=ws)
    assert h.get_error() == 9  # BSORT_ERR_INTERNAL: bounds check on the device
    with pytest.raises(bs.BsortError):
        bs.bsort_keys_segmented(to_device(W.make("uniform", "int16", 100)), torch.tensor([0, 100], dtype=torch.int64,
                                                                                         device="cuda"))
