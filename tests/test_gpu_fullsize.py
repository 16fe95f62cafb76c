"""Full-size parity: the plain-sort configuration at its own sizes (2^28
keys of 1/2/4-byte types, 2^27 of 8-byte types) and the float edge-case
stress at 2^26, sorted by the same call the benchmark times.  At these sizes
the oracle checks properties that pin the result completely: the output is
non-decreasing under the paper's order (the oracle's comparator) and is the
same multiset as the input, so it is the unique sorted sequence; two sampled
positions are also checked against the oracle's rank of their key."""
import numpy as np
import pytest

import workloads as W
from gpu_util import check_full_size

pytestmark = pytest.mark.gpu

NARROW = ["uint8", "int8", "uint16", "int16", "float16", "uint32", "int32", "float32"]
WIDE = ["uint64", "int64", "float64"]
OTHER_DISTS = ["zipf", "normal", "distinct8", "sorted", "reverse"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2603_08929_gb300 import build as b
    b.build()
    torch.cuda.set_device(0)


_sorted_cache = {}


def make(dist, dtype, n):
    """W.make(dist, dtype, n, seed=0); "reverse" reuses the "sorted" array of
    the same dtype (W.make defines it as that array reversed)."""
    if dist in ("sorted", "reverse"):
        if dtype not in _sorted_cache:
            _sorted_cache.clear()
            _sorted_cache[dtype] = W.make("sorted", dtype, n, seed=0)
        x = _sorted_cache[dtype]
        return x if dist == "sorted" else x[::-1].copy()
    return W.make(dist, dtype, n, seed=0)


def full_n(dtype):
    return 1 << 27 if dtype in WIDE else 1 << 28


def sort_like_bench(x, descending):
    """bsort_keys_ws with an explicit workspace on the current stream (the
    benchmark's call)."""
    import torch
    import paper_2603_08929_gb300 as bs
    t = torch.from_numpy(x).cuda()
    ws = torch.empty(bs.workspace_bytes(t.numel(), x.dtype.name), dtype=torch.uint8, device=t.device)
    h = bs.Handle()
    bs.bsort_keys_ws(h, t, ws, descending=descending, stream=torch.cuda.current_stream())
    assert h.get_error() == 0
    out = t.cpu().numpy()
    del t, ws
    return out


# every dtype x every distribution of the configuration, the direction
# alternating over the distributions (and flipped between neighbouring
# dtypes), plus uniform in the other direction for every dtype
DISTS = ["uniform"] + OTHER_DISTS
CASES = [(dt, dist, (i + k) % 2 == 1) for k, dt in enumerate(NARROW + WIDE) for i, dist in enumerate(DISTS)]
CASES += [(dt, "uniform", k % 2 == 0) for k, dt in enumerate(NARROW + WIDE)]


@pytest.mark.parametrize("dtype,dist,desc", CASES, ids=["%s-%s-%s" % (d, s, "desc" if r else "asc")
                                                        for d, s, r in CASES])
def test_full_size(dtype, dist, desc):
    x = make(dist, dtype, full_n(dtype))
    got = sort_like_bench(x, desc)
    check_full_size(x, got, desc, samples=2)


@pytest.mark.parametrize("desc", [False, True], ids=["asc", "desc"])
@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_float_edge_full_size(dtype, desc):
    x = W.make("float_edge", dtype, 1 << 26, seed=0)
    got = sort_like_bench(x, desc)
    check_full_size(x, got, desc, samples=2)
