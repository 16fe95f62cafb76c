"""bfloat16 keys (BSORT_BF16) through the C ABI, bit-exact against the oracle
with the (16, 8, 7) format: plain, in-place and key-value sorts, every
distribution of the float types, both directions; at 2^28 keys, by the rank
of every output pattern."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import assert_bit_exact

pytestmark = pytest.mark.gpu

DISTS = ["uniform", "normal", "float_edge", "distinct8", "zipf", "sorted", "reverse", "normal01"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2603_08929_gb300 import build as b
    b.build()
    torch.cuda.set_device(0)


def to_bf16(words):
    import torch
    return torch.from_numpy(np.ascontiguousarray(words)).cuda().view(torch.bfloat16)


def back(t):
    import torch
    return t.view(torch.int16).cpu().numpy().view(np.uint16)


def oracle_sort(words, desc):
    a = words.astype(np.uint64)
    O.bsort_words(a, O.BF16, desc)
    return a.astype(np.uint16)


@pytest.mark.parametrize("desc", [False, True], ids=["asc", "desc"])
@pytest.mark.parametrize("dist", DISTS)
@pytest.mark.parametrize("n", [2, 3, 1000, 65537, 300001, (1 << 22) + 3])
def test_bf16_parity(n, dist, desc):
    import paper_2603_08929_gb300 as bs
    x = W.make(dist, "bfloat16", n, seed=n % 89)
    t = to_bf16(x)
    bs.bsort_keys(t, descending=desc)
    assert_bit_exact(back(t), oracle_sort(x, desc), "bf16 %s n=%d" % (dist, n))


def test_bf16_inplace_and_default_call():
    import paper_2603_08929_gb300 as bs
    x = W.make("float_edge", "bfloat16", 500001, seed=4)
    t = to_bf16(x)
    bs.sort_(t, mode="inplace", descending=True)
    assert_bit_exact(back(t), oracle_sort(x, True), "bf16 in-place")


@pytest.mark.parametrize("desc", [False, True], ids=["asc", "desc"])
def test_bf16_pairs(desc):
    import torch
    import paper_2603_08929_gb300 as bs
    n = 200003
    x = W.make("float_edge", "bfloat16", n, seed=5)
    k = to_bf16(x)
    vals = torch.arange(n, dtype=torch.int32, device="cuda")
    _, v, ix = bs.sort_pairs_(k, vals, descending=desc, return_indices=True)
    p = O.stable_argsort_words(x.astype(np.uint64), O.BF16, desc)
    assert_bit_exact(back(k), x[p], "bf16 pairs keys")
    assert np.array_equal(ix.cpu().numpy(), p) and np.array_equal(v.cpu().numpy(), p.astype(np.int32))


def test_bf16_full_size_by_rank():
    """2^28 bfloat16 keys: the output holds every input pattern as often as
    the input (per-pattern counts) and the patterns appear in the oracle's
    order of all 2^16 patterns (non-decreasing rank)."""
    import paper_2603_08929_gb300 as bs
    n = 1 << 28
    x = W.make("uniform", "bfloat16", n, seed=6)
    t = to_bf16(x)
    bs.bsort_keys(t)
    got = back(t)
    assert np.array_equal(np.bincount(got, minlength=1 << 16), np.bincount(x, minlength=1 << 16))
    order = oracle_sort(np.arange(1 << 16, dtype=np.uint16), False)
    rank = np.empty(1 << 16, dtype=np.int64)
    rank[order] = np.arange(1 << 16)
    r = rank[got]
    assert np.all(r[1:] >= r[:-1])
