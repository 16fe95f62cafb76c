"""128-bit integer keys (uint128, int128) through the MSD pipeline on the
GPU, byte for byte against the oracle's two-word restatement of Algs. 1-3.
Keys travel as uint64 (n, 2) arrays, low word first."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import assert_bit_exact

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2603_08929_gb300 import build as b
    b.build()
    torch.cuda.set_device(0)


def gpu_sort(x, dtype, descending=False):
    import torch
    import paper_2603_08929_gb300 as bs
    t = torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda()
    bs.bsort_keys(t, descending=descending, dtype=dtype)
    return t.cpu().numpy().view(np.uint64)


SIZES = [2, 3, 1000, 1264, 1265, 5000, 70001, (1 << 20) + 3]


@pytest.mark.parametrize("desc", [False, True], ids=["asc", "desc"])
@pytest.mark.parametrize("dist", ["uniform", "zipf", "distinct8", "normal01"])
@pytest.mark.parametrize("dtype", ["uint128", "int128"])
@pytest.mark.parametrize("n", SIZES)
def test_wide_parity(n, dtype, dist, desc):
    x = W.make(dist, dtype, n, seed=n % 97)
    want = O.bsort128(x, signed=dtype == "int128", descending=desc)
    assert_bit_exact(gpu_sort(x, dtype, desc), want, "%s %s n=%d" % (dtype, dist, n))


@pytest.mark.parametrize("dtype", ["uint128", "int128"])
def test_wide_special_patterns(dtype):
    """Keys that differ only across the word boundary, only in the top or the
    bottom bit, all-equal runs and the extreme values."""
    rng = np.random.default_rng(3)
    base = [(0, 0), (2**64 - 1, 0), (0, 1), (0, 2**63), (2**64 - 1, 2**64 - 1), (1, 0), (0, 2**63 - 1),
            (2**63, 0), (2**64 - 1, 2**63 - 1), (0, 2**63 + 1)]
    x = np.array([base[i] for i in rng.integers(0, len(base), 50000)], dtype=np.uint64)
    x[:100] = x[100]  # a long run of one key
    for desc in (False, True):
        want = O.bsort128(x, signed=dtype == "int128", descending=desc)
        assert_bit_exact(gpu_sort(x, dtype, desc), want, "special %s" % dtype)


def test_wide_4m_keys():
    """2^22 uniform int128 keys: three 8-bit levels and the finish."""
    x = W.make("uniform", "int128", 1 << 22, seed=22)
    assert_bit_exact(gpu_sort(x, "int128"), O.bsort128(x, signed=True), "int128 2^22")


def test_wide_segmented():
    import torch
    import paper_2603_08929_gb300 as bs
    sizes = np.concatenate([[0, 1, 2], W.segment_sizes(8, 200, 15)])
    x = W.make("uniform", "uint128", int(sizes.sum()), seed=8)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    t = torch.from_numpy(x.view(np.int64).copy()).cuda()
    bs.bsort_keys_segmented(t, torch.from_numpy(off).cuda(), descending=True, dtype="uint128")
    got = t.cpu().numpy().view(np.uint64)
    want = x.copy()
    for a, b in zip(off[:-1], off[1:]):
        if b - a > 1:
            want[a:b] = O.bsort128(x[a:b], descending=True)
    assert_bit_exact(got, want, "segmented uint128")


def test_wide_unsupported_forms():
    """The in-place mode and the key-value sort take keys of up to 8 bytes;
    16-byte keys must be 16-byte aligned."""
    import torch
    import paper_2603_08929_gb300 as bs
    with pytest.raises(bs.BsortError):
        bs.workspace_bytes(1000, "uint128", mode=bs.MODE_INPLACE)
    with pytest.raises(bs.BsortError):
        bs.pairs_workspace_bytes(1000, "int128")
    buf = torch.zeros(2 * 1001, dtype=torch.int64, device="cuda")
    with pytest.raises(bs.BsortError):
        bs.bsort_keys(buf[1:2001], dtype="uint128")  # 8 bytes past a 16-byte boundary
