"""Intermediate parity of the digit passes: after L MSD levels of r bits the
GPU buffer is partitioned by the top L*r bits of the paper's order, with
the same bucket boundaries (invariants (i)/(ii) of Alg. 1 at each of those
bits).  The digit pass is not stable, so the check is the one the order
fixes: the oracle's STABLE partition of the GPU state by its first L*r bit
levels leaves it unchanged (a stable partition of an already partitioned
sequence is the identity), and the GPU state is the input's multiset."""
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


def partial(x, levels, descending=False, tuning=None):
    import torch
    import paper_2603_08929_gb300 as bs
    t = to_device(x)
    h = bs.Handle()
    if tuning:
        h.set_tuning(x.dtype.itemsize, tuning)
    ws = torch.empty(bs.workspace_bytes(t.numel(), x.dtype.name, tuning=tuning), dtype=torch.uint8, device=t.device)
    bs.bsort_keys_partial_ws(h, t, ws, levels, descending=descending)
    assert h.get_error() == 0
    return t.cpu().numpy()


def check_partitioned(x, g, bits, descending):
    assert O.multiset_digest(g) == O.multiset_digest(x), "not a permutation of the input"
    again = O.bsort(g.copy(), descending=descending, mode=O.STABLE, max_levels=bits)
    assert_bit_exact(again, g, "not partitioned by the top %d bits" % bits)


@pytest.mark.parametrize("desc", [False, True], ids=["asc", "desc"])
@pytest.mark.parametrize("dtype,n", [("uint32", 1 << 20), ("int32", 300001), ("float32", (1 << 21) + 3),
                                     ("int64", 300001), ("float64", 1 << 20)])
def test_partition_after_each_level(dtype, n, desc):
    x = W.make("uniform", dtype, n, seed=n % 89)
    w = x.dtype.itemsize * 8
    for levels in range(1, w // 8):
        g = partial(x, levels, desc)
        check_partitioned(x, g, 8 * levels, desc)
    # all levels: the complete sort
    assert_bit_exact(partial(x, w // 8, desc), O.bsort(x.copy(), descending=desc), "all levels")


@pytest.mark.parametrize("dist", ["zipf", "normal", "distinct8", "float_edge"])
def test_partition_distributions(dist):
    x = W.make(dist, "float32", 500003, seed=3)
    for levels in (1, 2, 3):
        check_partitioned(x, partial(x, levels), 8 * levels, False)


@pytest.mark.parametrize("r", [4, 5, 6])
def test_partition_with_narrow_digits(r):
    x = W.make("uniform", "int32", 1 << 20, seed=4)
    for levels in (1, 2, 3):
        check_partitioned(x, partial(x, levels, tuning={"radix_bits": r}), r * levels, False)
