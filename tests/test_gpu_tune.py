"""Tuned handles (digit width 4..8, smaller finish and merge thresholds) give
the same bytes as the oracle; the autotuner's choice sorts correctly."""
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


def sort_tuned(x, tuning, descending=False, mode=0):
    import torch
    import paper_2603_08929_gb300 as bs
    t = to_device(x)
    h = bs.Handle()
    h.set_tuning(x.dtype.itemsize, tuning)
    ws = torch.empty(bs.workspace_bytes(t.numel(), x.dtype.name, mode=mode, tuning=tuning), dtype=torch.uint8,
                     device=t.device)
    bs.bsort_keys_ws(h, t, ws, descending=descending, mode=mode)
    assert h.get_error() == 0
    return t.cpu().numpy()


TUNINGS = [{"radix_bits": 4}, {"radix_bits": 5}, {"radix_bits": 6}, {"radix_bits": 7},
           {"unit_keys": 256}, {"unit_keys": 1024, "merge_keys": 128}, {"radix_bits": 6, "unit_keys": 2048}]


@pytest.mark.parametrize("n", [3000, 300001, (1 << 22) + 7])
@pytest.mark.parametrize("dtype", ["int32", "float32", "uint64", "float64"])
@pytest.mark.parametrize("tuning", TUNINGS, ids=[str(t) for t in TUNINGS])
def test_tuned_parity(tuning, dtype, n):
    if n > 1 << 21 and dtype in ("float32", "uint64"):
        pytest.skip("large size: one 4- and one 8-byte type")
    x = W.make("uniform", dtype, n, seed=n % 97)
    assert_bit_exact(sort_tuned(x, tuning), O.bsort(x.copy()), "%s %s n=%d" % (tuning, dtype, n))


@pytest.mark.parametrize("dist", ["zipf", "distinct8", "float_edge"])
def test_tuned_distributions(dist):
    x = W.make(dist, "float64", 200003, seed=5)
    for tuning in ({"radix_bits": 5}, {"unit_keys": 512}):
        assert_bit_exact(sort_tuned(x, tuning, descending=True), O.bsort(x.copy(), descending=True), dist)


def test_tuned_inplace():
    x = W.make("uniform", "int32", 1 << 20, seed=6)
    assert_bit_exact(sort_tuned(x, {"radix_bits": 6}, mode=1), O.bsort(x.copy()), "in-place r=6")


def test_autotune_picks_a_candidate_that_sorts(tmp_path):
    from paper_2603_08929_gb300 import tune
    cands = [{"radix_bits": 8, "unit_keys": 0, "merge_keys": 0}, {"radix_bits": 6, "unit_keys": 2048, "merge_keys": 0}]
    table = tune.tune_table(["int32"], [1 << 20], str(tmp_path / "t.json"), candidates=cands, steps=2)
    best = tune.lookup(table, "int32", 1 << 20)
    assert best in [{k: c[k] for k in best} for c in cands]
    x = W.make("uniform", "int32", 1 << 20, seed=7)
    assert_bit_exact(sort_tuned(x, best), O.bsort(x.copy()), "autotuned")
