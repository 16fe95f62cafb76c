"""Tuned handles (digit width 1..11, smaller finish and merge thresholds,
chunks of one tile) give the same bytes as the oracle, in plain, in-place and
segmented sorts; the autotuners' choices sort correctly."""
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


TUNINGS = [{"radix_bits": 1}, {"radix_bits": 2}, {"radix_bits": 3}, {"radix_bits": 4}, {"radix_bits": 5}, {"radix_bits": 6}, {"radix_bits": 7},
           {"radix_bits": 9}, {"radix_bits": 10}, {"radix_bits": 11}, {"chunk_tiles": 1},
           {"unit_keys": 256}, {"unit_keys": 1024, "merge_keys": 128}, {"radix_bits": 6, "unit_keys": 2048},
           {"radix_bits": 11, "unit_keys": 1024, "chunk_tiles": 1}, {"radix_bits": 10, "unit_keys": 256}]


@pytest.mark.parametrize("n", [3000, 300001, (1 << 22) + 7])
@pytest.mark.parametrize("dtype", ["int32", "float32", "uint64", "float64"])
@pytest.mark.parametrize("tuning", TUNINGS, ids=[str(t) for t in TUNINGS])
def test_tuned_parity(tuning, dtype, n):
    if n > 1 << 21 and dtype in ("float32", "uint64"):
        pytest.skip("large size: one 4- and one 8-byte type")
    x = W.make("uniform", dtype, n, seed=n % 97)
    assert_bit_exact(sort_tuned(x, tuning), O.bsort(x.copy()), "%s %s n=%d" % (tuning, dtype, n))


@pytest.mark.parametrize("dist", ["zipf", "distinct8", "float_edge", "sorted", "reverse"])
@pytest.mark.parametrize("dtype", ["float64", "int32"])
def test_tuned_distributions(dist, dtype):
    if dist == "float_edge" and dtype == "int32":
        pytest.skip("float-only distribution")
    x = W.make(dist, dtype, 200003, seed=5)
    for tuning in ({"radix_bits": 5}, {"unit_keys": 512}, {"radix_bits": 11}, {"radix_bits": 9, "chunk_tiles": 1},
                   {"radix_bits": 1}, {"radix_bits": 2, "unit_keys": 256}):
        assert_bit_exact(sort_tuned(x, tuning, descending=True), O.bsort(x.copy(), descending=True),
                         "%s %s" % (dist, tuning))


@pytest.mark.parametrize("tuning", [{"radix_bits": 6}, {"radix_bits": 11}, {"radix_bits": 10, "chunk_tiles": 1},
                                    {"radix_bits": 1}, {"radix_bits": 3}],
                         ids=["r6", "r11-as-8", "r10-as-8-chunk1", "r1", "r3"])
def test_tuned_inplace(tuning):
    """In place, digits wider than 8 bits run as 8 bits: same bytes."""
    x = W.make("uniform", "int32", 1 << 20, seed=6)
    assert_bit_exact(sort_tuned(x, tuning, mode=1), O.bsort(x.copy()), "in-place %s" % tuning)


@pytest.mark.parametrize("dtype", ["int32", "float64"])
def test_wide_digits_full_size(dtype):
    """11-bit digits at the full sizes (2^28 4-byte, 2^27 8-byte keys),
    byte for byte against the oracle."""
    from gpu_util import check_full_size
    n = 1 << (28 if dtype == "int32" else 27)
    x = W.make("uniform", dtype, n, seed=11)
    check_full_size(x, sort_tuned(x, {"radix_bits": 11}), False)


def _segments(dtype, seed):
    import torch
    rng = np.random.default_rng(seed)
    sizes = np.concatenate([[0, 1, 2, 7], rng.integers(0, 60, 40), [5000, 70001, 300000, 1 << 20],
                            W.segment_sizes(seed, 200, 17)])
    rng.shuffle(sizes)
    n = int(sizes.sum())
    x = W.make("float_edge" if dtype.startswith("float") else "uniform", dtype, n, seed=seed)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    want = x.copy()
    for a, b in zip(off[:-1], off[1:]):
        if b - a > 1:
            want[a:b] = O.bsort(x[a:b])
    return x, torch.from_numpy(off).cuda(), want


@pytest.mark.parametrize("tuning", [{"radix_bits": 11}, {"radix_bits": 4, "chunk_tiles": 1},
                                    {"radix_bits": 9, "unit_keys": 512}], ids=["r11", "r4-chunk1", "r9-u512"])
@pytest.mark.parametrize("dtype", ["int32", "float64"])
def test_tuned_segmented(dtype, tuning):
    """The segmented call on a tuned handle (and its captured graph) follows
    the handle's tuning: same bytes as the oracle per segment."""
    import torch
    import paper_2603_08929_gb300 as bs
    x, off, want = _segments(dtype, 21)
    t = to_device(x)
    h = bs.Handle()
    h.set_tuning(x.dtype.itemsize, tuning)
    ws = torch.empty(bs.segmented_workspace_bytes(t.numel(), off.numel() - 1, dtype, tuning=tuning),
                     dtype=torch.uint8, device="cuda")
    bs.bsort_keys_segmented(t, off, handle=h, workspace=ws)
    assert h.get_error() == 0
    assert_bit_exact(t.cpu().numpy(), want, "segmented %s %s" % (dtype, tuning))
    g = bs.Graph(h, t, ws, offsets=off)
    t.copy_(torch.from_numpy(x).cuda())
    g.launch()
    assert g.error() == 0
    assert_bit_exact(t.cpu().numpy(), want, "segmented graph %s %s" % (dtype, tuning))


def test_tuned_workspace_too_small_for_the_segmented_call():
    """A tuned handle refuses a workspace sized for the defaults when its
    tuning needs more."""
    import torch
    import paper_2603_08929_gb300 as bs
    x, off, _ = _segments("int32", 22)
    t = to_device(x)
    h = bs.Handle()
    h.set_tuning(4, {"radix_bits": 11})
    ws = torch.empty(bs.segmented_workspace_bytes(t.numel(), off.numel() - 1, "int32"), dtype=torch.uint8,
                     device="cuda")
    with pytest.raises(bs.BsortError):
        bs.bsort_keys_segmented(t, off, handle=h, workspace=ws)


def test_autotune_picks_a_candidate_that_sorts(tmp_path):
    from paper_2603_08929_gb300 import tune
    cands = [{"radix_bits": 8, "unit_keys": 0, "merge_keys": 0, "chunk_tiles": 0},
             {"radix_bits": 11, "unit_keys": 2048, "merge_keys": 0, "chunk_tiles": 1}]
    table = tune.tune_table(["int32"], [1 << 20], str(tmp_path / "t.json"), candidates=cands, steps=2)
    best = tune.lookup(table, "int32", 1 << 20)
    assert best in [{k: c[k] for k in best} for c in cands]
    x = W.make("uniform", "int32", 1 << 20, seed=7)
    assert_bit_exact(sort_tuned(x, best), O.bsort(x.copy()), "autotuned")


def test_autotune_segmented_picks_a_candidate_that_sorts():
    import torch
    import paper_2603_08929_gb300 as bs
    from paper_2603_08929_gb300 import tune
    x, off, want = _segments("int32", 23)
    keys = to_device(x)
    log = []
    best = tune.autotune_segmented(keys, off, steps=1, log=log)
    assert len(log) == len(tune.CANDIDATES) and all(ms > 0 for _, ms in log)
    assert_bit_exact(keys.cpu().numpy(), x, "the tuner leaves its input unchanged")
    tuning = {f: best[f] for f in tune.FIELDS}
    assert tuning in tune.CANDIDATES
    h = bs.Handle()
    h.set_tuning(4, tuning)
    ws = torch.empty(bs.segmented_workspace_bytes(keys.numel(), off.numel() - 1, "int32", tuning=tuning),
                     dtype=torch.uint8, device="cuda")
    bs.bsort_keys_segmented(keys, off, handle=h, workspace=ws)
    assert_bit_exact(keys.cpu().numpy(), want, "autotuned segmented")
