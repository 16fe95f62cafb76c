"""Key-value sorting through the C ABI: the sorted keys, the values carried
along and the returned positions equal the oracle's stable permutation bit
for bit; at large sizes, the properties that make a permutation the stable
sorting one."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import assert_bit_exact, par_first_unsorted, to_device

pytestmark = pytest.mark.gpu

DTYPES = ["uint8", "int8", "uint16", "int16", "float16", "uint32", "int32", "float32", "uint64", "int64", "float64"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2603_08929_gb300 import build as b
    b.build()
    torch.cuda.set_device(0)


def run_pairs(x, values=None, desc=False, indices=True, tuning8=None):
    import torch
    import paper_2603_08929_gb300 as bs
    k = to_device(x)
    v = to_device(values) if values is not None else None
    h = bs.Handle()
    if tuning8:
        h.set_tuning(8, tuning8)
    ws = torch.empty(max(1, bs.pairs_workspace_bytes(k.numel(), k.dtype, tuning8=tuning8)), dtype=torch.uint8,
                     device="cuda")
    ix = torch.empty(k.numel(), dtype=torch.int64, device="cuda") if indices else None
    bs.bsort_pairs_ws(h, k, ws, values=v, indices=ix, descending=desc)
    assert h.get_error() == 0
    return (k.cpu().numpy(), v.cpu().numpy() if v is not None else None,
            ix.cpu().numpy() if ix is not None else None, h)


def check(x, vals, desc, got):
    k, v, ix, _ = got
    p = O.stable_argsort(x, desc)
    assert_bit_exact(k, x[p], "keys")
    if vals is not None:
        assert_bit_exact(v, vals[p], "values")
    if ix is not None:
        assert np.array_equal(ix, p), "positions differ from the stable permutation"


def _dists(dtype):
    base = ["uniform", "distinct8", "zipf", "sorted", "reverse"]
    return base + (["float_edge"] if dtype.startswith("float") else [])


@pytest.mark.parametrize("desc", [False, True], ids=["asc", "desc"])
@pytest.mark.parametrize("dtype", DTYPES)
def test_pairs_parity(dtype, desc):
    n = 100003
    for j, dist in enumerate(_dists(dtype)):
        x = W.make(dist, dtype, n, seed=40 + j)
        vals = (np.arange(n, dtype=np.int64) * 7919 + 3).astype(np.int32)
        check(x, vals, desc, run_pairs(x, vals, desc))


@pytest.mark.parametrize("n", [2, 3, 17, 5000, 300001, (1 << 22) + 5])
@pytest.mark.parametrize("dtype", ["int32", "float64", "uint16"])
def test_pairs_sizes(dtype, n):
    x = W.make("distinct8" if n % 2 else "uniform", dtype, n, seed=n % 101)
    vals = W.make("uniform", "float64", n, seed=7)
    check(x, vals, n % 3 == 0, run_pairs(x, vals, n % 3 == 0))


def test_pairs_tiny_and_empty():
    import torch
    import paper_2603_08929_gb300 as bs
    h = bs.Handle()
    ws = torch.empty(256, dtype=torch.uint8, device="cuda")
    k = torch.empty(0, dtype=torch.int32, device="cuda")
    bs.bsort_pairs_ws(h, k, ws, values=torch.empty(0, dtype=torch.int32, device="cuda"),
                      indices=torch.empty(0, dtype=torch.int64, device="cuda"))
    k = torch.tensor([5], dtype=torch.int32, device="cuda")
    ix = torch.full((1,), 99, dtype=torch.int64, device="cuda")
    bs.bsort_pairs_ws(h, k, ws, values=torch.tensor([7.0], device="cuda"), indices=ix)
    assert ix.item() == 0 and k.item() == 5


@pytest.mark.parametrize("vdtype", ["uint8", "int16", "float32", "int64"])
def test_pairs_value_widths(vdtype):
    n = 70001
    x = W.make("zipf", "int32", n, seed=3)
    vals = W.make("uniform", vdtype, n, seed=4)
    check(x, vals, False, run_pairs(x, vals, False))


def test_pairs_without_indices_or_values():
    n = 50001
    x = W.make("distinct8", "float32", n, seed=5)
    vals = W.make("uniform", "int64", n, seed=6)
    check(x, vals, True, run_pairs(x, vals, True, indices=False))
    check(x, None, False, run_pairs(x, None, False, indices=True))
    k, _, _, _ = run_pairs(x, None, False, indices=False)
    assert_bit_exact(k, O.bsort(x), "keys only")


@pytest.mark.parametrize("tuning8", [{"radix_bits": 11}, {"radix_bits": 6, "chunk_tiles": 1}], ids=["r11", "r6c1"])
def test_pairs_tuned_handle(tuning8):
    n = 300007
    for dtype in ("int32", "float64"):
        x = W.make("distinct8", dtype, n, seed=8)
        vals = np.arange(n, dtype=np.int32)
        check(x, vals, False, run_pairs(x, vals, False, tuning8=tuning8))


def test_pairs_launch_counts():
    """One value-carrying MSD pass sequence (init, four kernels per 8-bit
    level of the key words, finish, fill), plus one gather when values follow
    the positions; 1- and 2-byte keys add the widening and narrowing of
    their order codes around a 4-byte-key sequence."""
    n = 1 << 20
    for dtype, kb, extra in (("int32", 4, 0), ("float64", 8, 0), ("int16", 4, 2), ("uint8", 4, 2)):
        x = W.make("uniform", dtype, n, seed=9)
        vals = np.arange(n, dtype=np.int32)
        _, _, _, hp = run_pairs(x, vals, False, indices=False)
        assert hp.launch_count() == 3 + 4 * kb + extra, (dtype, hp.launch_count())
        _, _, _, hp = run_pairs(x, vals, False, indices=True)
        assert hp.launch_count() == 4 + 4 * kb + extra, (dtype, hp.launch_count())


KV_KEYS = ["int32", "uint32", "float32", "int64", "uint64", "float64"]


@pytest.mark.parametrize("vdtype", ["int32", "int64"])
@pytest.mark.parametrize("dtype", KV_KEYS)
def test_pairs_carried_values(dtype, vdtype):
    """Values of 4 and 8 bytes travel with their keys through every level
    (no positions asked for): equal to the oracle's stable permutation, for
    tie-heavy, skewed, presorted and uniform keys, ascending and descending,
    at a size spanning many scatter tiles with a ragged last one."""
    n = 3 * 4096 * 17 + 1234
    for j, dist in enumerate(_dists(dtype)):
        x = W.make(dist, dtype, n, seed=60 + j)
        vals = W.make("uniform", vdtype, n, seed=70 + j)
        desc = j % 2 == 1
        check(x, vals, desc, run_pairs(x, vals, desc, indices=False))


@pytest.mark.parametrize("dtype", ["int32", "uint64"])
@pytest.mark.parametrize("n", [2, 31, 2559, 2560, 2561, 3072, 3073, 5119, 5120, 5121, 65536 + 7])
def test_pairs_unit_boundaries(dtype, n):
    """Sizes around the finish capacity of each key/value width (one unit
    sorted directly, or the MSD levels first), every request form."""
    x = W.make("distinct8" if n % 2 else "uniform", dtype, n, seed=n)
    for vd in ("int32", "int64", "uint8"):
        vals = W.make("uniform", vd, n, seed=n + 1)
        check(x, vals, n % 3 == 0, run_pairs(x, vals, n % 3 == 0, indices=False))
        check(x, vals, n % 3 == 1, run_pairs(x, vals, n % 3 == 1, indices=True))
    check(x, None, False, run_pairs(x, None, False, indices=True))


@pytest.mark.parametrize("dtype", ["int64", "uint64", "int32"])
@pytest.mark.parametrize("n", [2000, 2559, 5000, 100003])
@pytest.mark.parametrize("high", [4, 256, 1 << 16])
def test_pairs_wide_units(dtype, n, high):
    """Finish units with more than 24 varying bits: stable passes over the
    top 16, then runs of ties there sorted by the whole key -- short runs
    (high = 2^16 top values: few ties), runs around the 16 keys the
    insertion sort takes (256 values for ~2000-key units) and runs far
    longer (high = 4), which take every pass.  Keys: a random high part
    above a gap of zero bits and a random low part."""
    rng = np.random.default_rng(n + high)
    shift = 40 if dtype != "int32" else 28
    lowbits = 20 if dtype != "int32" else 16
    hi_part = rng.integers(0, min(high, 1 << (63 - shift if dtype != "int32" else 3)), n).astype(np.int64)
    x = ((hi_part << shift) | rng.integers(0, 1 << lowbits, n)).astype(dtype)
    if dtype.startswith("int"):
        x[::7] = -x[::7]  # both signs
    vals = W.make("uniform", "int64", n, seed=n + 3)
    check(x, vals, False, run_pairs(x, vals, False, indices=False))
    check(x, vals, True, run_pairs(x, vals, True, indices=True))
    check(x, None, False, run_pairs(x, None, False, indices=True))


@pytest.mark.parametrize("dtype", ["int32", "float64"])
def test_pairs_degenerate_keys(dtype):
    """All keys equal (the whole array one run: values keep input order, the
    positions are the identity), two values only, and keys that agree on
    their top bytes (the levels re-open in place, keys still raw)."""
    n = 200003
    np_t = np.dtype(dtype)
    same = np.full(n, 3, dtype=np_t)
    two = np.where(np.arange(n) % 3 == 0, 1, -2).astype(np_t)
    low = (W.make("uniform", "uint32", n, seed=5) & 0x3ff).astype(np_t)
    for x in (same, two, low):
        vals = np.arange(n, dtype=np.int64) * 3
        check(x, vals, False, run_pairs(x, vals, False, indices=False))
        check(x, vals, True, run_pairs(x, vals, True, indices=True))
        check(x, None, False, run_pairs(x, None, False, indices=True))


def test_python_helpers():
    import torch
    import paper_2603_08929_gb300 as bs
    x = W.make("distinct8", "int64", 123457, seed=10)
    t = to_device(x)
    ix = bs.argsort(t, descending=True)
    assert np.array_equal(ix.cpu().numpy(), O.stable_argsort(x, True))
    assert_bit_exact(t.cpu().numpy(), x, "argsort leaves its input unchanged")
    vals = torch.arange(x.size, dtype=torch.float32, device="cuda")
    k, v, i = bs.sort_pairs_(t, vals, return_indices=True)
    p = O.stable_argsort(x)
    assert_bit_exact(k.cpu().numpy(), x[p], "sort_pairs_ keys")
    assert np.array_equal(v.cpu().numpy(), p.astype(np.float32)) and np.array_equal(i.cpu().numpy(), p)


@pytest.mark.parametrize("dtype,log2n", [("int32", 27), ("float64", 26)])
def test_pairs_large_properties(dtype, log2n):
    """At 2^27 / 2^26 keys, tie-heavy: the positions form a permutation, the
    keys they gather are the output keys, the output is monotone under the
    oracle's order, and ties are in input order -- together the stable
    sorting permutation, uniquely."""
    n = 1 << log2n
    x = W.make("distinct8", dtype, n, seed=11)
    k, _, ix, _ = run_pairs(x, None, False)
    check_stable_permutation(x, k, ix)


def check_stable_permutation(x, k, ix, desc=False):
    n = x.size
    assert ix.min() >= 0 and ix.max() < n
    seen = np.zeros(n, dtype=bool)
    seen[ix] = True
    assert seen.all(), "positions are not a permutation"
    assert_bit_exact(k, x[ix], "keys gathered by the positions")
    assert par_first_unsorted(k, desc) == -1
    kw = k.view({4: np.uint32, 8: np.uint64}[k.dtype.itemsize])
    same = kw[1:] == kw[:-1]
    assert np.all(ix[1:][same] > ix[:-1][same]), "ties out of input order"


@pytest.mark.parametrize("dist,vdtype", [("uniform", "int32"), ("distinct8", "int32"), ("uniform", "int64")])
def test_pairs_carried_at_size(dist, vdtype):
    """The key-value workload at full size: 2^28 int32 keys carrying int32
    values, or int64 values (the large-array finish of 12-byte pairs), the
    values being their input positions, so the carried values are the
    permutation: a permutation, the keys it gathers are the output, sorted,
    ties in input order."""
    n = 1 << 28
    x = W.make(dist, "int32", n, seed=12)
    vals = np.arange(n, dtype=vdtype)
    k, v, _, _ = run_pairs(x, vals, False, indices=False)
    check_stable_permutation(x, k, v.astype(np.int64))
