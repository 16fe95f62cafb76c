"""GPU sorts through the C ABI against the oracle, element by element."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import assert_bit_exact, check_full_size, gpu_sort, to_device

pytestmark = pytest.mark.gpu

INT_DISTS = ["uniform", "zipf", "distinct8", "sorted", "reverse", "normal"]
FLOAT_DISTS = INT_DISTS + ["float_edge"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2603_08929_gb300 import build as b
    b.build()
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)


def dists_of(dtype):
    return FLOAT_DISTS if dtype.startswith("float") else INT_DISTS


def check(dtype, dist, n, desc, seed=0):
    x = W.make(dist, dtype, n, seed=seed)
    want = O.bsort(x, descending=desc)
    got = gpu_sort(x, desc)
    assert_bit_exact(got, want, "%s %s n=%d desc=%s" % (dtype, dist, n, desc))


def test_config1_int32_65536_seed0():
    """65,536 int32 keys uniform over the full range from seed 0, ascending."""
    check("int32", "uniform", 65536, False, seed=0)


@pytest.mark.parametrize("desc", [False, True], ids=["asc", "desc"])
@pytest.mark.parametrize("n", [0, 1, 2, 3, 31, 32, 33, 1000, 4095, 4096, 4097, 8191, 8192, 8193,
                               16385, 65536, 100003])
@pytest.mark.parametrize("dtype", W.DTYPES)
def test_sizes(dtype, n, desc):
    check(dtype, "uniform", n, desc)


@pytest.mark.parametrize("desc", [False, True], ids=["asc", "desc"])
@pytest.mark.parametrize("dtype", W.DTYPES)
def test_distributions(dtype, desc):
    for dist in dists_of(dtype):
        check(dtype, dist, 300001, desc, seed=1)


@pytest.mark.parametrize("dtype", W.DTYPES)
def test_two_msd_levels(dtype):
    # 2^22 + 7 keys: buckets after the first 8-bit digit still exceed the
    # shared-memory finish, so a second level runs
    for dist in ("uniform", "zipf", "distinct8"):
        check(dtype, dist, (1 << 22) + 7, dist == "zipf", seed=2)


@pytest.mark.parametrize("dtype", ["float16", "float32", "float64"])
def test_special_values(dtype):
    from oracle_pins import _special_float_sequence
    seq = np.array(_special_float_sequence(dtype), dtype=np.uint64)
    w = np.dtype(dtype).itemsize * 8
    ut = {16: np.uint16, 32: np.uint32, 64: np.uint64}[w]
    rng = np.random.default_rng(0)
    x = np.tile(seq, 500)
    x = x[rng.permutation(x.size)].astype(ut).view(dtype)
    for desc in (False, True):
        got = gpu_sort(x, desc)
        assert_bit_exact(got, O.bsort(x, descending=desc), "special values desc=%s" % desc)


def test_desc_is_reverse_of_asc():
    x = W.make("float_edge", "float32", 200000, seed=5)
    a = gpu_sort(x, False)
    d = gpu_sort(x, True)
    assert_bit_exact(d, a[::-1].copy(), "desc vs reversed asc")


def test_deterministic_repeat():
    x = W.make("zipf", "int64", 500000, seed=6)
    assert_bit_exact(gpu_sort(x), gpu_sort(x), "repeat")


def test_explicit_workspace_and_stream():
    import torch
    import paper_2603_08929_gb300 as bs
    x = W.make("uniform", "uint32", 1 << 20, seed=7)
    t = to_device(x)
    ws = torch.empty(bs.workspace_bytes(x.size, "uint32"), dtype=torch.uint8, device="cuda")
    h = bs.Handle()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        bs.bsort_keys_ws(h, t, ws, descending=False, stream=s)
    s.synchronize()
    assert h.get_error(s) == 0
    assert_bit_exact(t.cpu().numpy(), O.bsort(x), "bsort_keys_ws")
    # a workspace one byte short is rejected before any launch
    with pytest.raises(bs.BsortError):
        bs.bsort_keys_ws(h, t, ws[:-257], stream=s)


def test_host_entry_point():
    import paper_2603_08929_gb300 as bs
    for dtype, dist in (("float64", "float_edge"), ("int16", "normal"), ("uint32", "sorted")):
        x = W.make(dist, dtype, 123457, seed=8)
        y = x.copy()
        bs.bsort_keys_host(y)
        assert_bit_exact(y, O.bsort(x), "bsort_keys_host %s" % dtype)


def test_misaligned_and_offset_views():
    import paper_2603_08929_gb300 as bs
    x = W.make("uniform", "int32", 50001, seed=9)
    t = to_device(np.concatenate([np.zeros(1, np.int32), x]))
    v = t[1:]  # 4-byte aligned, not 16-byte aligned
    bs.bsort_keys(v)
    assert_bit_exact(v.cpu().numpy(), O.bsort(x), "offset view")
    assert int(t[0]) == 0


def _sorted_with_profile(x, descending=False):
    import torch
    import paper_2603_08929_gb300 as bs
    t = to_device(x)
    h = bs.Handle()
    h.set_profiling(True)
    ws = torch.empty(bs.workspace_bytes(t.numel(), x.dtype.name), dtype=torch.uint8, device=t.device)
    bs.bsort_keys_ws(h, t, ws, descending=descending)
    prof = h.profile()
    assert h.get_error() == 0
    return t.cpu().numpy(), prof["finish_units"]


@pytest.mark.gpu
@pytest.mark.parametrize("dtype,n,desc", [("uint32", 4096, False), ("int32", 5104, True), ("uint64", 2100, False),
                                          ("uint32", 1023, False), ("float32", 4999, False)])
def test_counting_finish(dtype, n, desc):
    """One unit whose keys vary only in their low 16 bits (and enough keys to
    fill 2^12 sub-buckets): the one-pass counting finish sorts it."""
    rng = np.random.default_rng(n)
    if dtype == "float32":
        x = (1.0 + rng.integers(0, 1 << 16, n) * 2.0 ** -23).astype(np.float32)  # mantissa low 16 bits
    else:
        x = rng.integers(0, 1 << 16, n).astype(dtype)
    got, fu = _sorted_with_profile(x, desc)
    assert_bit_exact(got, O.bsort(x.copy(), descending=desc), dtype)
    want = {"counting": 1 if n >= 1024 else 0}
    assert fu["counting"] == want["counting"], fu


@pytest.mark.gpu
def test_counting_finish_overflow_falls_back():
    """Sixteen equal keys overflow a 4-bit counter: the unit is ranked by the
    split + comparison path instead, with the same result."""
    rng = np.random.default_rng(5)
    x = rng.integers(0, 1 << 16, 4000).astype(np.uint32)
    x[:40] = 12345
    rng.shuffle(x)
    got, fu = _sorted_with_profile(x)
    assert_bit_exact(got, O.bsort(x.copy()), "uint32")
    assert fu["counting"] == 0 and fu["compare"] + fu["lsd"] == 1, fu


@pytest.mark.gpu
def test_counting_finish_full_size():
    """2^27 uniform int32 keys: two 8-bit levels leave buckets of ~2048 keys
    with 16 varying bits, all finished by the counting pass."""
    x = W.make("uniform", "int32", 1 << 27, seed=78)
    got, fu = _sorted_with_profile(x)
    assert fu["counting"] > 0.99 * (fu["counting"] + fu["compare"] + fu["lsd"]), fu
    check_full_size(x, got, False)


@pytest.mark.gpu
def test_launch_count_is_every_kernel():
    """The count the benchmark reports as gpu_launches: every kernel of a call."""
    import torch
    import paper_2603_08929_gb300 as bs
    h = bs.Handle()
    for n, want in ((1 << 20, 1 + 4 * 4 + 2 + 1), (3000, 1 + 2), (1 << 19, None)):
        x = W.make("uniform", "int32", n, seed=1)
        t = to_device(x)
        ws = torch.empty(bs.workspace_bytes(n, "int32"), dtype=torch.uint8, device=t.device)
        bs.bsort_keys_ws(h, t, ws)
        if want is not None:
            assert h.launch_count() == want, (n, h.launch_count())
    x = W.make("uniform", "uint16", 1 << 20, seed=1)
    t = to_device(x)
    ws = torch.empty(bs.workspace_bytes(t.numel(), "uint16"), dtype=torch.uint8, device=t.device)
    bs.bsort_keys_ws(h, t, ws)
    assert h.launch_count() == 4  # histogram, reduce, scan, fill
