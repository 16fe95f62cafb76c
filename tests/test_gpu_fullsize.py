"""Full-size parity, byte for byte against the oracle: the plain-sort
configuration at its own sizes (2^28 keys of 1/2/4-byte types, 2^27 of 8-byte
types; every dtype x distribution x direction, 116 runs) and the float
edge-case stress at 2^26 (both float widths, both directions), sorted by the
call the benchmark times.

The expected output of each input is the oracle's own (``oracle_expected``:
the oracle over the pieces that Alg. 2's first partitions make independent).
Inputs with the same multiset share it: "sorted" is the uniform input sorted
ascending under the paper's order (the oracle's output, so floats are in the
paper's order, NaNs at both ends) and "reverse" is it sorted descending.  The
descending expectation is the exact reverse of the ascending one (reading R7:
equal keys are bit-identical, so the descending order is unique)."""
import numpy as np
import pytest

import workloads as W
from gpu_util import assert_bit_exact, oracle_expected

pytestmark = pytest.mark.gpu

NARROW = ["uint8", "int8", "uint16", "int16", "float16", "uint32", "int32", "float32"]
WIDE = ["uint64", "int64", "float64"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2603_08929_gb300 import build as b
    b.build()
    torch.cuda.set_device(0)


def full_n(dtype):
    return 1 << 27 if dtype in WIDE else 1 << 28


_cache = {}


def input_and_expected(dtype, dist, n):
    """(input, oracle's ascending output) of one run, computed once per
    (dtype, multiset): uniform, sorted and reverse share the uniform data."""
    family = "uniform" if dist in ("uniform", "sorted", "reverse") else dist
    key = (dtype, family, n)
    if key not in _cache:
        _cache.clear()
        x = W.make(family, dtype, n, seed=0)
        _cache[key] = (x, oracle_expected(x, False))
    x, asc = _cache[key]
    if dist == "sorted":
        return asc, asc
    if dist == "reverse":
        return asc[::-1].copy(), asc
    return x, asc


def sort_like_bench(x, descending):
    """bsort_keys_ws with an explicit workspace on the current stream (the
    benchmark's call)."""
    import torch
    import paper_2603_08929_gb300 as bs
    t = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    ws = torch.empty(bs.workspace_bytes(t.numel(), x.dtype.name), dtype=torch.uint8, device=t.device)
    h = bs.Handle()
    bs.bsort_keys_ws(h, t, ws, descending=descending, stream=torch.cuda.current_stream())
    assert h.get_error() == 0
    out = t.cpu().numpy()
    del t, ws
    return out


def check_run(dtype, dist, desc, n):
    x, asc = input_and_expected(dtype, dist, n)
    got = sort_like_bench(x, desc)
    assert_bit_exact(got, asc[::-1] if desc else asc, "%s %s %s" % (dtype, dist, "desc" if desc else "asc"))


def _dists(dtype):
    d = ["uniform", "sorted", "reverse", "zipf", "distinct8"]
    return d + ["normal"] if dtype.startswith("float") else d


# every dtype x distribution x direction of the configuration (8 integer
# dtypes x 5 distributions + 3 float dtypes x 6, both directions: 116 runs),
# runs that share a multiset adjacent so its oracle output is computed once
CASES = [(dt, dist, desc) for dt in NARROW + WIDE for dist in _dists(dt) for desc in (False, True)]
assert len(CASES) == 116


@pytest.mark.parametrize("dtype,dist,desc", CASES, ids=["%s-%s-%s" % (d, s, "desc" if r else "asc")
                                                        for d, s, r in CASES])
def test_full_size(dtype, dist, desc):
    check_run(dtype, dist, desc, full_n(dtype))


@pytest.mark.parametrize("desc", [False, True], ids=["asc", "desc"])
@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_float_edge_full_size(dtype, desc):
    check_run(dtype, "float_edge", desc, 1 << 26)
