"""bsort_keys_noalloc, the entry point for callers that cannot allocate device
memory (graph capture, pool-owned memory, engines that forbid allocation):
its output must equal bsort_keys' output, call after call, although every call
reuses the same static scratch array.  Kept in its own file, collected last."""
import ctypes

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

CODES = {"int32": 6, "float64": 10, "uint16": 2}


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2603_08929_gb300 import build as b
    b.build()
    import paper_2603_08929_gb300 as bs
    torch.cuda.set_device(0)
    return bs.lib()


def _sort_both(lib, x, desc):
    import torch
    a = torch.from_numpy(x.copy()).cuda()
    b = a.clone()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = CODES[x.dtype.name]
    assert lib.bsort_keys(ctypes.c_void_p(a.data_ptr()), a.numel(), code, int(desc), stream) == 0
    assert lib.bsort_keys_noalloc(ctypes.c_void_p(b.data_ptr()), b.numel(), code, int(desc), stream) == 0
    torch.cuda.synchronize()
    return a.cpu().numpy(), b.cpu().numpy()


def test_noalloc_matches_bsort_keys_two_calls_in_a_row(lib):
    # two calls in a row: the second finds the first one's scratch in the array
    for x, desc in ((W.make("uniform", "int32", (1 << 20) + 77, seed=21), False),
                    (W.make("float_edge", "float64", 300001, seed=22), True),
                    (W.make("zipf", "uint16", 500000, seed=23), False)):
        want, got = _sort_both(lib, x, desc)
        assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), x.dtype
        # and both are the sort the paper defines
        assert np.array_equal(got.view(np.uint8), O.bsort(x, descending=desc).view(np.uint8)), x.dtype


def _largest_n(dtype, cap=64 << 20):
    """Largest n whose workspace fits the library's 64 MiB static array."""
    import paper_2603_08929_gb300 as bs
    lo, hi = 0, 1 << 34
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if bs.workspace_bytes(mid, dtype) <= cap:
            lo = mid
        else:
            hi = mid - 1
    return lo


def test_noalloc_rejects_n_beyond_the_array(lib):
    import torch
    n = _largest_n("int32") + 1  # one more 4-byte key than the array serves
    t = torch.zeros(n, dtype=torch.int32, device="cuda")
    t[0] = 5
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.bsort_keys_noalloc(ctypes.c_void_p(t.data_ptr()), n, 6, 0, stream) == 5  # WORKSPACE_TOO_SMALL
    assert int(t[0]) == 5  # untouched
    assert lib.bsort_keys_noalloc(ctypes.c_void_p(t.data_ptr()), n - 1, 6, 0, stream) == 0
    torch.cuda.synchronize()
    assert int(t[n - 2]) == 5 and int(t[0]) == 0 and int(t[n - 1]) == 0
