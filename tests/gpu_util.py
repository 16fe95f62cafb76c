"""Helpers shared by the GPU parity tests."""
import numpy as np

import oracle as O


def to_device(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x).copy()).cuda()


def gpu_sort(x, descending=False):
    import paper_2603_08929_gb300 as bs
    t = to_device(x)
    bs.bsort_keys(t, descending=descending)
    return t.cpu().numpy()


def assert_bit_exact(got, want, what=""):
    assert got.dtype == want.dtype and got.shape == want.shape, what
    g = got.view(np.uint8).reshape(got.size, -1) if got.size else got.view(np.uint8)
    w = want.view(np.uint8).reshape(want.size, -1) if want.size else want.view(np.uint8)
    if not np.array_equal(g, w):
        bad = np.flatnonzero(np.any(g != w, axis=1))
        raise AssertionError("%s: %d of %d keys differ, first at %s: got %s want %s"
                             % (what, bad.size, got.size, bad[:4], got[bad[:4]], want[bad[:4]]))


def check_full_size(x, got, descending, samples=8, seed=0):
    """Properties that pin a sort at any size: monotone under the definition
    order, the same multiset as the input, and sampled positions holding the
    element of that rank."""
    assert got.size == x.size
    i = O.first_unsorted(got, descending)
    assert i == -1, "out of order at %d: %r %r" % (i, got[i], got[i + 1])
    assert O.multiset_digest(got) == O.multiset_digest(x), "not a permutation of the input"
    fmt = O.FORMATS[x.dtype]
    words = O.to_words(x)
    gw = O.to_words(got)
    rng = np.random.default_rng(seed)
    for p in [0, got.size - 1] + list(rng.integers(0, got.size, samples)):
        less, eq = O.rank(words, int(gw[p]), fmt, descending)
        assert less <= p < less + eq, "position %d holds a key of rank [%d, %d)" % (p, less, less + eq)
