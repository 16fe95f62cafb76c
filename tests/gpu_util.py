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


def _chunks(n, parts):
    step = max(1 << 20, (n + parts - 1) // parts)
    return [(a, min(n, a + step)) for a in range(0, n, step)]


def _pool():
    import os
    from concurrent.futures import ThreadPoolExecutor
    return ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1))


def par_first_unsorted(x, descending):
    """O.first_unsorted over chunks in threads (the oracle's C loops release
    the GIL); chunks overlap by one key so every adjacent pair is checked."""
    with _pool() as ex:
        parts = _chunks(x.size, 64)
        res = list(ex.map(lambda ab: O.first_unsorted(x[ab[0]:min(x.size, ab[1] + 1)], descending), parts))
    for (a, _), r in zip(parts, res):
        if r >= 0:
            return a + r
    return -1


def par_multiset_digest(x):
    """O.multiset_digest of chunks, combined (its sums add mod 2^64, its xor
    xors, its counts add)."""
    with _pool() as ex:
        ds = list(ex.map(lambda ab: O.multiset_digest(x[ab[0]:ab[1]]), _chunks(x.size, 64)))
    m = (1 << 64) - 1
    s1 = sum(d[0] for d in ds) & m
    s2 = sum(d[1] for d in ds) & m
    x3 = 0
    for d in ds:
        x3 ^= d[2]
    return (s1, s2, x3, sum(d[3] for d in ds))


def par_rank(x, value, fmt, descending):
    with _pool() as ex:
        rs = list(ex.map(lambda ab: O.rank(O.to_words(x[ab[0]:ab[1]]), value, fmt, descending),
                         _chunks(x.size, 64)))
    return sum(r[0] for r in rs), sum(r[1] for r in rs)


def check_full_size(x, got, descending, samples=8, seed=0):
    """Properties that pin a sort at any size: monotone under the oracle's
    order and the same multiset as the input (together: the unique sorted
    sequence), plus sampled positions holding the key of that rank."""
    assert got.size == x.size
    i = par_first_unsorted(got, descending)
    assert i == -1, "out of order at %d: %r %r" % (i, got[i], got[i + 1])
    assert par_multiset_digest(got) == par_multiset_digest(x), "not a permutation of the input"
    fmt = O.FORMATS[x.dtype]
    rng = np.random.default_rng(seed)
    for p in [0, got.size - 1] + list(rng.integers(0, got.size, samples)):
        key = int(O.to_words(got[p:p + 1])[0])
        less, eq = par_rank(x, key, fmt, descending)
        assert less <= p < less + eq, "position %d holds a key of rank [%d, %d)" % (p, less, less + eq)
