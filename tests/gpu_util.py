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
    got, want = np.ascontiguousarray(got), np.ascontiguousarray(want)
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


_UT = {1: np.uint8, 2: np.uint16, 4: np.uint32, 8: np.uint64}


def oracle_expected(x, descending=False, fmt=None, split_levels=8):
    """The oracle's sorted output of a large array, computed by the oracle on
    pieces that the method itself makes independent.

    Keys of at most 16 bits: the oracle orders every one of the 2^w patterns
    once, and each pattern is repeated by its count in ``x`` (keys that sort
    equal are bit-identical, so the sorted output is fixed by the counts).

    Wider keys, following Alg. 2's recursion: after its first
    ``split_levels`` bit partitions the array is a sequence of ranges, one per
    pattern of the top ``split_levels`` bits, ordered as the oracle orders
    those patterns, and each range is then sorted on its own.  So ``x`` is cut
    into pieces; the oracle partitions every piece by its first
    ``split_levels`` levels (threads, one piece each); the runs of each top
    pattern are gathered over the pieces; the oracle sorts each gathered range
    completely (threads again); the ranges are concatenated in the order the
    oracle gives the patterns' representatives ``pattern << (w -
    split_levels)``.  Every ordering decision is the oracle's."""
    x = np.ascontiguousarray(x)
    fmt = fmt or O.FORMATS[x.dtype]
    ut = _UT[x.dtype.itemsize]
    if fmt.w <= 16:
        counts = np.bincount(x.view(ut), minlength=1 << fmt.w)
        order = np.arange(1 << fmt.w, dtype=np.uint64)
        O.bsort_words(order, fmt, descending)
        return np.repeat(order.astype(ut), counts[order.astype(np.int64)]).view(x.dtype)
    k = split_levels
    words = x.view(ut).astype(np.uint64)
    pieces = _chunks(words.size, 16)

    def partition(ab):
        a, b = ab
        piece = words[a:b]
        O.bsort_words(piece, fmt, descending, O.LITERAL, max_levels=k)
        top = piece >> np.uint64(fmt.w - k)
        cut = np.flatnonzero(top[1:] != top[:-1]) + 1
        starts = np.concatenate(([0], cut))
        ends = np.concatenate((cut, [piece.size]))
        return [(int(top[s]), a + int(s), a + int(e)) for s, e in zip(starts, ends)]

    with _pool() as ex:
        runs = [r for rs in ex.map(partition, pieces) for r in rs]
    groups = {}
    for pat, a, b in runs:
        groups.setdefault(pat, []).append((a, b))
    reps = np.array(sorted(groups), dtype=np.uint64) << np.uint64(fmt.w - k)
    O.bsort_words(reps, fmt, descending)
    order = [int(r) >> (fmt.w - k) for r in reps]
    bounds = np.cumsum([0] + [sum(b - a for a, b in groups[p]) for p in order])
    out = np.empty_like(words)

    def finish(i):
        dst = out[bounds[i]:bounds[i + 1]]
        o = 0
        for a, b in groups[order[i]]:
            dst[o:o + b - a] = words[a:b]
            o += b - a
        O.bsort_words(dst, fmt, descending)

    with _pool() as ex:
        list(ex.map(finish, sorted(range(len(order)), key=lambda i: bounds[i] - bounds[i + 1])))
    return out.astype(ut).view(x.dtype)


def oracle_segments(x, off, descending=False):
    """The oracle's sort of every segment [off[i], off[i+1]) of x, the
    segments spread over threads (each is independent)."""
    out = x.copy()
    segs = [(int(a), int(b)) for a, b in zip(off[:-1], off[1:]) if b - a > 1]
    segs.sort(key=lambda ab: ab[0] - ab[1])  # largest first

    def one(ab):
        a, b = ab
        out[a:b] = O.bsort(x[a:b], descending=descending)

    with _pool() as ex:
        list(ex.map(one, segs))
    return out


def check_full_size(x, got, descending, samples=8, seed=0, fmt=None):
    """The whole output, byte for byte, against the oracle's sorted output of
    the same input (``oracle_expected``)."""
    assert got.size == x.size
    assert_bit_exact(got, oracle_expected(x, descending, fmt=fmt), "full-size parity")


def check_by_properties(x, got, descending, samples=8, seed=0):
    """Properties that pin a sort at any size, for arrays too large to hold
    the oracle's output beside them: monotone under the oracle's order and the
    same multiset as the input (together: the unique sorted sequence), plus
    sampled positions holding the key of that rank."""
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
