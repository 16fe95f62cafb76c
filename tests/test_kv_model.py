"""Host model of the value-carrying key-value sort (no GPU).

The device ranks a tile stably: items sit warp-striped (item j of lane l of
warp w is tile position (w * IT + j) * 32 + l); a warp takes its items in
order, the lanes of one digit find each other (peer mask) and the lowest one
advances the warp's counter of that digit; then the digit totals are scanned
and each warp's counter becomes its start inside the digit.  A chunk's tiles
are ranked in order, each digit's destination moving on by the tile's count.
The finish sorts a unit by stable passes of at most 8 bits over its varying
bits, least significant first, the width split evenly.  Here the same
protocol runs in plain Python / numpy and must give exactly the stable
order: per tile, per chunk, and for whole MSD + finish sorts against the
oracle's stable argsort.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

UINT = {1: np.uint8, 2: np.uint16, 4: np.uint32, 8: np.uint64}


def code(x: np.ndarray, fmt: O.KeyFormat, descending: bool) -> np.ndarray:
    """The order code of Sec. III restated (not the library's): the sign bit
    inverted for signed keys, every bit of a negative float inverted, the sign
    bit of a non-negative float set; descending inverts all bits.  Also the
    32-bit word a 1- or 2-byte key is widened to before a key-value sort."""
    w = fmt.w
    u = x.view(UINT[w // 8]).astype(np.uint64)
    sign = np.uint64(1) << np.uint64(w - 1)
    full = np.uint64((1 << w) - 1) if w < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    if fmt.kind == O.SIGNED:
        k = u ^ sign
    elif fmt.kind == O.FLOAT:
        k = np.where(u & sign, u ^ full, u ^ sign)
    else:
        k = u
    return k ^ full if descending else k


def model_places(digits: np.ndarray, n_valid: int, warps: int, it: int) -> np.ndarray:
    """Places of a tile's valid items by the warp-striped peer-group protocol.
    digits[p] is the digit of tile position p (p < n_valid)."""
    nd = int(digits[:n_valid].max()) + 1 if n_valid else 1
    wc = np.zeros((nd, warps), dtype=np.int64)
    place = np.full(n_valid, -1, dtype=np.int64)
    for w in range(warps):
        for j in range(it):
            lanes = [(w * it + j) * 32 + l for l in range(32)]
            valid = [p for p in lanes if p < n_valid]
            groups = {}
            for p in valid:  # lanes in order: the peer mask's bits
                groups.setdefault(int(digits[p]), []).append(p)
            for d, members in groups.items():
                before = wc[d, w]
                for r, p in enumerate(members):  # rank = lower lanes of the group
                    place[p] = before + r
                wc[d, w] = before + len(members)  # the lowest lane advances the counter
    # digit totals, exclusive prefix over digits, then each warp's start
    totals = wc.sum(axis=1)
    start = np.concatenate([[0], np.cumsum(totals)[:-1]])
    warp_start = start[:, None] + np.concatenate([np.zeros((nd, 1), dtype=np.int64),
                                                  np.cumsum(wc, axis=1)[:, :-1]], axis=1)
    for p in range(n_valid):
        w = (p // 32) // it
        place[p] += warp_start[int(digits[p]), w]
    return place


def stable_places(digits: np.ndarray) -> np.ndarray:
    order = np.argsort(digits, kind="stable")
    place = np.empty_like(order)
    place[order] = np.arange(order.size)
    return place


@pytest.mark.parametrize("warps,it", [(8, 16), (8, 20), (8, 3), (2, 5)])
@pytest.mark.parametrize("dist", ["uniform", "few", "one"])
def test_tile_ranking_is_stable(warps, it, dist):
    rng = np.random.default_rng(warps * 100 + it)
    tile = warps * it * 32
    for n_valid in (tile, tile - 1, tile // 3 + 7, 1):
        if dist == "uniform":
            d = rng.integers(0, 256, n_valid)
        elif dist == "few":
            d = rng.integers(0, 3, n_valid) * 85
        else:
            d = np.full(n_valid, 17)
        assert np.array_equal(model_places(d, n_valid, warps, it), stable_places(d))


def test_chunk_of_tiles_carries_destinations():
    """Tiles of one chunk ranked in order, each digit's destination advanced
    by the tile's count, partition the chunk stably by digit."""
    rng = np.random.default_rng(5)
    warps, it = 4, 2
    tile = warps * it * 32
    n = 3 * tile + 77
    d = rng.integers(0, 16, n)
    counts = np.bincount(d, minlength=16)
    dest = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)  # from the histogram pass
    out = np.full(n, -1, dtype=np.int64)
    for t0 in range(0, n, tile):
        td = d[t0:t0 + tile]
        place = model_places(td, td.size, warps, it)
        tstart = np.concatenate([[0], np.cumsum(np.bincount(td, minlength=16))[:-1]])
        for q, p in enumerate(place):  # staging slot p of digit td[q] -> dest - tile start + p
            out[dest[td[q]] - tstart[td[q]] + p] = t0 + q
        dest += np.bincount(td, minlength=16)
    assert np.array_equal(out, np.argsort(d, kind="stable"))


def lsd_passes(lo: int, hi: int):
    """The finish's pass split of the varying bits [lo, hi): (shift, width)."""
    passes = (hi - lo + 7) // 8
    width = (hi - lo + passes - 1) // passes
    return [(lo + p * width, min(width, hi - lo - p * width)) for p in range(passes)]


@pytest.mark.parametrize("lo,hi", [(0, 1), (0, 8), (0, 9), (3, 19), (0, 16), (5, 64), (0, 64), (63, 64)])
def test_pass_split_covers_the_varying_bits(lo, hi):
    ps = lsd_passes(lo, hi)
    assert all(1 <= w <= 8 for _, w in ps)
    covered = [b for s, w in ps for b in range(s, s + w)]
    assert covered == list(range(lo, hi))


def model_kv_sort(codes: np.ndarray, bits: int, unit_cap: int, warps: int = 2) -> np.ndarray:
    """MSD levels of 8-bit digits with stable tile ranking (one tile per chunk
    here), buckets of at most unit_cap keys finished by stable LSD passes
    over their varying bits; returns the permutation."""
    it = 4
    tile = warps * it * 32
    perm = np.arange(codes.size)

    def finish(idx):
        k = codes[idx]
        a, o = np.bitwise_and.reduce(k), np.bitwise_or.reduce(k)
        diff = int(a ^ o)
        if diff == 0:
            return idx
        lo = (diff & -diff).bit_length() - 1
        hi = diff.bit_length()
        for s, w in lsd_passes(lo, hi):
            dg = ((codes[idx] >> np.uint64(s)) & np.uint64((1 << w) - 1)).astype(np.int64)
            out = np.empty_like(idx)
            # the unit is one tile with ceil(len / threads) items per thread
            place = model_places(dg, dg.size, warps, (idx.size + warps * 32 - 1) // (warps * 32))
            out[place] = idx
            idx = out
        return idx

    def level(idx, h):
        if idx.size <= unit_cap or h <= 0:
            return finish(idx)
        s = max(h - 8, 0)
        dg = ((codes[idx] >> np.uint64(s)) & np.uint64((1 << (h - s)) - 1)).astype(np.int64)
        counts = np.bincount(dg, minlength=1 << (h - s))
        dest = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
        out = np.empty_like(idx)
        for t0 in range(0, idx.size, tile):
            td = dg[t0:t0 + tile]
            place = model_places(td, td.size, warps, it)
            tstart = np.concatenate([[0], np.cumsum(np.bincount(td, minlength=counts.size))[:-1]])
            out[dest[td] - tstart[td] + place] = idx[t0:t0 + tile]
            dest += np.bincount(td, minlength=counts.size)
        res = []
        base = 0
        for c in counts:
            res.append(level(out[base:base + c], s))
            base += c
        return np.concatenate(res) if res else out

    return level(perm, bits)


@pytest.mark.parametrize("dist", ["uniform", "distinct8", "zipf", "sorted"])
@pytest.mark.parametrize("dtype,desc", [("int32", False), ("float32", True), ("uint16", False)])
def test_model_sort_is_the_stable_permutation(dist, dtype, desc):
    n = 3000
    x = W.make(dist, dtype, n, seed=21)
    fmt = O.FORMATS[x.dtype]
    k = code(x, fmt, desc)
    got = model_kv_sort(k, fmt.w, unit_cap=300)
    assert np.array_equal(got, O.stable_argsort(x, desc))


@pytest.mark.parametrize("dtype", ["uint8", "int8", "uint16", "int16", "float16"])
@pytest.mark.parametrize("desc", [False, True])
def test_small_keys_widened_to_order_codes(dtype, desc):
    """1- and 2-byte keys are sorted as their order codes widened to 32-bit
    words: a stable sort of the words (unsigned, ascending) is the oracle's
    stable permutation of the keys, and narrowing the sorted words gives the
    sorted keys."""
    x = W.make("zipf", dtype, 20000, seed=4)
    k = code(x, O.FORMATS[x.dtype], desc).astype(np.uint32)
    p = np.argsort(k, kind="stable")
    assert np.array_equal(p, O.stable_argsort(x, desc))
    assert np.array_equal(k[p], np.sort(k))


def model_wide_finish(codes: np.ndarray, tie_run: int = 16):
    """The finish of a unit of 8-byte keys with many varying bits [lo, hi):
    stable passes over the top 16 of them, then every run of keys still tied
    there sorted by the whole key with a stable insertion sort when it holds
    at most tie_run keys; a longer run sends the unit through the passes of
    the low bits and then the top bits again, from that order.  Returns the
    permutation and whether the long-run path was taken."""
    idx = np.arange(codes.size)
    a, o = np.bitwise_and.reduce(codes), np.bitwise_or.reduce(codes)
    diff = int(a ^ o)
    lo = (diff & -diff).bit_length() - 1
    hi = diff.bit_length()
    top = hi - 16

    def passes(idx, frm, to):
        for s, w in lsd_passes(frm, to):
            dg = ((codes[idx] >> np.uint64(s)) & np.uint64((1 << w) - 1)).astype(np.int64)
            idx = idx[np.argsort(dg, kind="stable")]
        return idx

    idx = passes(idx, top, hi)
    k = codes[idx]
    tops = k >> np.uint64(top)
    starts = np.flatnonzero(np.concatenate([[True], tops[1:] != tops[:-1]]))
    ends = np.concatenate([starts[1:], [k.size]])
    if (ends - starts).max() > tie_run:
        return passes(passes(idx, lo, top), top, hi), True
    idx = idx.copy()
    for s, e in zip(starts, ends):
        for x in range(s + 1, e):  # insertion sort, strict comparison: stable
            y = x
            while y > s and codes[idx[y - 1]] > codes[idx[y]]:
                idx[y - 1], idx[y] = idx[y], idx[y - 1]
                y -= 1
    return idx, False


@pytest.mark.parametrize("high,expect_long", [(1 << 16, False), (4096, False), (256, True), (4, True)])
def test_wide_finish_is_stable(high, expect_long):
    """Keys = random high part above zero bits and a random low part, with
    repeats: few ties in the top 16 varying bits (high = 2^16), short tie
    runs (4096), runs too long for the insertion sort (256: ~8 keys per top
    value, the longest over 16; 4): the finish gives the stable order (ties
    in input order) in every case."""
    rng = np.random.default_rng(high)
    n = 2000
    hi_part = rng.integers(0, high, n).astype(np.uint64)
    x = (hi_part << np.uint64(40)) | rng.integers(0, 1 << 20, n).astype(np.uint64)
    x[rng.integers(0, n, 300)] = x[rng.integers(0, n, 300)]  # exact duplicates
    got, long_path = model_wide_finish(x)
    assert long_path == expect_long
    assert np.array_equal(got, np.argsort(x, kind="stable"))
