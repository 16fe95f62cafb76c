"""Host model of the counting path of the shared-memory finish (no GPU).

A unit whose keys vary in at most 16 bits is sorted by one counting pass:
the bits above the low four pick a sub-bucket, sixteen 4-bit counters per
sub-bucket (one 64-bit word, updated as two 32-bit halves) count the low
values, and the value an add returns is the key's arrival rank.  A counter
that would pass 15 sends the unit to the comparison path.  When every
sub-bucket holds fewer than 16 keys, multiplying a word by 0x1111...1 and
shifting left by four turns it into exclusive prefix counts (no nibble can
carry); otherwise the counts below a key's low value are summed per key.
This model runs those steps with the arrivals in random orders and checks:
whenever the counting path is taken the positions are a permutation that
sorts the unit, and every unit with 16 equal keys is sent away.
"""
import numpy as np
import pytest

M64 = (1 << 64) - 1


def counting_finish(keys, rng):
    """Positions by the counting path, or None when a counter overflows."""
    k = np.asarray(keys, dtype=np.uint64)
    a, o = int(np.bitwise_and.reduce(k)), int(np.bitwise_or.reduce(k))
    v = a ^ o
    assert v, "one repeated key is written directly"
    lo = (v & -v).bit_length() - 1
    hi = v.bit_length()
    span = hi - lo
    lbits = min(span, 4)
    sbits = span - lbits
    assert span <= 16 and (1 << sbits) <= 4 * len(k)
    fmask, lmask = (1 << span) - 1, (1 << lbits) - 1
    w32 = [0] * (2 << sbits)
    totals = [0] * (1 << sbits)
    arr = [0] * len(k)
    ovf = False
    for i in rng.permutation(len(k)):  # arrival order: any
        f = (int(k[i]) >> lo) & fmask
        low, sb = f & lmask, f >> lbits
        sh = 4 * (low & 7)
        idx = 2 * sb + (low >> 3)
        old = w32[idx]
        w32[idx] = (old + (1 << sh)) & 0xFFFFFFFF
        totals[sb] += 1
        r = (old >> sh) & 15
        ovf |= r == 15
        arr[i] = r
    if ovf:
        return None
    starts = np.concatenate([[0], np.cumsum(totals)[:-1]])
    small = all(t < 16 for t in totals)
    words = [w32[2 * s] | (w32[2 * s + 1] << 32) for s in range(1 << sbits)]
    if small:
        words = [((w * 0x1111111111111111) & M64) << 4 & M64 for w in words]
    pos = []
    for i in range(len(k)):
        f = (int(k[i]) >> lo) & fmask
        low, sb = f & lmask, f >> lbits
        if small:
            below = (words[sb] >> (4 * low)) & 15
        else:
            below = sum((words[sb] >> (4 * j)) & 15 for j in range(low))
        pos.append(int(starts[sb]) + below + arr[i])
    return np.array(pos)


def _unit(rng, n, span, dup):
    base = int(rng.integers(0, 1 << 16)) << 16
    if dup:
        vals = rng.integers(0, 1 << span, max(1, n // dup))
        return base | rng.choice(vals, n)
    return base | rng.integers(0, 1 << span, n)


@pytest.mark.parametrize("seed", range(30))
def test_counting_positions_sort_the_unit(seed):
    rng = np.random.default_rng(seed)
    taken = sent = 0
    for n, span, dup in [(4096, 16, 0), (300, 10, 0), (5000, 16, 0), (64, 6, 0), (2000, 12, 40), (20, 4, 0),
                         (700, 9, 3), (4096, 14, 0), (33, 5, 0)]:
        keys = _unit(rng, n, span, dup)
        k = np.asarray(keys, dtype=np.uint64)
        v = int(np.bitwise_and.reduce(k)) ^ int(np.bitwise_or.reduce(k))
        if v == 0 or (1 << max(0, v.bit_length() - ((v & -v).bit_length() - 1) - 4)) > 4 * n:
            continue
        pos = counting_finish(keys, rng)
        counts = np.unique(keys, return_counts=True)[1]
        if pos is None:
            assert counts.max() >= 16, "overflow reported without 16 equal keys"
            sent += 1
            continue
        assert counts.max() < 16, "16 equal keys were not sent away"
        assert np.array_equal(np.sort(pos), np.arange(n)), "not a permutation"
        out = np.empty(n, dtype=np.uint64)
        out[pos] = keys
        assert np.all(out[1:] >= out[:-1]), "positions do not sort the unit"
        taken += 1
    assert taken > 0


def test_sixteen_equal_keys_overflow_any_order():
    rng = np.random.default_rng(7)
    keys = np.array([5] * 16 + list(range(6, 40)), dtype=np.uint64) | (1 << 20)
    for _ in range(10):
        assert counting_finish(keys, rng) is None


def test_prefix_multiply_is_exact_below_sixteen():
    """At most 15 keys in a word: w * 0x1111...1 << 4 holds exclusive prefix
    counts in every nibble (no carry between nibbles)."""
    rng = np.random.default_rng(8)
    for _ in range(2000):
        c = rng.multinomial(int(rng.integers(0, 16)), [1 / 16] * 16)
        w = sum(int(x) << (4 * i) for i, x in enumerate(c))
        p = ((w * 0x1111111111111111) & M64) << 4 & M64
        assert [(p >> (4 * i)) & 15 for i in range(16)] == [int(c[:i].sum()) for i in range(16)]
