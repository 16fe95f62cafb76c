"""Pins of the CPU oracle against facts fixed by the paper and by arithmetic.

Each ``pin_*`` function raises ``AssertionError`` if the oracle disagrees with
what it pins.  ``tests/test_oracle.py`` runs them one by one; the planted-
mistake test runs all of them against oracle builds with a deliberate bug and
requires each bug to trip at least one pin.
"""
from __future__ import annotations

import functools
import itertools
import os
import random
from fractions import Fraction

import numpy as np

import oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

_KIND = {"unsigned": O.UNSIGNED, "signed": O.SIGNED, "float": O.FLOAT}


def load_trace(name):
    """(format, ascending, rows) of a golden trace file."""
    fmt = asc = None
    rows = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("w="):
                kv = dict(p.split("=") for p in line.split())
                fmt = O.KeyFormat(int(kv["w"]), _KIND[kv["kind"]], int(kv["e"]), int(kv["f"]))
                asc = kv["asc"] == "1"
                continue
            lvl, vals = line.split(":")
            toks = vals.split()
            if fmt.kind == O.FLOAT:
                words = [int(t, 2) for t in toks]
            else:
                words = [int(t) & ((1 << fmt.w) - 1) for t in toks]
            rows[int(lvl)] = words
    return fmt, asc, rows


def _run_levels(words, fmt, asc, mode, levels, **kw):
    """State after ``levels`` bit levels; None = untouched input, 0 = full sort."""
    a = np.array(words, dtype=np.uint64)
    if levels is not None:
        v, _ = O.bsort_words(a, fmt, not asc, mode, levels, check=True, **kw)
        assert v == 0, "invariant violations: %d" % v
    return a.tolist()


def _check_trace(name):
    fmt, asc, rows = load_trace(name)
    last = max(rows)
    for lvl, row in rows.items():
        got = _run_levels(rows[0], fmt, asc, O.STABLE, lvl if lvl else None)
        assert got == row, "%s level %d: %s != %s" % (name, lvl, got, row)
    # the literal (swapping) partition reaches the same final row
    got = _run_levels(rows[0], fmt, asc, O.LITERAL, 0)
    assert got == rows[last], "%s literal final: %s" % (name, got)
    got = np.array(rows[0], dtype=np.uint64)
    O.sort_words_by_definition(got, fmt, not asc)
    assert got.tolist() == rows[last], "%s definition order: %s" % (name, got.tolist())


def pin_fig1_trace():
    """Fig. 1: every row of the unsigned 3-bit trace."""
    _check_trace("fig1_unsigned_trace.txt")


def pin_fig2_trace():
    """Fig. 2: every row of the signed 4-bit descending trace (Alg. 3)."""
    _check_trace("fig2_signed_trace.txt")


def pin_fig4_trace():
    """Fig. 4: every row of the 6-bit minifloat trace (Algs. 4/5)."""
    _check_trace("fig4_minifloat_trace.txt")


def pin_fig4_printed_alg4_is_wrong():
    """Alg. 4 as printed (both halves ascending) misorders Fig. 4's negatives."""
    fmt, asc, rows = load_trace("fig4_minifloat_trace.txt")
    got = _run_levels(rows[0], fmt, asc, O.STABLE, 0, literal_alg4=True)
    assert got != rows[max(rows)], "printed Alg. 4 unexpectedly matches Fig. 4"


def pin_theorem2_counterexamples():
    """Thm. 2's arrays sort to numeric order in both float widths."""
    for dt in (np.float32, np.float64, np.float16):
        for arr in ([-2.0, 0.0, 0.5], [0.75, 2.0], [2.0, 0.75], [0.5, 0.0, -2.0]):
            x = np.array(arr, dtype=dt)
            got = O.bsort(x)
            assert got.tolist() == sorted(arr), (dt, arr, got)
            got = O.bsort(x, descending=True)
            assert got.tolist() == sorted(arr, reverse=True), (dt, arr, got)


# --- an independent Python restatement of the order, with exact rationals ---

def py_order_key(word: int, fmt: O.KeyFormat):
    """Sort key of one pattern under the paper's order (exact arithmetic)."""
    w = fmt.w
    if fmt.kind == O.UNSIGNED:
        return (word,)
    if fmt.kind == O.SIGNED:
        return (word - (1 << w) if word >> (w - 1) else word,)
    s = word >> (w - 1)
    e = (word >> fmt.f) & ((1 << fmt.e) - 1)
    m = word & ((1 << fmt.f) - 1)
    bias = (1 << (fmt.e - 1)) - 1
    if e == (1 << fmt.e) - 1:
        if m:
            return (0, -m) if s else (4, m)          # NaNs at both ends
        return (1,) if s else (3,)                   # -inf, +inf
    if e == 0:
        mag = Fraction(m) * Fraction(2) ** (1 - bias - fmt.f)
    else:
        mag = Fraction((1 << fmt.f) + m) * Fraction(2) ** (e - bias - fmt.f)
    return (2, -mag if s else mag, 0 if s else 1)   # -0 before +0


def pin_bruteforce_tiny():
    """All permutations of tiny inputs: the unique ordered one is the oracle's."""
    rnd = random.Random(1234)
    fmts = [O.KeyFormat(3, O.UNSIGNED), O.KeyFormat(4, O.SIGNED), O.KeyFormat(5, O.UNSIGNED),
            O.KeyFormat(6, O.SIGNED), O.KeyFormat(6, O.FLOAT, 3, 2), O.KeyFormat(5, O.FLOAT, 2, 2),
            O.KeyFormat(4, O.FLOAT, 2, 1)]
    for fmt in fmts:
        for trial in range(40):
            n = rnd.randint(0, 6)
            xs = [rnd.randrange(1 << fmt.w) for _ in range(n)]
            for asc in (True, False):
                want = None
                for p in itertools.permutations(xs):
                    ks = [py_order_key(v, fmt) for v in p]
                    ok = all((ks[i] <= ks[i + 1]) if asc else (ks[i] >= ks[i + 1])
                             for i in range(len(ks) - 1))
                    if ok:
                        if want is None:
                            want = list(p)
                        assert list(p) == want, "two different ordered permutations"
                want = want if want is not None else []
                for mode in (O.LITERAL, O.STABLE):
                    a = np.array(xs, dtype=np.uint64)
                    v, _ = O.bsort_words(a, fmt, not asc, mode, check=True)
                    assert v == 0
                    assert a.tolist() == want, (fmt, xs, asc, mode, a.tolist(), want)
                a = np.array(xs, dtype=np.uint64)
                O.sort_words_by_definition(a, fmt, not asc)
                assert a.tolist() == want, (fmt, xs, asc, "definition", a.tolist(), want)


def _special_float_sequence(dtype):
    """Patterns in ascending order, from the paper's special-value rules."""
    w = np.dtype(dtype).itemsize * 8
    f = {16: 10, 32: 23, 64: 52}[w]
    e = w - 1 - f
    S = 1 << (w - 1)
    E = ((1 << e) - 1) << f
    Q = 1 << (f - 1)
    M = (1 << f) - 1
    one = ((1 << (e - 1)) - 1) << f
    pos = [0, 1, M, 1 << f, one, E - 1, E, E | 1, E | (Q - 1), E | Q, E | M]
    neg = [S | p for p in reversed(pos)]
    return neg + pos


def pin_special_values():
    """-NaNs < -inf < negatives < -0 < +0 < positives < +inf < +NaNs (Sec. III-C)."""
    rnd = random.Random(7)
    for dt in (np.float16, np.float32, np.float64):
        fmt = O.FORMATS[np.dtype(dt)]
        seq = _special_float_sequence(dt)
        for i in range(len(seq) - 1):
            assert py_order_key(seq[i], fmt) < py_order_key(seq[i + 1], fmt)
        for trial in range(5):
            sh = seq[:]
            rnd.shuffle(sh)
            for desc in (False, True):
                want = list(reversed(seq)) if desc else seq
                a = np.array(sh, dtype=np.uint64)
                O.bsort_words(a, fmt, desc, O.LITERAL)
                assert a.tolist() == want, (dt, desc, "bsort")
                a = np.array(sh, dtype=np.uint64)
                O.sort_words_by_definition(a, fmt, desc)
                assert a.tolist() == want, (dt, desc, "definition")


def pin_float_values_match_numpy():
    """The comparator's value of every finite fp16 pattern, and random fp32 /
    fp64 patterns, equals numpy's conversion of the same bits."""
    fmt = O.FORMATS[np.dtype(np.float16)]
    allv = np.arange(1 << 16, dtype=np.uint16)
    fin = allv[np.isfinite(allv.view(np.float16))]
    ref = fin.view(np.float16).astype(np.float64)
    for i in range(0, fin.size, 97):
        assert O.float_value(int(fin[i]), fmt) == ref[i], hex(int(fin[i]))
    for i in list(range(0, 64)) + list(range(1024, 1100)):  # subnormals, smallest normals
        assert O.float_value(int(fin[i]), fmt) == ref[i], hex(int(fin[i]))
    rng = np.random.default_rng(5)
    for dt, ut in ((np.float32, np.uint32), (np.float64, np.uint64)):
        fmt = O.FORMATS[np.dtype(dt)]
        bits = rng.integers(0, np.iinfo(ut).max, size=4000, dtype=ut, endpoint=True)
        bits[:8] = [0, 1, 2, 3, 5, 7, 9, 11]  # subnormals
        vals = bits.view(dt)
        for b, v in zip(bits, vals):
            if np.isfinite(v):
                assert O.float_value(int(b), fmt) == float(v), hex(int(b))


def pin_exhaustive_small_words():
    """Every 8- and 16-bit pattern, shuffled: integers match numpy's sort,
    floats match the definition sort and numpy on their non-NaN part, and
    descending is the exact reverse of ascending."""
    rng = np.random.default_rng(11)
    for dt in (np.uint8, np.int8, np.uint16, np.int16, np.float16):
        w = np.dtype(dt).itemsize * 8
        ut = np.uint8 if w == 8 else np.uint16
        x = rng.permutation(np.arange(1 << w, dtype=np.uint64).astype(ut)).view(dt)
        asc = O.bsort(x)
        desc = O.bsort(x, descending=True)
        assert np.array_equal(desc.view(ut), asc.view(ut)[::-1])
        assert np.array_equal(asc.view(ut), O.sort_by_definition(x).view(ut))
        if np.dtype(dt).kind in "iu":
            assert np.array_equal(asc, np.sort(x))
        else:
            vals = asc[~np.isnan(asc)]
            assert np.all(vals[:-1] <= vals[1:])
            n_neg_nan = int(np.sum(np.isnan(asc) & np.signbit(asc)))
            assert np.all(np.isnan(asc[:n_neg_nan])) and np.all(np.signbit(asc[:n_neg_nan]))
            z = np.flatnonzero(asc.view(ut) == 0)[0]
            assert asc.view(ut)[z - 1] == 0x8000  # -0 right before +0


def pin_random_vs_numpy_and_definition():
    """Random arrays of every machine type: the bit partition equals the
    definition sort; integers also equal numpy's sort; NaN-free floats have
    numpy's numeric order."""
    rng = np.random.default_rng(3)
    for dt in O.FORMATS:
        w = dt.itemsize * 8
        ut = {8: np.uint8, 16: np.uint16, 32: np.uint32, 64: np.uint64}[w]
        bits = rng.integers(0, np.iinfo(ut).max, size=3000, dtype=ut, endpoint=True)
        x = bits.view(dt)
        for desc in (False, True):
            got = O.bsort(x, descending=desc)
            want = O.sort_by_definition(x, descending=desc)
            assert np.array_equal(got.view(ut), want.view(ut)), (dt, desc)
            if dt.kind in "iu":
                ns = np.sort(x)
                assert np.array_equal(got, ns[::-1] if desc else ns), (dt, desc)
            else:
                clean = x[np.isfinite(x) & (x != 0)]
                g = O.bsort(clean, descending=desc)
                ns = np.sort(clean)
                assert np.array_equal(g, ns[::-1] if desc else ns), (dt, desc)


def pin_invariants_every_partition():
    """Invariants (i)/(ii) of Sec. II hold after every partition, both modes."""
    rng = np.random.default_rng(9)
    for dt in O.FORMATS:
        w = dt.itemsize * 8
        ut = {8: np.uint8, 16: np.uint16, 32: np.uint32, 64: np.uint64}[w]
        x = rng.integers(0, np.iinfo(ut).max, size=1500, dtype=ut, endpoint=True).view(dt)
        for mode in (O.LITERAL, O.STABLE):
            for desc in (False, True):
                words = O.to_words(x)
                v, parts = O.bsort_words(words, O.FORMATS[dt], desc, mode, check=True)
                assert v == 0 and parts > 0


def pin_at_most_w_levels():
    """Thm. 4: w bit levels sort fully; limiting to w levels changes nothing."""
    rng = np.random.default_rng(4)
    for dt in O.FORMATS:
        w = dt.itemsize * 8
        ut = {8: np.uint8, 16: np.uint16, 32: np.uint32, 64: np.uint64}[w]
        x = rng.integers(0, np.iinfo(ut).max, size=800, dtype=ut, endpoint=True).view(dt)
        full = O.bsort(x, mode=O.STABLE)
        lim = O.bsort(x, mode=O.STABLE, max_levels=w)
        assert np.array_equal(full.view(ut), lim.view(ut))


def pin_idempotent_and_modes_agree():
    rng = np.random.default_rng(6)
    for dt in O.FORMATS:
        w = dt.itemsize * 8
        ut = {8: np.uint8, 16: np.uint16, 32: np.uint32, 64: np.uint64}[w]
        x = rng.integers(0, np.iinfo(ut).max, size=1000, dtype=ut, endpoint=True).view(dt)
        a = O.bsort(x)
        assert np.array_equal(O.bsort(a).view(ut), a.view(ut))
        assert np.array_equal(O.bsort(x, mode=O.STABLE).view(ut), a.view(ut))


# --- bfloat16 ------------------------------------------------------------------

def pin_bf16_values_are_binary32_high_halves():
    """Every finite bfloat16 pattern's value, by the oracle's comparator
    arithmetic, is the binary32 value of the pattern shifted into the high
    half (numpy's conversion, exact)."""
    b = np.arange(1 << 16, dtype=np.uint32)
    f32 = (b << 16).view(np.float32)
    for bits in b[((b >> 7) & 0xFF) != 0xFF].tolist():
        assert O.float_value(bits, O.BF16) == float(f32[bits]), hex(bits)


def pin_bf16_exhaustive_order():
    """All 2^16 bfloat16 patterns: the oracle's sort (both modes, both
    directions) equals the exact-rational restatement's order, and on the
    non-NaN patterns numpy's numeric order of the binary32 values with -0
    before +0."""
    words = np.arange(1 << 16, dtype=np.uint64)
    want = sorted(words.tolist(), key=lambda v: py_order_key(v, O.BF16))
    for mode in (O.LITERAL, O.STABLE):
        a = words[::-1].copy()
        O.bsort_words(a, O.BF16, False, mode)
        assert a.tolist() == want
        d = words.copy()
        O.bsort_words(d, O.BF16, True, mode)
        assert d.tolist() == want[::-1]
    nonnan = [v for v in want if not (((v >> 7) & 0xFF) == 0xFF and (v & 0x7F))]
    f = (np.array(nonnan, dtype=np.uint32) << 16).view(np.float32)
    assert np.all(f[1:] >= f[:-1])
    sign = np.array(nonnan, dtype=np.uint32) >> 15
    zeros = np.flatnonzero(f == 0)
    assert sign[zeros].tolist() == [1, 0]


# --- key-value sorting: the stable permutation -------------------------------

def _py_stable_perm(xs, fmt, asc):
    """Stable order of positions by py_order_key (the exact-rational
    restatement), equal keys by position."""
    keys = [py_order_key(v, fmt) for v in xs]

    def cmp(i, j):
        if keys[i] != keys[j]:
            return (-1 if keys[i] < keys[j] else 1) * (1 if asc else -1)
        return (i > j) - (i < j)
    return sorted(range(len(xs)), key=functools.cmp_to_key(cmp))


def pin_stable_argsort_tiny():
    """Tiny inputs full of ties in every kind of format: the oracle's stable
    permutation equals the independent restatement's."""
    rnd = random.Random(4321)
    fmts = [O.KeyFormat(3, O.UNSIGNED), O.KeyFormat(4, O.SIGNED), O.KeyFormat(6, O.SIGNED),
            O.KeyFormat(6, O.FLOAT, 3, 2), O.KeyFormat(5, O.FLOAT, 2, 2), O.KeyFormat(8, O.FLOAT, 4, 3)]
    for fmt in fmts:
        for trial in range(60):
            n = rnd.randint(0, 12)
            pool = [rnd.randrange(1 << fmt.w) for _ in range(rnd.randint(1, 4))]
            xs = [rnd.choice(pool) if rnd.random() < 0.7 else rnd.randrange(1 << fmt.w) for _ in range(n)]
            for asc in (True, False):
                got = O.stable_argsort_words(np.array(xs, dtype=np.uint64), fmt, not asc).tolist()
                assert got == _py_stable_perm(xs, fmt, asc), (fmt, xs, asc, got)


def pin_stable_argsort_machine_types():
    """Every machine type, many ties: the permutation is one, the keys it
    gathers are the (pinned) sorted keys, and identical keys keep their input
    order."""
    rng = np.random.default_rng(9)
    for dt in O.FORMATS:
        ut = {8: np.uint8, 16: np.uint16, 32: np.uint32, 64: np.uint64}[dt.itemsize * 8]
        pool = rng.integers(0, np.iinfo(ut).max, size=24, dtype=ut, endpoint=True)
        x = np.where(rng.random(5000) < 0.8, rng.choice(pool, 5000),
                     rng.integers(0, np.iinfo(ut).max, size=5000, dtype=ut, endpoint=True)).astype(ut).view(dt)
        for desc in (False, True):
            p = O.stable_argsort(x, desc)
            assert np.array_equal(np.sort(p), np.arange(x.size))
            assert np.array_equal(x[p].view(ut), O.bsort(x, desc).view(ut)), dt
            w = O.to_words(x)[p]
            same = w[1:] == w[:-1]
            assert np.all(p[1:][same] > p[:-1][same]), "ties out of input order (%s)" % dt


# --- the checkers behind the full-size parity tests ---------------------------
#
# first_unsorted, rank and multiset_digest certify GPU outputs too large to
# compare with a full oracle run inside one test; each is pinned here against
# a brute-force restatement (py_order_key) or against the arithmetic fact it
# relies on, and each has planted mistakes that these pins must catch.

_SMALL_FMTS = [O.KeyFormat(3, O.UNSIGNED), O.KeyFormat(4, O.SIGNED), O.KeyFormat(6, O.SIGNED),
               O.KeyFormat(6, O.FLOAT, 3, 2), O.KeyFormat(5, O.FLOAT, 2, 2), O.KeyFormat(8, O.FLOAT, 4, 3)]


def _py_first_unsorted(xs, fmt, asc):
    ks = [py_order_key(v, fmt) for v in xs]
    for i in range(len(ks) - 1):
        if (ks[i] > ks[i + 1]) if asc else (ks[i] < ks[i + 1]):
            return i
    return -1


def pin_first_unsorted_bruteforce():
    """first_unsorted equals the first adjacent pair out of order under the
    exact-rational restatement: random tie-heavy arrays, their sorted forms
    (answer -1, ties included) and sorted forms with one planted inversion at
    the front, the back and in between."""
    rnd = random.Random(2468)
    for fmt in _SMALL_FMTS:
        for trial in range(80):
            n = rnd.randint(0, 10)
            pool = [rnd.randrange(1 << fmt.w) for _ in range(rnd.randint(1, 4))]
            xs = [rnd.choice(pool) if rnd.random() < 0.6 else rnd.randrange(1 << fmt.w) for _ in range(n)]
            for asc in (True, False):
                ordered = sorted(xs, key=lambda v: py_order_key(v, fmt), reverse=not asc)
                cases = [xs, ordered]
                for i in (0, n - 2, n // 2 - 1):
                    if 0 <= i < n - 1 and py_order_key(ordered[i], fmt) != py_order_key(ordered[i + 1], fmt):
                        bad = list(ordered)
                        bad[i], bad[i + 1] = bad[i + 1], bad[i]
                        cases.append(bad)
                for c in cases:
                    got = O.first_unsorted_words(np.array(c, dtype=np.uint64), fmt, not asc)
                    assert got == _py_first_unsorted(c, fmt, asc), (fmt, c, asc, got)
                assert O.first_unsorted_words(np.array(ordered, dtype=np.uint64), fmt, not asc) == -1


def pin_first_unsorted_machine_types():
    """On every machine type a sorted output reads as sorted, and one adjacent
    swap of distinct keys is found at exactly its index (first pair, last pair,
    middle); for floats also -0/+0 and two same-sign NaN payloads swapped."""
    rng = np.random.default_rng(13)
    for dt in O.FORMATS:
        ut = {8: np.uint8, 16: np.uint16, 32: np.uint32, 64: np.uint64}[dt.itemsize * 8]
        x = rng.integers(0, np.iinfo(ut).max, size=3000, dtype=ut, endpoint=True).view(dt)
        x[:40] = x[40:80]  # ties
        for desc in (False, True):
            s = O.bsort(x, descending=desc)
            assert O.first_unsorted(s, desc) == -1, dt
            sw = s.view(ut)
            for i in (0, s.size - 2, s.size // 2):
                j = i
                while sw[j] == sw[j + 1]:  # nearest distinct pair (back from the end)
                    j += 1 if i < s.size - 2 else -1
                bad = s.copy()
                bad[[j, j + 1]] = bad[[j + 1, j]]
                assert O.first_unsorted(bad, desc) == j, (dt, desc, j)
        if dt.kind == "f":
            w = dt.itemsize * 8
            f = {16: 10, 32: 23, 64: 52}[w]
            S, E = 1 << (w - 1), ((1 << (w - 1 - f)) - 1) << f
            pairs = [(S, 0), (E | 1, E | (1 << (f - 1))), (S | E | (1 << (f - 1)), S | E | 1)]
            for lo_hi in pairs:
                for desc in (False, True):
                    a = np.array(lo_hi if not desc else lo_hi[::-1], dtype=np.uint64)
                    fmt = O.FORMATS[dt]
                    assert O.first_unsorted_words(a, fmt, desc) == -1, (dt, lo_hi, desc)
                    assert O.first_unsorted_words(a[::-1].copy(), fmt, desc) == 0, (dt, lo_hi, desc)


def pin_rank_bruteforce():
    """rank(a, x) = (keys strictly before x, keys bit-identical to x) by a
    brute count under the exact-rational restatement, for every pattern x of
    small formats against tie-heavy arrays, both directions."""
    rnd = random.Random(1357)
    for fmt in _SMALL_FMTS:
        for trial in range(12):
            n = rnd.randint(0, 24)
            pool = [rnd.randrange(1 << fmt.w) for _ in range(3)]
            xs = [rnd.choice(pool) if rnd.random() < 0.5 else rnd.randrange(1 << fmt.w) for _ in range(n)]
            a = np.array(xs, dtype=np.uint64)
            for x in range(1 << fmt.w):
                kx = py_order_key(x, fmt)
                for asc in (True, False):
                    less = sum(1 for v in xs if v != x and ((py_order_key(v, fmt) < kx) if asc
                                                            else (py_order_key(v, fmt) > kx)))
                    eq = xs.count(x)
                    assert O.rank(a, x, fmt, not asc) == (less, eq), (fmt, xs, x, asc)


def pin_rank_places_sorted_keys():
    """Machine types: the key at every position p of the oracle's sort has
    rank [less, less + equal) containing p."""
    rng = np.random.default_rng(17)
    for dt in O.FORMATS:
        ut = {8: np.uint8, 16: np.uint16, 32: np.uint32, 64: np.uint64}[dt.itemsize * 8]
        pool = rng.integers(0, np.iinfo(ut).max, size=5, dtype=ut, endpoint=True)
        x = np.where(rng.random(400) < 0.5, rng.choice(pool, 400),
                     rng.integers(0, np.iinfo(ut).max, size=400, dtype=ut, endpoint=True)).astype(ut).view(dt)
        words = O.to_words(x)
        for desc in (False, True):
            s = O.to_words(O.bsort(x, descending=desc))
            for p in range(0, s.size, 7):
                less, eq = O.rank(words, int(s[p]), O.FORMATS[dt], desc)
                assert less <= p < less + eq, (dt, desc, p)


def pin_multiset_digest():
    """The digest is a function of the multiset: equal under any
    permutation; different after one bit of one element flips (every bit of
    the first, last and a middle element), after an element is replaced by a
    copy of another (count unchanged), after one is dropped or duplicated, and
    for {+0, +0} against {+0, -0}."""
    rng = np.random.default_rng(19)
    for dt in (np.uint8, np.int16, np.float16, np.uint32, np.float32, np.int64, np.float64):
        dt = np.dtype(dt)
        w = dt.itemsize * 8
        ut = {8: np.uint8, 16: np.uint16, 32: np.uint32, 64: np.uint64}[w]
        x = rng.integers(0, np.iinfo(ut).max, size=257, dtype=ut, endpoint=True)
        x[5] = x[6]
        words = x.astype(np.uint64)
        d0 = O.multiset_digest_words(words)
        assert d0[3] == x.size
        for trial in range(4):
            assert O.multiset_digest_words(rng.permutation(words)) == d0
        for i in (0, x.size - 1, x.size // 2):
            for b in range(w):
                y = words.copy()
                y[i] ^= np.uint64(1) << np.uint64(b)
                assert O.multiset_digest_words(y) != d0, (dt, i, b)
        y = words.copy()
        y[0] = y[1]
        assert O.multiset_digest_words(y) != d0
        y = words.copy()
        y[-1] = y[0]
        assert O.multiset_digest_words(y) != d0
        assert O.multiset_digest_words(words[1:]) != d0
        assert O.multiset_digest_words(np.append(words, words[3])) != d0
    z = np.array([0, 0], dtype=np.uint64)
    for w in (16, 32, 64):
        mz = np.array([0, 1 << (w - 1)], dtype=np.uint64)
        assert O.multiset_digest_words(z) != O.multiset_digest_words(mz)


def pin_parallel_checkers_combine():
    """The chunked checkers of the GPU tests (threads over 64 chunks) agree
    with one plain call on arrays spanning several chunks, and an inversion
    straddling a chunk boundary is found at its index."""
    import gpu_util as G
    rng = np.random.default_rng(23)
    n = 3 * (1 << 20) + 777
    x = rng.integers(-(1 << 31), (1 << 31) - 1, size=n, dtype=np.int64).astype(np.int32)
    assert G.par_multiset_digest(x) == O.multiset_digest(x)
    s = O.bsort(x)
    assert G.par_first_unsorted(s, False) == -1
    for i in ((1 << 20) - 1, 2 * (1 << 20) - 1, n - 2, 0):
        j = i
        while s[j] == s[j + 1]:
            j += 1 if i < n - 2 else -1
        bad = s.copy()
        bad[[j, j + 1]] = bad[[j + 1, j]]
        assert G.par_first_unsorted(bad, False) == j, j
    fmt = O.FORMATS[x.dtype]
    words = O.to_words(x)
    for p in (0, n // 3, n - 1):
        key = int(O.to_words(s[p:p + 1])[0])
        assert G.par_rank(x, key, fmt, False) == O.rank(words, key, fmt, False)


# --- keys of two words (65..128 bits) -----------------------------------------

_M64 = (1 << 64) - 1


def _two_word(keys):
    hi = np.array([v >> 64 for v in keys], dtype=np.uint64)
    lo = np.array([v & _M64 for v in keys], dtype=np.uint64)
    return hi, lo


def _int_value(v, w, kind):
    return v - (1 << w) if kind == O.SIGNED and v >> (w - 1) else v


def pin_two_word_traces():
    """Figs. 1 and 2 through the two-word path: every printed row (stable
    split, level limit) and the final row (swap loop)."""
    for name in ("fig1_unsigned_trace.txt", "fig2_signed_trace.txt"):
        fmt, asc, rows = load_trace(name)
        for lvl, row in rows.items():
            hi, lo = _two_word(rows[0])
            if lvl:
                v, _ = O.bsort_words2(hi, lo, fmt.w, fmt.kind, not asc, O.STABLE, lvl, check=True)
                assert v == 0
            assert lo.tolist() == row and not hi.any(), (name, lvl, lo.tolist())
        hi, lo = _two_word(rows[0])
        O.bsort_words2(hi, lo, fmt.w, fmt.kind, not asc, O.LITERAL)
        assert lo.tolist() == rows[max(rows)]


def pin_two_word_random_vs_integers():
    """Unsigned and signed keys of 65..128 bits, tie-heavy and spread over
    the word boundary: both partition modes and directions give the order of
    the numbers they encode (Python integers), with invariants (i)/(ii) after
    every partition."""
    rnd = random.Random(77)
    for w in (65, 66, 100, 127, 128):
        for kind in (O.UNSIGNED, O.SIGNED):
            pool = [rnd.getrandbits(w) for _ in range(6)]
            keys = [rnd.choice(pool) if rnd.random() < 0.4 else rnd.getrandbits(w) for _ in range(600)]
            keys += [1 << 63, 1 << 64, (1 << 64) - 1, (1 << 64) + 1, 0, (1 << w) - 1, 1 << (w - 1),
                     (1 << (w - 1)) - 1]
            for desc in (False, True):
                want = sorted(keys, key=lambda v: _int_value(v, w, kind), reverse=desc)
                for mode in (O.LITERAL, O.STABLE):
                    hi, lo = _two_word(keys)
                    v, _ = O.bsort_words2(hi, lo, w, kind, desc, mode, check=True)
                    assert v == 0
                    got = [(int(h) << 64) | int(l) for h, l in zip(hi, lo)]
                    assert got == want, (w, kind, desc, mode)


def pin_two_word_window_exhaustive():
    """Every pattern of bits 61..66 (across the word boundary) in 128-bit
    keys whose other bits are fixed, shuffled: sorted as the integers, and
    the definition comparator agrees with integer comparison."""
    rnd = random.Random(5)
    for kind in (O.UNSIGNED, O.SIGNED):
        for fixed in (0, (1 << 127) | 0xABCDEF, (1 << 70) | 3):
            keys = [(fixed & ~(63 << 61)) | (p << 61) for p in range(64)]
            rnd.shuffle(keys)
            for desc in (False, True):
                hi, lo = _two_word(keys)
                O.bsort_words2(hi, lo, 128, kind, desc)
                got = [(int(h) << 64) | int(l) for h, l in zip(hi, lo)]
                assert got == sorted(keys, key=lambda v: _int_value(v, 128, kind), reverse=desc)
            for x, y in zip(keys, keys[1:] + keys[:1]):
                a, b = _int_value(x, 128, kind), _int_value(y, 128, kind)
                assert O.cmp2(x >> 64, x & _M64, y >> 64, y & _M64, 128, kind) == (a > b) - (a < b)


ALL_PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]


def failing():
    """Names of the pins that fail (used against planted-mistake builds)."""
    bad = []
    for p in ALL_PINS:
        try:
            p()
        except Exception:  # noqa: BLE001 - any failure counts
            bad.append(p.__name__)
    return bad
