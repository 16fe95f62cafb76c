"""Host model of the counting fill (no GPU).

The 8/16-bit path writes the sorted output from counts: the nonempty bins
become runs (output start, value), and each CTA fills output spans: two
warps find the runs holding the span's first and last key with a 32-ary
search, the runs between are staged when they fit a window, and each thread
writes 16-byte vectors j = t, t + T, ... of the span, resuming its run search
from its previous vector and writing a vector that lies inside one run as the
replicated value.  This model restates those steps in Python (same span
sizing, window bound and search order) and checks the output against
np.repeat on count patterns that stress them: uniform, sparse, one bin, a
run per key, runs straddling spans, and sizes below one vector unit.
"""
import numpy as np
import pytest


def runs_of(counts):
    nz = np.flatnonzero(counts)
    rstart = np.concatenate([[0], np.cumsum(counts[nz])]).astype(np.int64)
    return rstart, nz


def warp_search(starts, lo, hi, p):
    """32 probes per round; the probes at or below p form a prefix."""
    rounds = 0
    while lo < hi:
        step = (hi - lo + 31) // 32
        oks = [lo + (l + 1) * step <= hi and starts[lo + (l + 1) * step] <= p for l in range(32)]
        k = sum(oks)
        assert oks == [True] * k + [False] * (32 - k), "probes not a prefix"
        lo += k * step
        hi = min(hi, lo + step - 1)
        rounds += 1
    assert rounds <= 4  # 32^4 > 65536 runs
    return lo


def bin_of(starts, lo, hi, p):
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if starts[mid] <= p:
            lo = mid
        else:
            hi = mid - 1
    return lo


def model_fill(counts, kvec, threads=256, ctas=1216, window=2048, min_vecs=4):
    n = int(counts.sum())
    rstart, rval = runs_of(counts)
    nr = len(rval)
    unit = threads * kvec
    span = -(-n // (2 * ctas))
    span = max(-(-span // unit) * unit, min_vecs * unit)
    out = np.full(n, -1, dtype=np.int64)
    fast = 0
    for sp in range(-(-n // span)):
        p0, p1 = sp * span, min(n, sp * span + span)
        r0, r1 = warp_search(rstart, 0, nr - 1, p0), warp_search(rstart, 0, nr - 1, p1 - 1)
        assert rstart[r0] <= p0 < rstart[r0 + 1] and rstart[r1] <= p1 - 1 < rstart[r1 + 1]
        windowed = r1 - r0 + 2 <= window + 1
        for t in range(threads):
            r_prev = r0
            for j in range(t, span // kvec, threads):
                p = p0 + j * kvec
                if p >= p1:
                    break
                r = r_prev if p < rstart[r_prev + 1] else bin_of(rstart, r_prev, r1, p)
                assert r0 <= r <= r1 and (windowed or True)
                nxt, val = rstart[r + 1], rval[r]
                cnt = min(kvec, p1 - p)
                if cnt == kvec and p + kvec <= nxt:
                    out[p:p + kvec] = val
                    fast += 1
                else:
                    for q in range(p, p + cnt):
                        while q >= nxt:
                            r += 1
                            assert r <= r1, "stepped past the span's last run"
                            nxt, val = rstart[r + 1], rval[r]
                        out[q] = val
                r_prev = r
    return out, fast


def _counts(kind, bins, n, rng):
    if kind == "uniform":
        return np.bincount(rng.integers(0, bins, n), minlength=bins)
    if kind == "sparse":
        c = np.zeros(bins, dtype=np.int64)
        c[rng.choice(bins, 8, replace=False)] = rng.multinomial(n, [1 / 8] * 8)
        return c
    if kind == "one":
        c = np.zeros(bins, dtype=np.int64)
        c[rng.integers(bins)] = n
        return c
    if kind == "per_key":  # a run of one key in most places
        c = np.zeros(bins, dtype=np.int64)
        c[:min(n, bins)] = 1
        c[0] += n - c.sum()
        return c
    if kind == "zipf":
        w = 1.0 / np.arange(1, bins + 1) ** 1.2
        return rng.multinomial(n, w / w.sum())
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["uniform", "sparse", "one", "per_key", "zipf"])
@pytest.mark.parametrize("bins,kvec", [(256, 16), (65536, 8)], ids=["8bit", "16bit"])
@pytest.mark.parametrize("n", [1, 15, 4096 + 3, 70001])
def test_fill_model_equals_repeat(n, bins, kvec, kind):
    rng = np.random.default_rng(n + bins)
    counts = _counts(kind, bins, n, rng)
    got, _ = model_fill(counts, kvec, ctas=4)  # few CTAs: several spans at these sizes
    assert np.array_equal(got, np.repeat(np.arange(bins), counts))


def test_fill_model_takes_the_fast_path_on_long_runs():
    counts = np.zeros(256, dtype=np.int64)
    counts[[3, 200]] = [40000, 30001]
    got, fast = model_fill(counts, 16, ctas=4)
    assert np.array_equal(got, np.repeat(np.arange(256), counts))
    assert fast >= (70001 // 16) - 8  # every vector but those at the run boundary and the tail


def test_warp_search_matches_binary_search():
    rng = np.random.default_rng(3)
    starts = np.concatenate([[0], np.cumsum(rng.integers(1, 50, 70000))])
    for p in rng.integers(0, starts[-1], 200):
        assert warp_search(starts, 0, len(starts) - 2, p) == bin_of(starts, 0, len(starts) - 2, p)
