"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module only draws numbers: it holds none of the sort's arithmetic, and
neither the oracle nor the CUDA library imports it.  Every value comes from
one counter-based generator, SplitMix64 (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014): for a seed and a
stream number the i-th word (i = 0, 1, ...) is the generator's i-th output
from the state ``seed ^ (stream << 40)``, i.e.

    mix64(state + (i + 1) * 0x9e3779b97f4a7c15)

with the published 64-bit finaliser ``mix64``.  Being counter based, any slice
of a stream can be produced independently.

Distributions (the paper's experiments use arrays of 1e5..5e9 elements of
Table II's types and give no distribution; these stand in for them):
  uniform    the low w bits of each word: every bit pattern equally likely,
             so floats include +-inf and NaN patterns
  zipf       Zipf(s=1.2) over K = min(2^16, 2^w) distinct patterns drawn
             uniformly without replacement; rank r has weight r^-1.2
  normal     normal(0, 1e3) by Box-Muller, rounded to nearest (integers are
             rounded to the nearest integer and clipped)
  distinct8  8 distinct uniform patterns, one picked uniformly per key
  sorted     `uniform` put in ascending numeric order by numpy's own sort
             (numpy puts NaNs last and treats -0 == +0, so float inputs are
             only nearly sorted under the paper's order)
  reverse    `sorted` reversed
  float_edge floats only: 90% normal(0, 1e3), 2% +-0, 2% subnormal, 2% +-inf,
             4% NaN (half quiet, half signalling, random sign and payload)
  normal01   normal(0, 1) by Box-Muller, rounded like `normal` (integers
             collapse onto a handful of values near 0)
"""
from __future__ import annotations

import math
import os

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

DTYPES = ["uint8", "int8", "uint16", "int16", "float16", "uint32", "int32", "float32",
          "uint64", "int64", "float64", "bfloat16"]
WIDE_DTYPES = ["uint128", "int128"]  # uint64 (n, 2) arrays, low word first
DISTS = ["uniform", "zipf", "normal", "distinct8", "sorted", "reverse", "float_edge", "normal01"]

_UINT = {1: np.uint8, 2: np.uint16, 4: np.uint32, 8: np.uint64}
_CHUNK = 1 << 22


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def words(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Words start..start+count-1 of (seed, stream) as uint64."""
    state = np.uint64((seed ^ (stream << 40)) & 0xFFFFFFFFFFFFFFFF)
    out = np.empty(count, dtype=np.uint64)

    def fill(c0):
        c1 = min(count, c0 + _CHUNK)
        i = np.arange(start + c0 + 1, start + c1 + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            out[c0:c1] = _mix64(state + i * GAMMA)

    starts = range(0, count, _CHUNK)
    if count > 4 * _CHUNK:  # chunks are independent (counter-based): fill them in threads
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
            list(ex.map(fill, starts))
    else:
        for c0 in starts:
            fill(c0)
    return out


def uniform01(seed: int, stream: int, count: int) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of each word."""
    return (words(seed, stream, 0, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def _threaded(count: int, fill) -> None:
    """Runs fill(c0, c1) over [0, count) in _CHUNK pieces, in threads when
    large (numpy releases the GIL inside its array loops)."""
    starts = range(0, count, _CHUNK)
    if count > 4 * _CHUNK:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
            list(ex.map(lambda c0: fill(c0, min(count, c0 + _CHUNK)), starts))
    else:
        for c0 in starts:
            fill(c0, min(count, c0 + _CHUNK))


def normal(seed: int, stream: int, count: int, mean: float = 0.0, std: float = 1.0) -> np.ndarray:
    """Box-Muller (cosine branch) on the pair of words (2i, 2i+1)."""
    out = np.empty(count, dtype=np.float64)

    def fill(c0, c1):
        w = words(seed, stream, 2 * c0, 2 * (c1 - c0))
        u1 = 1.0 - (w[0::2] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)  # (0, 1]
        u2 = (w[1::2] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        out[c0:c1] = mean + std * np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)

    _threaded(count, fill)
    return out


def stream_id(dist: str, dtype: str, sub: int = 0) -> int:
    """Stream number of (distribution, dtype, sub-stream); fits in 24 bits."""
    return ((DISTS.index(dist) << 8 | (DTYPES + WIDE_DTYPES).index(dtype)) << 4) | sub


def _bits_dtype(dtype: np.dtype):
    return _UINT[dtype.itemsize]


def _uniform_patterns(seed, stream, n, dtype):
    w = dtype.itemsize * 8
    u = words(seed, stream, 0, n)
    if w < 64:
        u = u & np.uint64((1 << w) - 1)
    return u.astype(_bits_dtype(dtype)).view(dtype)


def _round_to(x: np.ndarray, dtype: np.dtype) -> np.ndarray:
    if dtype.kind == "f":
        return x.astype(dtype)
    info = np.iinfo(dtype)
    return np.clip(np.rint(x), info.min, info.max).astype(dtype)


def _distinct_patterns(seed, stream, k, dtype):
    """k distinct uniform patterns in first-draw order."""
    w = dtype.itemsize * 8
    if w <= 16 and k >= (1 << w):
        # every pattern: a random permutation by sorting random words
        order = np.argsort(words(seed, stream, 0, 1 << w), kind="stable")
        return order.astype(_bits_dtype(dtype))
    got = np.empty(0, dtype=np.uint64)
    draw = 0
    while got.size < k:
        cand = words(seed, stream, draw, 2 * k + 16)
        draw += cand.size
        if w < 64:
            cand = cand & np.uint64((1 << w) - 1)
        allv = np.concatenate([got, cand])
        _, first = np.unique(allv, return_index=True)
        got = allv[np.sort(first)]
    return got[:k].astype(_bits_dtype(dtype))


def _bf16_bits(x: np.ndarray) -> np.ndarray:
    """bfloat16 patterns of finite doubles: to binary32, then the high half
    rounded to nearest, ties to even."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)
    return r.astype(np.uint16)


def _make_bf16(dist: str, n: int, seed: int) -> np.ndarray:
    """bfloat16 inputs as uint16 bit patterns (numpy has no bfloat16 dtype);
    the same distributions as the other float types."""
    name, u16 = "bfloat16", np.dtype(np.uint16)
    if dist == "uniform":
        return _uniform_patterns(seed, stream_id(dist, name), n, u16)
    if dist in ("sorted", "reverse"):
        x = _uniform_patterns(seed, stream_id("uniform", name), n, u16)
        x = x[np.argsort((x.astype(np.uint32) << np.uint32(16)).view(np.float32), kind="stable")]
        return x if dist == "sorted" else x[::-1].copy()
    if dist in ("normal", "normal01"):
        return _bf16_bits(normal(seed, stream_id(dist, name), n, 0.0, 1e3 if dist == "normal" else 1.0))
    if dist in ("distinct8", "zipf"):
        return make(dist, np.uint16, n, seed + 0x5BF16)
    if dist == "float_edge":
        return _float_edge_bits(seed, n, name, 8, 7, np.uint16,
                                lambda: _bf16_bits(normal(seed, stream_id("float_edge", name, 0), n, 0.0, 1e3)))
    raise ValueError("unknown distribution %r" % dist)


def _make_wide(dist: str, n: int, seed: int, name: str) -> np.ndarray:
    """128-bit integer inputs as a uint64 array of shape (n, 2), low word
    first (numpy has no 128-bit dtype): uniform bits; Zipf(1.2) over 2^16
    patterns and 8 patterns, both drawn as uniform 128-bit words (repeats
    among 2^16 such draws are vanishingly unlikely); normal(0, 1) rounded to
    the nearest integer (clipped at 0 for unsigned keys), sign-extended."""
    if dist == "uniform":
        return np.stack([words(seed, stream_id(dist, name, 0), 0, n), words(seed, stream_id(dist, name, 1), 0, n)],
                        axis=1)
    if dist in ("zipf", "distinct8"):
        k = 1 << 16 if dist == "zipf" else 8
        vals = np.stack([words(seed, stream_id(dist, name, 3), 0, k), words(seed, stream_id(dist, name, 4), 0, k)],
                        axis=1)
        if dist == "distinct8":
            pick = (words(seed, stream_id(dist, name, 2), 0, n) >> np.uint64(61)).astype(np.int64)
        else:
            cdf = np.cumsum(np.arange(1, k + 1, dtype=np.float64) ** -1.2)
            cdf /= cdf[-1]
            pick = np.minimum(np.searchsorted(cdf, uniform01(seed, stream_id(dist, name, 2), n), side="right"), k - 1)
        return vals[pick]
    if dist == "normal01":
        v = np.rint(normal(seed, stream_id(dist, name), n, 0.0, 1.0)).astype(np.int64)
        if name == "uint128":
            v = np.maximum(v, 0)
        lo = v.view(np.uint64)
        hi = np.where(v < 0, np.uint64(0xFFFFFFFFFFFFFFFF), np.uint64(0))
        return np.stack([lo, hi], axis=1)
    raise ValueError("unknown distribution %r for 128-bit keys" % dist)


def make(dist: str, dtype, n: int, seed: int = 0) -> np.ndarray:
    """One input array of ``n`` keys; identical for identical arguments.
    ``dtype`` "bfloat16" gives uint16 bit patterns; "uint128" / "int128" a
    uint64 array of shape (n, 2), low word first."""
    if str(dtype) == "bfloat16":
        return _make_bf16(dist, n, seed)
    if str(dtype) in ("uint128", "int128"):
        return _make_wide(dist, n, seed, str(dtype))
    dtype = np.dtype(dtype)
    name = dtype.name
    if dist == "uniform":
        return _uniform_patterns(seed, stream_id(dist, name), n, dtype)
    if dist in ("sorted", "reverse"):
        x = np.sort(_uniform_patterns(seed, stream_id("uniform", name), n, dtype), kind="stable")
        return x if dist == "sorted" else x[::-1].copy()
    if dist == "normal":
        return _round_to(normal(seed, stream_id(dist, name), n, 0.0, 1e3), dtype)
    if dist == "normal01":
        return _round_to(normal(seed, stream_id(dist, name), n, 0.0, 1.0), dtype)
    if dist == "distinct8":
        vals = _distinct_patterns(seed, stream_id(dist, name, 1), 8, dtype)
        pick = (words(seed, stream_id(dist, name, 2), 0, n) >> np.uint64(61)).astype(np.int64)
        return vals[pick].view(dtype)
    if dist == "zipf":
        k = min(1 << 16, 1 << (dtype.itemsize * 8))
        vals = _distinct_patterns(seed, stream_id(dist, name, 1), k, dtype)
        weights = np.arange(1, k + 1, dtype=np.float64) ** -1.2
        cdf = np.cumsum(weights)
        cdf /= cdf[-1]
        u = uniform01(seed, stream_id(dist, name, 2), n)
        out = np.empty(n, dtype=vals.dtype)

        def fill(c0, c1):
            r = np.minimum(np.searchsorted(cdf, u[c0:c1], side="right"), k - 1)
            out[c0:c1] = vals[r]

        _threaded(n, fill)
        return out.view(dtype)
    if dist == "float_edge":
        return _float_edge(seed, n, dtype)
    raise ValueError("unknown distribution %r" % dist)


def _float_edge(seed: int, n: int, dtype: np.dtype) -> np.ndarray:
    if dtype.kind != "f":
        raise ValueError("float_edge needs a float dtype")
    name = dtype.name
    w = dtype.itemsize * 8
    f_bits = {16: 10, 32: 23, 64: 52}[w]
    ut = _bits_dtype(dtype)
    normal_bits = lambda: _round_to(normal(seed, stream_id("float_edge", name, 0), n, 0.0, 1e3),  # noqa: E731
                                    dtype).view(ut).copy()
    return _float_edge_bits(seed, n, name, w - 1 - f_bits, f_bits, ut, normal_bits).view(dtype)


def _float_edge_bits(seed: int, n: int, name: str, e_bits: int, f_bits: int, ut, normal_bits) -> np.ndarray:
    """Bit patterns of the float edge mix (format with e_bits / f_bits, bits
    type ut): 90% normal(0, 1e3) from normal_bits(), 2% +-0, 2% subnormal, 2%
    +-inf, 4% NaN (half quiet, half signalling, random payloads and signs)."""
    w = 1 + e_bits + f_bits
    out = normal_bits()
    cat = uniform01(seed, stream_id("float_edge", name, 1), n)
    r = words(seed, stream_id("float_edge", name, 2), 0, n)
    sign = ((r >> np.uint64(63)) & np.uint64(1)).astype(ut) << ut(w - 1)
    mant_mask = np.uint64((1 << f_bits) - 1)
    mant = ((r >> np.uint64(1)) & mant_mask)
    exp_all = ut(((1 << e_bits) - 1) << f_bits)
    quiet = ut(1 << (f_bits - 1))

    zero = (cat >= 0.90) & (cat < 0.92)
    sub = (cat >= 0.92) & (cat < 0.94)
    inf = (cat >= 0.94) & (cat < 0.96)
    nan = cat >= 0.96
    out[zero] = sign[zero]
    m_nz = np.where(mant == 0, np.uint64(1), mant).astype(ut)
    out[sub] = sign[sub] | m_nz[sub]
    out[inf] = sign[inf] | exp_all
    is_quiet = ((r >> np.uint64(62)) & np.uint64(1)).astype(bool)
    rest = (mant & np.uint64((1 << (f_bits - 1)) - 1)).astype(ut)
    qn = nan & is_quiet
    sn = nan & ~is_quiet
    out[qn] = sign[qn] | exp_all | quiet | rest[qn]
    rest_nz = np.where(rest == 0, ut(1), rest)
    out[sn] = sign[sn] | exp_all | rest_nz[sn]
    return out


def segment_sizes(seed: int, count: int, max_log2: int = 20, min_size: int = 1,
                  stream: int = 0xF00) -> np.ndarray:
    """Log-uniform sizes floor(2^(max_log2 * u)), at least ``min_size``."""
    u = uniform01(seed, stream, count)
    return np.maximum(np.floor(2.0 ** (max_log2 * u)).astype(np.int64), min_size)


SERVE_DTYPES = ("int16", "int32", "float32", "float64")
SERVE_MIX = (0.25, 0.35, 0.30, 0.10)


def serve_trace(seed: int, rate: float, seconds: float, lo_log2: int = 10, hi_log2: int = 24,
                stream: int = 0xF10) -> dict:
    """An open-loop request trace: Poisson arrivals at ``rate`` per second over
    ``seconds``; sizes floor(2^(lo + (hi - lo) u)); dtype drawn from
    SERVE_DTYPES with probabilities SERVE_MIX; values "uniform" or "normal01"
    with equal probability.  Arrays: t (arrival, s), n, dtype (index into
    SERVE_DTYPES), dist (0 uniform, 1 normal01)."""
    count = int(rate * seconds * 1.5) + 64
    u = uniform01(seed, stream, 4 * count).reshape(count, 4)
    gaps = -np.log(1.0 - u[:, 0]) / rate
    t = np.cumsum(gaps)
    keep = t < seconds
    n = np.floor(2.0 ** (lo_log2 + (hi_log2 - lo_log2) * u[:, 1])).astype(np.int64)
    dt = np.searchsorted(np.cumsum(SERVE_MIX), u[:, 2], side="right").clip(0, len(SERVE_DTYPES) - 1)
    dist = (u[:, 3] >= 0.5).astype(np.int64)
    return {"t": t[keep], "n": n[keep], "dtype": dt[keep], "dist": dist[keep]}
