"""bsort oracle -- TEST INFRASTRUCTURE ONLY.

Python front of ``bsort_oracle.c``: a plain single-threaded CPU restatement of
the paper's Algorithms 1-5 plus a definition-order sort used to pin it.  Only
``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package; the CUDA library never does.

Keys travel as ``uint64`` words holding the raw ``w``-bit pattern, so the same
code sorts the paper's 3-, 4- and 6-bit examples and 8..64-bit machine types.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bsort_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")

UNSIGNED, SIGNED, FLOAT = 0, 1, 2
LITERAL, STABLE = 0, 1


@dataclass(frozen=True)
class KeyFormat:
    """Word size ``w``, key kind and (floats) exponent/mantissa widths."""

    w: int
    kind: int
    e: int = 0
    f: int = 0


# Table II of the paper plus the unsigned, 8/16-bit and half types named by the
# workload; fp16 follows the IEEE layout with (w, e, f) = (16, 5, 10).
FORMATS = {
    np.dtype(np.uint8): KeyFormat(8, UNSIGNED),
    np.dtype(np.int8): KeyFormat(8, SIGNED),
    np.dtype(np.uint16): KeyFormat(16, UNSIGNED),
    np.dtype(np.int16): KeyFormat(16, SIGNED),
    np.dtype(np.float16): KeyFormat(16, FLOAT, 5, 10),
    np.dtype(np.uint32): KeyFormat(32, UNSIGNED),
    np.dtype(np.int32): KeyFormat(32, SIGNED),
    np.dtype(np.float32): KeyFormat(32, FLOAT, 8, 23),
    np.dtype(np.uint64): KeyFormat(64, UNSIGNED),
    np.dtype(np.int64): KeyFormat(64, SIGNED),
    np.dtype(np.float64): KeyFormat(64, FLOAT, 11, 52),
}

_UINT_OF_WIDTH = {8: np.uint8, 16: np.uint16, 32: np.uint32, 64: np.uint64}

# bfloat16 (the high half of a binary32), which numpy has no dtype for: its
# keys travel as uint16 bit patterns with this format passed explicitly.
BF16 = KeyFormat(16, FLOAT, 8, 7)


def _compile(out_path: str, plant: int = 0) -> None:
    tmp = out_path + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    if plant:
        cmd.insert(1, "-DORC_PLANT=%d" % plant)
    subprocess.check_call(cmd)
    os.replace(tmp, out_path)


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (seconds)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        _compile(_LIB_PATH)
    return _LIB_PATH


def build_planted(plant: int, out_path: str) -> str:
    """Build a copy of the oracle with one deliberate mistake (pin tests only)."""
    _compile(out_path, plant)
    return out_path


_lib = None


def _load():
    global _lib
    if _lib is None:
        path = os.environ.get("BSORT_ORACLE_LIB") or build()
        lib = ctypes.CDLL(path)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        sz = ctypes.c_size_t
        i = ctypes.c_int
        lib.orc_bsort.argtypes = [u64p, sz, i, i, i, i, i, i, i, i, i, u64p]
        lib.orc_bsort.restype = i
        lib.orc_sort_by_definition.argtypes = [u64p, sz, i, i, i, i, i]
        lib.orc_sort_by_definition.restype = i
        lib.orc_cmp_total.argtypes = [ctypes.c_uint64, ctypes.c_uint64, i, i, i, i]
        lib.orc_cmp_total.restype = i
        lib.orc_float_value.argtypes = [ctypes.c_uint64, i, i, i]
        lib.orc_float_value.restype = ctypes.c_double
        lib.orc_first_unsorted.argtypes = [u64p, sz, i, i, i, i, i]
        lib.orc_first_unsorted.restype = ctypes.c_int64
        lib.orc_rank.argtypes = [u64p, sz, ctypes.c_uint64, i, i, i, i, i, u64p, u64p]
        lib.orc_rank.restype = None
        lib.orc_multiset_digest.argtypes = [u64p, sz, u64p]
        lib.orc_multiset_digest.restype = None
        lib.orc_stable_argsort.argtypes = [u64p, sz, i, i, i, i, i, u64p]
        lib.orc_stable_argsort.restype = i
        lib.orc_bsort2.argtypes = [u64p, u64p, sz, i, i, i, i, i, i, u64p]
        lib.orc_bsort2.restype = i
        lib.orc_cmp2.argtypes = [ctypes.c_uint64] * 4 + [i, i]
        lib.orc_cmp2.restype = i
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def to_words(x: np.ndarray) -> np.ndarray:
    """Raw bit patterns of a numpy array as contiguous uint64 words."""
    x = np.ascontiguousarray(x)
    fmt = FORMATS[x.dtype]
    return x.view(_UINT_OF_WIDTH[fmt.w]).astype(np.uint64)


def from_words(words: np.ndarray, dtype) -> np.ndarray:
    dtype = np.dtype(dtype)
    fmt = FORMATS[dtype]
    return words.astype(_UINT_OF_WIDTH[fmt.w]).view(dtype)


def bsort_words(words: np.ndarray, fmt: KeyFormat, descending: bool = False, mode: int = LITERAL,
                max_levels: int = 0, literal_alg4: bool = False, check: bool = False):
    """Sort raw ``w``-bit words in place with Algs. 1-5; returns (violations, partitions)."""
    assert words.dtype == np.uint64 and words.flags.c_contiguous
    stats = np.zeros(2, dtype=np.uint64)
    st = _load().orc_bsort(_ptr(words), words.size, fmt.w, fmt.kind, fmt.e, fmt.f,
                           0 if descending else 1, mode, max_levels, int(literal_alg4),
                           int(check), _ptr(stats))
    if st != 0:
        raise ValueError("oracle rejected the input (status %d)" % st)
    return int(stats[0]), int(stats[1])


def bsort(x: np.ndarray, descending: bool = False, mode: int = LITERAL, max_levels: int = 0,
          literal_alg4: bool = False, check: bool = False) -> np.ndarray:
    """Sorted copy of ``x`` (any dtype of ``FORMATS``) by the paper's method."""
    words = to_words(x)
    v, _ = bsort_words(words, FORMATS[np.dtype(x.dtype)], descending, mode, max_levels,
                       literal_alg4, check)
    if check and v:
        raise AssertionError("invariants (i)/(ii) violated %d times" % v)
    return from_words(words, x.dtype)


def sort_words_by_definition(words: np.ndarray, fmt: KeyFormat, descending: bool = False) -> None:
    assert words.dtype == np.uint64 and words.flags.c_contiguous
    st = _load().orc_sort_by_definition(_ptr(words), words.size, fmt.w, fmt.kind, fmt.e, fmt.f,
                                        0 if descending else 1)
    if st != 0:
        raise ValueError("oracle rejected the input (status %d)" % st)


def sort_by_definition(x: np.ndarray, descending: bool = False) -> np.ndarray:
    """Sorted copy of ``x`` by the definition order (qsort + comparator)."""
    words = to_words(x)
    sort_words_by_definition(words, FORMATS[np.dtype(x.dtype)], descending)
    return from_words(words, x.dtype)


def cmp_total(a: int, b: int, fmt: KeyFormat) -> int:
    return _load().orc_cmp_total(a, b, fmt.w, fmt.kind, fmt.e, fmt.f)


def float_value(bits: int, fmt: KeyFormat) -> float:
    return _load().orc_float_value(bits, fmt.w, fmt.e, fmt.f)


def first_unsorted_words(words: np.ndarray, fmt: KeyFormat, descending: bool = False) -> int:
    """Index of the first adjacent pair of raw words out of order, or -1."""
    words = np.ascontiguousarray(words, dtype=np.uint64)
    return int(_load().orc_first_unsorted(_ptr(words), words.size, fmt.w, fmt.kind, fmt.e,
                                          fmt.f, 0 if descending else 1))


def first_unsorted(x: np.ndarray, descending: bool = False) -> int:
    """Index of the first adjacent pair out of order, or -1."""
    return first_unsorted_words(to_words(x), FORMATS[np.dtype(x.dtype)], descending)


def rank(x_words: np.ndarray, value: int, fmt: KeyFormat, descending: bool = False):
    """(elements strictly before ``value``, elements bit-identical to it)."""
    less = np.zeros(1, dtype=np.uint64)
    eq = np.zeros(1, dtype=np.uint64)
    _load().orc_rank(_ptr(x_words), x_words.size, int(value), fmt.w, fmt.kind, fmt.e, fmt.f,
                     0 if descending else 1, _ptr(less), _ptr(eq))
    return int(less[0]), int(eq[0])


def multiset_digest_words(words: np.ndarray) -> tuple:
    """Order-independent digest of a multiset of raw words: (sum, sum, xor, count)."""
    words = np.ascontiguousarray(words, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    _load().orc_multiset_digest(_ptr(words), words.size, _ptr(out))
    return tuple(int(v) for v in out)


def multiset_digest(x: np.ndarray) -> tuple:
    return multiset_digest_words(to_words(x))


def stable_argsort_words(words: np.ndarray, fmt: KeyFormat, descending: bool = False) -> np.ndarray:
    """Input positions in the order of a stable sort of raw words by the
    definition order (equal keys keep input order)."""
    words = np.ascontiguousarray(words, dtype=np.uint64)
    perm = np.zeros(words.size, dtype=np.uint64)
    st = _load().orc_stable_argsort(_ptr(words), words.size, fmt.w, fmt.kind, fmt.e, fmt.f,
                                    0 if descending else 1, _ptr(perm))
    if st != 0:
        raise ValueError("oracle rejected the input (status %d)" % st)
    return perm.astype(np.int64)


def stable_argsort(x: np.ndarray, descending: bool = False) -> np.ndarray:
    """Key-value sorting by definition: the permutation (int64 positions) a
    stable sort of ``x`` under the paper's order applies; ``x[p]`` is the
    sorted keys and ``v[p]`` the values carried along."""
    return stable_argsort_words(to_words(x), FORMATS[np.dtype(x.dtype)], descending)


# --- keys of two words (up to 128 bits): unsigned and signed integers --------
#
# A key array is a uint64 array of shape (n, 2): column 0 the low word, column
# 1 the high word (the little-endian layout of a 16-byte integer), so the same
# memory is the GPU library's 128-bit keys.

U128 = KeyFormat(128, UNSIGNED)
I128 = KeyFormat(128, SIGNED)


def bsort_words2(hi: np.ndarray, lo: np.ndarray, w: int, kind: int, descending: bool = False,
                 mode: int = LITERAL, max_levels: int = 0, check: bool = False):
    """Sorts the two-word keys (hi[i], lo[i]) of w bits in place with Algs.
    1-3; returns (invariant violations, partitions)."""
    assert hi.dtype == lo.dtype == np.uint64 and hi.flags.c_contiguous and lo.flags.c_contiguous
    stats = np.zeros(2, dtype=np.uint64)
    st = _load().orc_bsort2(_ptr(hi), _ptr(lo), hi.size, w, kind, 0 if descending else 1, mode, max_levels,
                            int(check), _ptr(stats))
    if st != 0:
        raise ValueError("oracle rejected the input (status %d)" % st)
    return int(stats[0]), int(stats[1])


def bsort128(x: np.ndarray, signed: bool = False, descending: bool = False, mode: int = LITERAL,
             check: bool = False) -> np.ndarray:
    """Sorted copy of 128-bit keys given as a uint64 (n, 2) array [lo, hi]."""
    x = np.asarray(x, dtype=np.uint64).reshape(-1, 2)
    lo = np.ascontiguousarray(x[:, 0])
    hi = np.ascontiguousarray(x[:, 1])
    v, _ = bsort_words2(hi, lo, 128, SIGNED if signed else UNSIGNED, descending, mode, check=check)
    if check and v:
        raise AssertionError("invariants (i)/(ii) violated %d times" % v)
    return np.stack([lo, hi], axis=1)


def cmp2(xh: int, xl: int, yh: int, yl: int, w: int, kind: int) -> int:
    return _load().orc_cmp2(xh, xl, yh, yl, w, kind)
