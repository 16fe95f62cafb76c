"""Host model of the key-value method (no GPU).

The library sorts key-value pairs by sorting distinct 64-bit words: a key's
order-preserving code in the high half and its input position in the low
half; 8-byte keys take two such sorts, on the low and then the high half of
their code, the second with the position in the first sort's output as its
low half.  Here the same composition runs with numpy's sort of the words and
a restatement of the code (Sec. III: the sign bit inverted for signed keys,
negative floats' bits inverted, descending = all bits inverted), and its
permutation must equal the oracle's stable argsort -- for every dtype, with
many ties, both directions.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

UINT = {1: np.uint8, 2: np.uint16, 4: np.uint32, 8: np.uint64}


def code(x: np.ndarray, fmt: O.KeyFormat, descending: bool) -> np.ndarray:
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


def model_perm(x: np.ndarray, descending: bool, fmt: O.KeyFormat = None) -> np.ndarray:
    fmt = fmt or O.FORMATS[x.dtype]
    k = code(x, fmt, descending)
    n = k.size
    pos = np.arange(n, dtype=np.uint64)
    lo32 = np.uint64(0xFFFFFFFF)
    if fmt.w <= 32:
        words = np.sort((k << np.uint64(32)) | pos)
        return (words & lo32).astype(np.int64)
    words = np.sort(((k & lo32) << np.uint64(32)) | pos)
    perm1 = (words & lo32).astype(np.int64)
    words = np.sort(((k[perm1] >> np.uint64(32)) << np.uint64(32)) | pos)
    return perm1[(words & lo32).astype(np.int64)]


@pytest.mark.parametrize("desc", [False, True], ids=["asc", "desc"])
@pytest.mark.parametrize("dtype", [str(d) for d in O.FORMATS])
def test_packed_words_give_the_stable_permutation(dtype, desc):
    for j, dist in enumerate(["distinct8", "zipf", "uniform", "sorted", "reverse"]):
        x = W.make(dist, dtype, 4099, seed=60 + j)
        assert np.array_equal(model_perm(x, desc), O.stable_argsort(x, desc)), (dtype, dist)


@pytest.mark.parametrize("desc", [False, True], ids=["asc", "desc"])
def test_packed_words_bf16_and_float_edges(desc):
    for dtype in ("float16", "float32", "float64"):
        x = W.make("float_edge", dtype, 5003, seed=70)
        assert np.array_equal(model_perm(x, desc), O.stable_argsort(x, desc)), dtype
    w = W.make("float_edge", "bfloat16", 5003, seed=71)
    want = O.stable_argsort_words(w.astype(np.uint64), O.BF16, desc)
    assert np.array_equal(model_perm(w, desc, O.BF16), want)


def test_one_sort_of_the_low_half_is_not_enough():
    """The two 8-byte passes are needed: sorting by the high half of the code
    alone (with positions) misorders keys that differ only below bit 32."""
    x = np.array([5, 3, (1 << 32) + 1, 1 << 32, 4], dtype=np.uint64)
    k = code(x, O.FORMATS[x.dtype], False)
    words = np.sort(((k >> np.uint64(32)) << np.uint64(32)) | np.arange(5, dtype=np.uint64))
    wrong = (words & np.uint64(0xFFFFFFFF)).astype(np.int64)
    assert not np.array_equal(wrong, O.stable_argsort(x))
    assert np.array_equal(model_perm(x, False), O.stable_argsort(x))
