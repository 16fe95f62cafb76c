"""The shared-memory finish's fast counting path (units whose keys agree
above bit 16, read as vectors, one counter per (sub-bucket, low value)) and
its hand-offs, byte for byte against the oracle.  Inputs are built so that
every finish unit is one bucket of known shape: key = (u << 16) | low with
u < 256 the unit, so the top digit is constant, the next one selects the
unit, and the unit's keys vary in their low 16 bits only."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import assert_bit_exact, oracle_expected, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2603_08929_gb300 import build as b
    b.build()
    torch.cuda.set_device(0)


def sorted_with_profile(x, descending=False, offset=0):
    """bsort_keys_ws on x placed `offset` keys into a device buffer (offset 0:
    16-byte aligned); returns the output and the finish units by path."""
    import torch
    import paper_2603_08929_gb300 as bs
    buf = torch.zeros(x.size + offset, dtype=getattr(torch, x.dtype.name), device="cuda")
    t = buf[offset:]
    t.copy_(torch.from_numpy(x).cuda())
    h = bs.Handle()
    h.set_profiling(True)
    ws = torch.empty(bs.workspace_bytes(t.numel(), x.dtype.name), dtype=torch.uint8, device=t.device)
    bs.bsort_keys_ws(h, t, ws, descending=descending)
    prof = h.profile()
    assert h.get_error() == 0
    return t.cpu().numpy(), prof["finish_units"]


def units(values_per_unit, rng, dtype=np.uint32, nunits=256, top=False):
    """Concatenation of units u = 0..nunits-1: (u << 16) | low for each low
    value the callback gives, shuffled.  top: bits 24-25 also take u & 3, so
    the top digit is scattered too and the units end in the caller's buffer
    (two scatters) instead of the alternate one."""
    parts = [(np.uint64(((u & 3) << 24) if top else 0) | (np.uint64(u) << np.uint64(16)))
             | values_per_unit(u, rng).astype(np.uint64) for u in range(nunits)]
    x = np.concatenate(parts)
    rng.shuffle(x)
    return x.astype(dtype)


@pytest.mark.parametrize("desc", [False, True], ids=["asc", "desc"])
@pytest.mark.parametrize("dtype", ["uint32", "int32", "float32", "uint64"])
def test_fast_path_uniform_units(dtype, desc):
    """Units of ~4096 keys, low 16 bits uniform: every unit takes the fast path."""
    rng = np.random.default_rng(1)
    ut = np.uint64 if dtype == "uint64" else np.uint32
    size = 2000 if dtype == "uint64" else 4000  # below the 8-byte finish tile of 2544 keys
    x = units(lambda u, r: r.integers(0, 1 << 16, size + int(r.integers(0, 200))), rng, ut).view(dtype)
    got, fu = sorted_with_profile(x, desc)
    assert_bit_exact(got, O.bsort(x, descending=desc), dtype)
    assert fu["counting_fast"] == 256 and fu["compare"] + fu["lsd"] == 0, fu


def test_fast_path_fifteen_copies():
    """Every sub-bucket holds one value 15 times (counters reach 15, ranks 14,
    totals 15): still the fast path, exact."""
    rng = np.random.default_rng(2)

    def vals(u, r):
        v = np.arange(273, dtype=np.int64) * 16 + r.integers(0, 16, 273)
        return np.repeat(v, 15)
    x = units(vals, rng)
    got, fu = sorted_with_profile(x)
    assert_bit_exact(got, O.bsort(x), "fifteen copies")
    assert fu["counting_fast"] == 256, fu


@pytest.mark.parametrize("case", ["sixteen_copies", "sub_bucket_of_16", "few_values"])
def test_fast_path_hands_off(case):
    """A counter that would wrap (16 equal keys), a sub-bucket of 16 keys
    over two values, or a handful of values: the fast path gives up with
    nothing written and the unit is finished by the general path, exactly."""
    rng = np.random.default_rng(3)

    def vals(u, r):
        v = r.integers(0, 1 << 16, 4000)
        if u % 7 == 0:
            if case == "sixteen_copies":
                v[:16] = 4242
            elif case == "sub_bucket_of_16":
                v = np.where((v >> 4) == 0x123, 0x4444, v)  # sub-bucket 0x123: these 16 keys only
                v[:8] = 0x1230
                v[8:16] = 0x123F
            else:
                v = r.choice(np.array([7, 900, 65535], dtype=np.int64), 4000)
        return v
    x = units(vals, rng)
    got, fu = sorted_with_profile(x)
    assert_bit_exact(got, O.bsort(x), case)
    handed = (256 + 6) // 7  # units u % 7 == 0
    assert fu["counting_fast"] == 256 - handed, fu
    assert fu["counting"] + fu["compare"] + fu["lsd"] == 256, fu


@pytest.mark.parametrize("bits", [8, 10, 12])
def test_dense_units_skip_the_fast_path(bits):
    """Units whose keys are dense in their few free bits (~2000 keys over
    2^8 .. 2^12 values: sub-buckets of 16 values would hold 16 keys or more)
    go to the general path without trying the fast one -- 8 and 10 free bits
    to the direct counting (one counter per value), 12 to the counting pass;
    exact either way."""
    rng = np.random.default_rng(5 + bits)
    parts = [(np.uint64(u) << np.uint64(bits)) | rng.integers(0, 1 << bits, 2000 + int(rng.integers(0, 100)))
             .astype(np.uint64) for u in range(256)]
    x = np.concatenate(parts).astype(np.uint32)
    rng.shuffle(x)
    got, fu = sorted_with_profile(x)
    assert_bit_exact(got, O.bsort(x), "dense units, %d bits" % bits)
    assert fu["counting_fast"] == 0, fu
    assert fu["counting"] + fu["compare"] + fu["lsd"] == 256, fu


@pytest.mark.parametrize("two_scatters", [False, True], ids=["units_in_alt", "units_in_caller_buffer"])
@pytest.mark.parametrize("offset", [1, 2, 3])
def test_fast_path_unaligned_buffer(offset, two_scatters):
    """The caller's buffer off the 16-byte boundary.  Units in the alternate
    buffer (one scatter) still take the fast path and write the caller's
    buffer key by key; units in the caller's buffer (two scatters) cannot be
    read as vectors and go to the general path."""
    rng = np.random.default_rng(4)
    x = units(lambda u, r: r.integers(0, 1 << 16, 3000 + int(r.integers(0, 2000))), rng, top=two_scatters)
    got, fu = sorted_with_profile(x, False, offset)
    assert_bit_exact(got, O.bsort(x), "offset %d" % offset)
    assert fu["counting"] == 256, fu
    assert fu["counting_fast"] == (0 if two_scatters else 256), fu


@pytest.mark.parametrize("dtype,desc", [("int32", False), ("float32", True), ("uint32", True)])
def test_fast_path_2p26(dtype, desc):
    """2^26 uniform keys: two 8-bit levels leave ~1024-key children with 16
    varying bits (the fast path) and merged groups of the smaller ones (24
    varying bits: the general path); the whole output byte for byte against
    the oracle."""
    x = W.make("uniform", dtype, 1 << 26, seed=26)
    got, fu = sorted_with_profile(x, desc)
    assert_bit_exact(got, oracle_expected(x, desc), "%s 2^26" % dtype)
    assert fu["counting_fast"] == fu["counting"], fu
    assert fu["counting_fast"] > 0.4 * (fu["counting"] + fu["compare"] + fu["lsd"]), fu


def test_fast_path_2p27():
    """2^27 uniform int32: every ~2048-key unit takes the fast path."""
    x = W.make("uniform", "int32", 1 << 27, seed=27)
    got, fu = sorted_with_profile(x)
    assert_bit_exact(got, oracle_expected(x), "int32 2^27")
    assert fu["counting_fast"] > 0.99 * (fu["counting"] + fu["compare"] + fu["lsd"]), fu


@pytest.mark.parametrize("case", ["int32_pos", "int32_neg", "uint32", "float32_pos", "float32_neg"])
@pytest.mark.parametrize("n", [600, 3000, 5100])
def test_direct_counting_of_raw_units(case, n):
    """A small array is one unit read straight from the caller's buffer
    (still in its own encoding); keys that differ only in 8 to 10 low bits of
    the sort order (one sign: the sign bit is a sort-order bit) take the
    direct counting finish: exact, both directions."""
    rng = np.random.default_rng(n)
    x = {"int32_pos": lambda: rng.integers(1000, 1256, n).astype(np.int32),
         "int32_neg": lambda: rng.integers(-300, -44, n).astype(np.int32),
         "uint32": lambda: ((0xABCD << 16) | rng.integers(0, 1024, n)).astype(np.uint32),
         "float32_pos": lambda: (1.0 + rng.integers(0, 256, n) / 256.0).astype(np.float32),
         "float32_neg": lambda: -(1.0 + rng.integers(0, 256, n) / 256.0).astype(np.float32)}[case]()
    for desc in (False, True):
        got, fu = sorted_with_profile(x, desc)
        assert_bit_exact(got, O.bsort(x, descending=desc), "%s n=%d desc=%s" % (case, n, desc))
        assert fu["counting"] == 1 and fu["counting_fast"] == 0, fu
