"""The C-ABI library loads and exports every declared entry point (CPU only;
no call here reaches the GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_08929_gb300 import build as b
    b.build()
    import paper_2603_08929_gb300 as pkg
    return pkg.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "bsort.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bsort_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("bsort_keys", "bsort_keys_ws", "bsort_workspace_bytes", "bsort_keys_host",
                     "bsort_handle_create", "bsort_handle_destroy", "bsort_get_error",
                     "bsort_status_string"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    import paper_2603_08929_gb300 as pkg
    for code in range(10):
        assert pkg.status_string(code).startswith("BSORT_")
    assert pkg.status_string(99) == "BSORT_ERR_UNKNOWN"


def test_argument_checks_before_any_launch(lib):
    # rejected calls return before touching CUDA
    assert lib.bsort_keys(None, 0, 6, 0, None) == 0            # n == 0: nothing to do
    assert lib.bsort_keys(None, 1, 6, 0, None) == 0            # n == 1: nothing to do
    assert lib.bsort_keys(None, 5, 6, 0, None) == 1            # NULL keys
    assert lib.bsort_keys(ctypes.c_void_p(0x1002), 5, 6, 0, None) == 3  # int32 at 2 mod 4
    assert lib.bsort_keys(ctypes.c_void_p(0x1000), 5, 42, 0, None) == 1  # bad dtype
    assert lib.bsort_keys(ctypes.c_void_p(0x1000), 1 << 33, 6, 0, None) == 2  # n >= 2^32, 4-byte keys


def test_workspace_sizes(lib):
    import paper_2603_08929_gb300 as pkg
    for dt in pkg.DTYPES:
        small = pkg.workspace_bytes(1000, dt)
        big = pkg.workspace_bytes(1 << 28, dt)
        assert 0 < small <= big
    # ping-pong: the alternate buffer dominates for wide keys; metadata is
    # bounded by the worst case of buckets just above the finish threshold
    n = 1 << 28
    assert n * 4 <= pkg.workspace_bytes(n, "int32") <= n * 4 * 1.25
    assert n * 8 <= pkg.workspace_bytes(n, "float64") <= n * 8 * 1.25
    # counting path: no alternate buffer
    assert pkg.workspace_bytes(n, "uint8") < 1 << 20
    # in-place: no alternate buffer; the reservation (metadata, block buffers
    # for the worst case of buckets just above the shared-memory capacity,
    # slot states) stays well below one copy of the keys
    for dt, b in (("int32", 4), ("float64", 8)):
        ip = pkg.workspace_bytes(n, dt, mode=pkg.MODE_INPLACE)
        assert ip < 0.75 * n * b, (dt, ip / (n * b))
        assert ip < pkg.workspace_bytes(n, dt)
    assert pkg.workspace_bytes(n, "uint16", mode=pkg.MODE_INPLACE) == pkg.workspace_bytes(n, "uint16")
    with pytest.raises(pkg.BsortError):
        pkg.workspace_bytes(100, "int32", mode=7)
