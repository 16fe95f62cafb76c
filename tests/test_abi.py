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


def test_more_argument_checks_without_a_gpu(lib):
    """Entry points added for tuning, intermediate states, serving and
    in-place accounting validate their arguments before any CUDA call."""
    import paper_2603_08929_gb300 as pkg
    h = ctypes.c_void_p()
    assert lib.bsort_handle_create(ctypes.byref(h)) == 0
    try:
        T = pkg._Tuning
        bad = T(12, 0, 0, 0)
        assert lib.bsort_handle_set_tuning(h, 4, ctypes.byref(bad)) == 1   # digit width out of range
        assert lib.bsort_handle_set_tuning(h, 4, ctypes.byref(T(11, 0, 0, 3))) == 1  # chunk of 3 tiles
        assert lib.bsort_handle_set_tuning(h, 4, ctypes.byref(T(11, 0, 0, 1))) == 0
        assert lib.bsort_handle_set_tuning(h, 3, None) == 1                 # key width
        assert lib.bsort_handle_set_tuning(h, 8, ctypes.byref(T(6, 1024, 128, 0))) == 0
        assert lib.bsort_handle_set_tuning(h, 8, None) == 0                 # back to defaults
        ws = ctypes.c_void_p(0x100000)
        # intermediate state: levels >= 1, 4/8-byte keys, keys and workspace checked
        assert lib.bsort_keys_partial_ws(h, ctypes.c_void_p(0x1000), 10, 6, 0, 0, ws, 1 << 20, None) == 1
        assert lib.bsort_keys_partial_ws(h, ctypes.c_void_p(0x1000), 10, 3, 0, 1, ws, 1 << 20, None) == 2
        assert lib.bsort_keys_partial_ws(h, None, 10, 6, 0, 1, ws, 1 << 20, None) == 1
        assert lib.bsort_keys_partial_ws(h, ctypes.c_void_p(0x1000), 10, 6, 0, 1, ctypes.c_void_p(0x100010),
                                         1 << 20, None) == 3                # workspace not 256-byte aligned
        # bsort_keys_ws: unknown mode, missing workspace
        assert lib.bsort_keys_ws(h, ctypes.c_void_p(0x1000), 10, 6, 0, 7, ws, 1 << 20, None) == 1
        assert lib.bsort_keys_ws(h, ctypes.c_void_p(0x1000), 10, 6, 0, 1, None, 0, None) == 1
        # the segmented form takes 4- and 8-byte keys only
        assert lib.bsort_keys_segmented(ctypes.c_void_p(0x1000), 10, ctypes.c_void_p(0x2000), 2, 3, 0, None) == 2
        # no call yet: no auxiliary bytes
        n = ctypes.c_size_t(123)
        assert lib.bsort_last_aux_bytes(h, ctypes.byref(n)) == 0 and n.value == 0
    finally:
        lib.bsort_handle_destroy(h)
    # server configuration checks
    srv = ctypes.c_void_p()
    C = pkg._ServerConfig
    assert lib.bsort_server_create(ctypes.byref(C(0, 1, 1 << 30, 1 << 20, 1 << 16, 0, 0)), ctypes.byref(srv)) == 1
    assert lib.bsort_server_create(ctypes.byref(C(2, 0, 1 << 30, 1 << 20, 1 << 16, 0, 0)), ctypes.byref(srv)) == 1
    assert lib.bsort_server_create(ctypes.byref(C(2, 1, 1 << 30, 1 << 20, 1 << 16, 5, 0)), ctypes.byref(srv)) == 1
    assert lib.bsort_server_submit(None, None, 0, 6, 0, 0) == 1


def test_pairs_argument_checks_without_a_gpu(lib):
    """Key-value sorting validates everything before any CUDA call."""
    import paper_2603_08929_gb300 as pkg
    h = ctypes.c_void_p()
    assert lib.bsort_handle_create(ctypes.byref(h)) == 0
    try:
        k, v, ix = ctypes.c_void_p(0x1000), ctypes.c_void_p(0x2000), ctypes.c_void_p(0x3000)
        ws = ctypes.c_void_p(0x100000)
        big = 1 << 30
        assert lib.bsort_pairs_ws(None, k, v, 4, ix, 10, 6, 0, ws, big, None) == 1      # no handle
        assert lib.bsort_pairs_ws(h, k, v, 4, ix, 10, 42, 0, ws, big, None) == 1        # bad dtype
        assert lib.bsort_pairs_ws(h, k, v, 3, ix, 10, 6, 0, ws, big, None) == 1         # 3-byte values
        assert lib.bsort_pairs_ws(h, k, v, 4, ix, 1 << 32, 6, 0, ws, big, None) == 2    # positions need 32 bits
        assert lib.bsort_pairs_ws(h, None, v, 4, ix, 0, 6, 0, None, 0, None) == 0       # n == 0
        assert lib.bsort_pairs_ws(h, k, None, 0, None, 1, 6, 0, None, 0, None) == 0     # n == 1, nothing to write
        assert lib.bsort_pairs_ws(h, None, v, 4, ix, 10, 6, 0, ws, big, None) == 1      # NULL keys
        assert lib.bsort_pairs_ws(h, ctypes.c_void_p(0x1002), v, 4, ix, 10, 6, 0, ws, big, None) == 3
        assert lib.bsort_pairs_ws(h, k, ctypes.c_void_p(0x2004), 8, ix, 10, 6, 0, ws, big, None) == 3
        assert lib.bsort_pairs_ws(h, k, v, 4, ctypes.c_void_p(0x3004), 10, 6, 0, ws, big, None) == 3
        assert lib.bsort_pairs_ws(h, k, v, 4, ix, 10, 6, 0, None, big, None) == 1       # no workspace
        assert lib.bsort_pairs_ws(h, k, v, 4, ix, 10, 6, 0, ctypes.c_void_p(0x100010), big, None) == 3
        need = pkg.pairs_workspace_bytes(10, "int32")
        assert lib.bsort_pairs_ws(h, k, v, 4, ix, 10, 6, 0, ws, need - 1, None) == 5
    finally:
        lib.bsort_handle_destroy(h)
    # the value-carrying sort (alternate keys, two 4-byte position buffers, an
    # 8-byte gather target); 1- and 2-byte keys add their 32-bit order codes;
    # no tuning changes it (the key-value levels have a fixed shape)
    n = 1 << 20
    assert pkg.pairs_workspace_bytes(n, "float64") - pkg.pairs_workspace_bytes(n, "float32") >= 4 * n
    assert pkg.pairs_workspace_bytes(n, "int32") >= (4 + 4 + 4 + 8) * n
    assert pkg.pairs_workspace_bytes(n, "uint8") - pkg.pairs_workspace_bytes(n, "int32") >= 4 * n
    for dt in ("int32", "uint8", "float64"):
        assert pkg.pairs_workspace_bytes(n, dt, tuning8={"radix_bits": 11}) == pkg.pairs_workspace_bytes(n, dt)
        assert pkg.pairs_workspace_bytes(n, dt, tuning8={}) == pkg.pairs_workspace_bytes(n, dt)
