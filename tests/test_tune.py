"""Host side of the tuning: workspace sizes of tuned layouts, argument checks
and the autotuner's table (no GPU needed)."""
import json

import pytest


@pytest.fixture(scope="module")
def pkg():
    from paper_2603_08929_gb300 import build as b
    b.build()
    import paper_2603_08929_gb300 as p
    return p


def test_tuned_workspace_sizes(pkg):
    n = 1 << 24
    base = pkg.workspace_bytes(n, "int32")
    assert pkg.workspace_bytes(n, "int32", tuning={}) == base
    # a smaller finish threshold needs longer work lists; a narrower digit more levels
    assert pkg.workspace_bytes(n, "int32", tuning={"unit_keys": 512}) > base
    assert pkg.workspace_bytes(n, "int32", tuning={"radix_bits": 4}) > base
    # one bit per level: 32 levels' worth of work lists
    assert pkg.workspace_bytes(n, "int32", tuning={"radix_bits": 1}) > pkg.workspace_bytes(
        n, "int32", tuning={"radix_bits": 4})
    # wider digits: 2048-entry tables per chunk and bucket
    assert pkg.workspace_bytes(n, "int32", tuning={"radix_bits": 11}) > base
    assert pkg.workspace_bytes(n, "int32", tuning={"radix_bits": 9}) == pkg.workspace_bytes(
        n, "int32", tuning={"radix_bits": 9, "chunk_tiles": 2})
    # a chunk of one tile doubles the chunk lists
    assert pkg.workspace_bytes(n, "int32", tuning={"chunk_tiles": 1}) > base
    assert pkg.workspace_bytes(n, "int32", tuning={"chunk_tiles": 2}) == base
    # the in-place mode runs digits wider than 8 bits as 8 bits
    ip8 = pkg.workspace_bytes(n, "int32", mode=pkg.MODE_INPLACE, tuning={"radix_bits": 8})
    assert pkg.workspace_bytes(n, "int32", mode=pkg.MODE_INPLACE, tuning={"radix_bits": 11}) == ip8
    # 1/2-byte keys ignore the tuning
    assert pkg.workspace_bytes(n, "uint16", tuning={"radix_bits": 4}) == pkg.workspace_bytes(n, "uint16")


def test_tuned_segmented_workspace_sizes(pkg):
    n, s = 1 << 24, 5000
    base = pkg.segmented_workspace_bytes(n, s, "float32")
    assert pkg.segmented_workspace_bytes(n, s, "float32", tuning={}) == base
    assert pkg.segmented_workspace_bytes(n, s, "float32", tuning={"radix_bits": 11}) > base
    assert pkg.segmented_workspace_bytes(n, s, "float32", tuning={"unit_keys": 512}) > base
    with pytest.raises(pkg.BsortError):
        pkg.segmented_workspace_bytes(n, s, "float32", tuning={"radix_bits": 12})


@pytest.mark.parametrize("bad", [{"radix_bits": -1}, {"radix_bits": 12}, {"unit_keys": 100}, {"unit_keys": 1 << 20},
                                 {"merge_keys": 10}, {"unit_keys": 1000, "merge_keys": 900}, {"chunk_tiles": 3},
                                 {"chunk_tiles": -1}])
def test_invalid_tuning_rejected(pkg, bad):
    with pytest.raises(pkg.BsortError):
        pkg.workspace_bytes(1000, "int32", tuning=bad)


def test_candidates_cover_the_digit_widths():
    from paper_2603_08929_gb300 import tune
    assert {c["radix_bits"] for c in tune.CANDIDATES} == {4, 6, 8, 11}
    assert {c["chunk_tiles"] for c in tune.CANDIDATES} == {0, 1}
    assert all(set(c) == set(tune.FIELDS) for c in tune.CANDIDATES)


def test_table_roundtrip_and_lookup(tmp_path):
    from paper_2603_08929_gb300 import tune
    table = {"int32": {"20": {"radix_bits": 6, "unit_keys": 2048, "merge_keys": 0, "ms": 0.1},
                       "28": {"radix_bits": 8, "unit_keys": 0, "merge_keys": 0, "ms": 3.3}}}
    p = str(tmp_path / "t.json")
    tune.save_table(table, p)
    assert tune.load_table(p) == json.loads(json.dumps(table))
    assert tune.lookup(table, "int32", 1 << 21)["radix_bits"] == 6  # nearest class 20
    assert tune.lookup(table, "int32", 1 << 27)["radix_bits"] == 8  # nearest class 28
    assert tune.lookup(table, "int32", 1 << 24)["radix_bits"] == 6  # tie: the smaller class
    assert tune.lookup(table, "float64", 1 << 24) == {"radix_bits": 0, "unit_keys": 0, "merge_keys": 0,
                                                      "chunk_tiles": 0}
    assert tune.size_class(3) == 2 and tune.size_class(1 << 28) == 28
