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
    # 1/2-byte keys ignore the tuning
    assert pkg.workspace_bytes(n, "uint16", tuning={"radix_bits": 4}) == pkg.workspace_bytes(n, "uint16")


@pytest.mark.parametrize("bad", [{"radix_bits": 3}, {"radix_bits": 9}, {"unit_keys": 100}, {"unit_keys": 1 << 20},
                                 {"merge_keys": 10}, {"unit_keys": 1000, "merge_keys": 900}])
def test_invalid_tuning_rejected(pkg, bad):
    with pytest.raises(pkg.BsortError):
        pkg.workspace_bytes(1000, "int32", tuning=bad)


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
    assert tune.lookup(table, "float64", 1 << 24) == {"radix_bits": 0, "unit_keys": 0, "merge_keys": 0}
    assert tune.size_class(3) == 2 and tune.size_class(1 << 28) == 28
