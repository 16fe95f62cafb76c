"""The oracle against its pins (CPU only)."""
import os
import subprocess
import sys

import pytest

import oracle as O
import oracle_pins as P


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin()


# Each deliberate mistake compiled into the oracle must trip at least one pin.
PLANTS = {
    1: "signed sign pass in the requested direction",
    2: "upper-side recursion skips a bit",
    4: "-0 and +0 swapped by the comparator",
    5: "negative NaNs ordered by ascending payload",
    6: "subnormal exponent off by one",
    7: "stable split reverses the back side",
    8: "stable argsort takes ties from the right run",
    9: "first_unsorted never checks the last pair",
    10: "rank counts identical keys as before",
    11: "multiset digest ignores the first element",
    12: "first_unsorted flags equal neighbours",
    13: "multiset digest ignores the high half of a word",
    14: "two-word recursion sorts the lower side in the wrong direction",
}


@pytest.mark.parametrize("plant", sorted(PLANTS), ids=lambda k: PLANTS[k].replace(" ", "_"))
def test_planted_mistake_is_caught(plant, tmp_path):
    lib = O.build_planted(plant, str(tmp_path / ("liboracle_p%d.so" % plant)))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, BSORT_ORACLE_LIB=lib,
               PYTHONPATH=os.pathsep.join([root, os.path.join(root, "tests")]))
    out = subprocess.run([sys.executable, "-c", "import oracle_pins as P; print(P.failing())"],
                         env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    failed = eval(out.stdout.strip().splitlines()[-1])
    assert failed, "planted mistake %d (%s) passed every pin" % (plant, PLANTS[plant])
