"""The oracle reproduces its stored end states for the 32x32 torus (tests/golden/)."""
import json
import os
import sys

from conftest import GOLDEN

sys.path.insert(0, GOLDEN)


def test_small_torus_golden():
    import make_golden
    with open(os.path.join(GOLDEN, "small_torus.json")) as f:
        stored = json.load(f)
    assert make_golden.compute() == stored
