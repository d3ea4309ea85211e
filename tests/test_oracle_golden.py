"""The oracle reproduces its committed regression fixtures exactly (the
fixtures are written by tests/golden/make_golden.py from the oracle alone;
a change to the oracle's arithmetic must regenerate them and say why)."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402
from paper_1006_0252_gb300 import inputs  # noqa: E402


def _load(name):
    with open(os.path.join(HERE, "golden", name)) as f:
        return json.load(f)["rows"]


def test_oracle_reproduces_l4_prefix():
    want = _load("oracle_l4_prefix.json")
    got = make_golden.trajectory(inputs.config_small_3d()[0], len(want) - 1)
    assert got == want


def test_oracle_reproduces_chain96():
    want = _load("oracle_chain96.json")
    chain = inputs.RunSpec(1, 96, 2, 7, 500, inputs.linear_schedule(4.0, 41), 5)
    got = make_golden.trajectory(chain, len(want) - 1)
    assert got == want
