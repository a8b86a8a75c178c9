"""The oracle reproduces its stored c1 summary (written by tests/golden/make_golden.py)."""
import json
import os

import pytest


def test_c1_golden(oracle_lib):
    from tests.golden.make_golden import c1_summary

    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c1_levels.json")
    want = json.load(open(here))
    got = c1_summary()
    q_sum = got.pop("q_sum")
    assert q_sum == pytest.approx(want.pop("q_sum"), rel=1e-12)
    assert got == want
