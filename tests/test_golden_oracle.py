"""The oracle still reproduces the stored snapshots under tests/golden/.

The snapshots were written by tests/golden/make_golden.py from the oracle
alone; a change to the oracle's arithmetic shows up here first.
"""
import glob
import json
import os

import pytest

from tests.golden.make_golden import snapshot

FILES = sorted(glob.glob(os.path.join(os.path.dirname(__file__), "golden", "*.json")))


@pytest.mark.parametrize("path", FILES, ids=[os.path.basename(p) for p in FILES])
def test_oracle_matches_golden(orc, path):
    with open(path) as f:
        data = json.load(f)
    assert snapshot(data["case"]) == data["snapshots"]
