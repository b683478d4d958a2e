"""The oracle against digests of its own earlier small runs
(tests/golden/oracle_regression.txt, written by make_oracle_fixtures.py from
the oracle alone): a change to the oracle's arithmetic fails here and has to
be made on purpose, with the passage that justifies it named in its commit."""
from __future__ import annotations

import importlib.util
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def _generator():
    path = os.path.join(HERE, "golden", "make_oracle_fixtures.py")
    spec = importlib.util.spec_from_file_location("make_oracle_fixtures", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_oracle_runs_match_their_recorded_digests():
    stored = {}
    with open(os.path.join(HERE, "golden", "oracle_regression.txt")) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                name, e, m, d = ln.split()
                stored[name] = (int(e), int(m), d)
    now = {name: (e, m, d) for name, e, m, d in _generator().cases()}
    assert set(now) == set(stored)
    for name in stored:
        assert now[name] == stored[name], name
