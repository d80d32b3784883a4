"""The stored oracle fixture (tests/golden/rt_16x32_3steps.txt, written by
tests/golden/make_golden.py from the CPU oracle alone) still matches the oracle: a guard
against unintended change of the oracle's arithmetic or of the seeded inputs."""
import importlib.util
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "rt_16x32_3steps.txt")


def load_golden():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#"):
                continue
            parts = line.split()
            rows.append([float.fromhex(v) for v in parts[1:]])
    return rows


def maker():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_fixture_has_every_population():
    rows = load_golden()
    assert len(rows) == 37 and all(len(r) == 4 for r in rows)


def test_oracle_reproduces_the_fixture():
    want = load_golden()
    got = maker().compute()
    for i in range(37):
        for a, b in zip(got[i], want[i]):
            assert a == pytest.approx(b, rel=1e-14, abs=0), (i, a, b)
