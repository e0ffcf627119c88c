"""The oracle still reproduces its committed regression fixture: R(Q) at 24 sampled cells of a seeded
warped-grid Navier-Stokes case, written by tests/golden/make_golden.py from the oracle alone."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))


def test_oracle_regression_fixture():
    import make_golden
    cells, R = make_golden.fixture()
    rows = np.loadtxt(os.path.join(HERE, "golden", "oracle_residual_warped.txt"))
    assert len(rows) == len(cells)
    for row in rows:
        k, j, i = (int(v) for v in row[:3])
        ref = row[3:]
        got = R[:, k, j, i]
        assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))
