"""The oracle against the hand-derived fixtures under tests/golden/ (each file
states its derivation and the passages it follows)."""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                yield line.split()


STEP0 = list(rows("step0_forces.txt"))


@pytest.mark.parametrize("row", STEP0, ids=[r[0] for r in STEP0])
def test_step0_link_counts_and_forces(row):
    name, nx, ny, cells = row[0], int(row[1]), int(row[2]), row[3]
    counts = [int(v) for v in row[4:12]]
    bx, by, ax, ay = (float(Fraction(v)) for v in row[12:16])
    m = np.zeros((ny, nx), np.uint8)
    for c in cells.split(";"):
        x, y = (int(v) for v in c.split(","))
        m[y, x] = 1
    s = oracle.Sim(m, 0.7, 0.05, bc=oracle.BC_PERIODIC)
    links = s.links()
    assert np.bincount(links % 8 + 1, minlength=9)[1:].tolist() == counts, name
    s.step(1)
    np.testing.assert_allclose(s.force(oracle.SCHEME_B), (bx, by), rtol=0, atol=1e-15)
    np.testing.assert_allclose(s.force(oracle.SCHEME_A), (ax, ay), rtol=0, atol=1e-15)
    # A' pairs the pre- and post-collision populations, both feq at t = 0
    np.testing.assert_allclose(s.force(oracle.SCHEME_A_RTT), (bx, by), rtol=0, atol=1e-15)
