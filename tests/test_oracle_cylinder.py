"""Pins of the oracle's circular-cylinder mask (Section VI) against hand counts
and the lattice-point bounds of a disc."""
import math

import numpy as np
import pytest

import oracle
from paper_2210_10377_gb300 import inputs


@pytest.mark.parametrize("d,count", [(2.0, 5), (3.0, 9), (4.0, 13)])
def test_small_discs_by_hand(d, count):
    # r = 1: centre + 4 axis neighbours; r = 1.5: the 3 x 3 block (diagonals at
    # sqrt 2); r = 2: adds the 4 nodes at distance 2
    m = oracle.cylinder_mask(11, 11, 5.0, 5.0, d)
    assert int(m.sum()) == count
    assert m[5, 5] == 1


@pytest.mark.parametrize("d", [10.0, 15.0, 27.0, 40.0])
def test_disc_count_bounds_and_symmetry(d):
    r = d / 2
    n = int(6 * d)
    m = oracle.cylinder_mask(n, n, (n - 1) / 2, (n - 1) / 2, d)
    # unit squares centred on the nodes inside the disc lie within r + sqrt(2)/2
    # and cover the disc of radius r - sqrt(2)/2
    lo, hi = math.pi * (r - math.sqrt(0.5)) ** 2, math.pi * (r + math.sqrt(0.5)) ** 2
    assert lo <= m.sum() <= hi
    assert np.array_equal(m, m[::-1, :]) and np.array_equal(m, m[:, ::-1])
    assert np.array_equal(m, m.T)
    # every node at distance <= r is solid, every node beyond is fluid
    yy, xx = np.mgrid[0:n, 0:n]
    dist2 = (xx - (n - 1) / 2) ** 2 + (yy - (n - 1) / 2) ** 2
    assert np.array_equal(m.astype(bool), dist2 <= r * r)


def test_workload_recipe_geometry():
    w = inputs.cylinder(20)
    assert (w.nx, w.ny, w.chord, w.xc, w.re) == (1200, 100, 20.0, 300.0, 100.0)
    assert w.tau == pytest.approx(0.5 + 3 * 0.05 * 20 / 100)
    m = oracle.cylinder_mask(w.nx, w.ny, w.xc, w.yc, w.chord)
    ys, xs = np.nonzero(m)
    # centre (300, 49.5): the rows nearest the centre are half a node away, so
    # the solid extends |dx| <= sqrt(10^2 - 0.5^2) = 9.99 about x = 15 d
    assert xs.min() == 291 and xs.max() == 309
    assert np.array_equal(m, m[::-1, :])  # on the mid-line
    links = oracle.links(m)
    cnt = np.bincount(links % 8 + 1, minlength=9)
    opp = [0, 3, 4, 1, 2, 7, 8, 5, 6]
    assert all(cnt[i] == cnt[opp[i]] for i in range(1, 9))
