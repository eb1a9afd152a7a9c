"""Pins of the oracle's lattice and equilibrium against exact identities.

Section II of the paper (Table tabD2Q9 and the moment conditions that follow
the second-order equilibrium) fixes the D2Q9 set, its weights and the first
moments of feq.  Rational arithmetic makes the weight identities exact.
"""
from fractions import Fraction as Fr
import itertools

import numpy as np
import pytest


def test_velocity_set_and_opposites(oracle_mod):
    cx, cy, w, opp = oracle_mod.lattice()
    vecs = set(zip(cx.tolist(), cy.tolist()))
    assert vecs == set(itertools.product((-1, 0, 1), repeat=2))
    assert (cx[0], cy[0]) == (0, 0)
    for i in range(9):
        assert cx[opp[i]] == -cx[i] and cy[opp[i]] == -cy[i]
    # energy shells of Table tabD2Q9: zero, SC-1 (|c|^2 = 1), FCC-1 (|c|^2 = 2)
    shells = cx * cx + cy * cy
    assert sorted(shells.tolist()) == [0, 1, 1, 1, 1, 2, 2, 2, 2]


def test_weights_are_table_values(oracle_mod):
    cx, cy, w, _ = oracle_mod.lattice()
    table = {0: Fr(16, 36), 1: Fr(4, 36), 2: Fr(1, 36)}
    for i in range(9):
        assert w[i] == float(table[cx[i] ** 2 + cy[i] ** 2])


def test_weight_moments_exact():
    # P1 with the rational weights of the table: sum w = 1, sum w c c = theta0 delta,
    # sum w cccc = theta0^2 Delta (Delta = symmetric isotropic 4th-rank tensor)
    import oracle
    cx, cy, w, _ = oracle.lattice()
    wr = [Fr(16, 36) if cx[i] ** 2 + cy[i] ** 2 == 0 else
          Fr(4, 36) if cx[i] ** 2 + cy[i] ** 2 == 1 else Fr(1, 36) for i in range(9)]
    c = [(int(cx[i]), int(cy[i])) for i in range(9)]
    th = Fr(1, 3)
    assert sum(wr) == 1
    for a in range(2):
        for b in range(2):
            assert sum(wr[i] * c[i][a] * c[i][b] for i in range(9)) == th * (a == b)
    for a, b, g, d in itertools.product(range(2), repeat=4):
        lhs = sum(wr[i] * c[i][a] * c[i][b] * c[i][g] * c[i][d] for i in range(9))
        delta = (a == b) * (g == d) + (a == g) * (b == d) + (a == d) * (b == g)
        assert lhs == th * th * delta
    # odd moments vanish
    for a in range(2):
        assert sum(wr[i] * c[i][a] for i in range(9)) == 0


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_equilibrium_moments(oracle_mod, seed):
    # P2: sum feq = rho, sum c feq = rho u, sum cc feq = rho uu + rho theta0 I
    g = np.random.default_rng(seed)
    cx, cy, _, _ = oracle_mod.lattice()
    rho = g.uniform(0.8, 1.2)
    ux, uy = g.uniform(-0.1, 0.1, 2)
    f = oracle_mod.feq(rho, ux, uy)
    assert abs(f.sum() - rho) < 1e-15
    assert abs((cx * f).sum() - rho * ux) < 1e-15
    assert abs((cy * f).sum() - rho * uy) < 1e-15
    assert abs((cx * cx * f).sum() - (rho * ux * ux + rho / 3)) < 1e-15
    assert abs((cy * cy * f).sum() - (rho * uy * uy + rho / 3)) < 1e-15
    assert abs((cx * cy * f).sum() - rho * ux * uy) < 1e-15
    # third moment Q_xxy = rho u_y / 3 (a D2Q9 property of the second-order feq)
    assert abs((cx * cx * cy * f).sum() - rho * uy / 3) < 1e-15


def test_equilibrium_rest_state_and_value(oracle_mod):
    _, _, w, _ = oracle_mod.lattice()
    np.testing.assert_array_equal(oracle_mod.feq(1.0, 0.0, 0.0), w)
    # hand value: feq_1(rho=1, u=(0.05,0)) = (1/9)(1 + 0.15 + 4.5*0.0025 - 1.5*0.0025)
    assert abs(oracle_mod.feq(1.0, 0.05, 0.0)[1] - 1.1575 / 9) < 1e-16
