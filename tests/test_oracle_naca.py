"""Pins of the oracle's NACA 4-digit section and its voxelisation.

The paper names the NACA0012 section (12% thickness to chord) without printing
its thickness law; the oracle uses the standard 4-digit closed form.  These
tests check it against properties of that closed form that do not come from
evaluating it: the maximum thickness t at 30% chord, the trailing-edge
thickness, the leading-edge radius 1.1019 t^2 C, the area 0.68508 t C^2 from
integrating the law term by term, and exact mirror symmetries of the grid.
"""
import math

import numpy as np
import pytest


def test_max_thickness_at_30_percent(oracle_mod):
    t = 0.12
    s = np.linspace(0.0, 1.0, 20001)
    yt = np.array([oracle_mod.naca_thickness(v, t) for v in s])
    k = int(np.argmax(yt))
    assert abs(s[k] - 0.30) < 0.01
    assert abs(2 * yt[k] - t) < 1e-4 * t * 10  # full thickness = t (to 0.1%)


def test_trailing_edge_thickness(oracle_mod):
    t = 0.12
    # open trailing edge: the coefficients sum to 0.0021, closed: 0
    assert abs(oracle_mod.naca_thickness(1.0, t) - 5 * t * 0.0021) < 1e-15
    assert abs(oracle_mod.naca_thickness(1.0, t, closed_te=True)) < 1e-15
    assert oracle_mod.naca_thickness(0.0, t) == 0.0


def test_leading_edge_radius(oracle_mod):
    # y_t^2 -> 2 r s near the nose, r = 1.1019 t^2 (chord 1)
    t = 0.15
    s = 1e-10
    r = oracle_mod.naca_thickness(s, t) ** 2 / (2 * s)
    assert abs(r / (1.1019 * t * t) - 1) < 1e-3


@pytest.mark.parametrize("alpha", [0.0, 4.0, -6.0])
def test_area_matches_integral(oracle_mod, alpha):
    # area of the section = 10 t C^2 * integral of the bracket
    #   = 10 t C^2 (0.2969*2/3 - 0.1260/2 - 0.3516/3 + 0.2843/4 - 0.1015/5)
    t, C = 0.12, 256.0
    area = 10 * t * C * C * (0.2969 * 2 / 3 - 0.1260 / 2 - 0.3516 / 3 + 0.2843 / 4 - 0.1015 / 5)
    m = oracle_mod.naca_mask(1024, 512, C, t, alpha, 400.0, 255.5)
    assert abs(m.sum() / area - 1) < 0.01


def test_alpha0_extent_and_mirror(oracle_mod):
    t, C, nx, ny, xc = 0.12, 64.0, 256, 128, 80.0
    yc = (ny - 1) / 2
    m = oracle_mod.naca_mask(nx, ny, C, t, 0.0, xc, yc)
    np.testing.assert_array_equal(m, m[::-1])  # mirror-exact about y = yc
    ys, xs = np.nonzero(m)
    # with yc half-integer no node lies on the chord line, so the sharp ends are
    # trimmed where the half-thickness drops below half a node
    assert math.ceil(xc - C / 2) <= xs.min() <= math.ceil(xc - C / 2) + 1
    assert math.floor(xc + C / 2) - 4 <= xs.max() <= math.floor(xc + C / 2)
    assert abs(m.sum(axis=0).max() - t * C) <= 1.0  # thickest column spans ~ t*C nodes


def test_thickest_columns_near_30_percent(oracle_mod):
    t, C, nx, ny, xc = 0.12, 256.0, 512, 128, 200.0
    m = oracle_mod.naca_mask(nx, ny, C, t, 0.0, xc, (ny - 1) / 2)
    span = m.sum(axis=0)
    plateau = np.nonzero(span == span.max())[0]
    assert abs(plateau.mean() - (xc - C / 2 + 0.3 * C)) <= 0.05 * C
    assert abs(span.max() - t * C) <= 1.0


@pytest.mark.parametrize("alpha", [3.0, 6.0, 8.0])
def test_negative_alpha_is_mirror_image(oracle_mod, alpha):
    nx, ny = 300, 160
    yc = (ny - 1) / 2
    mp = oracle_mod.naca_mask(nx, ny, 100.0, 0.12, alpha, 120.0, yc)
    mn = oracle_mod.naca_mask(nx, ny, 100.0, 0.12, -alpha, 120.0, yc)
    np.testing.assert_array_equal(mn, mp[::-1])


def test_positive_alpha_is_nose_up(oracle_mod):
    nx, ny, C = 400, 200, 160.0
    yc = (ny - 1) / 2
    m = oracle_mod.naca_mask(nx, ny, C, 0.12, 10.0, 200.0, yc)
    ys, xs = np.nonzero(m)
    lead = ys[xs <= xs.min() + 2].mean()
    trail = ys[xs >= xs.max() - 2].mean()
    # leading edge rotated up by (C/2) sin(alpha), trailing edge down
    assert lead - yc == pytest.approx(C / 2 * math.sin(math.radians(10)), abs=2.0)
    assert trail - yc == pytest.approx(-C / 2 * math.sin(math.radians(10)), abs=2.0)
