"""Pins of the oracle's default control volume (the DRTT box of Eq. rtt7 and
the Appendix).

The paper runs its DRTT box around the body with a margin (the Appendix gives
index ranges for a cylinder, 1.5 D on a side) but fixes no rule for an
arbitrary body.  The reading used on both sides: the bounding box of the solid
nodes, widened on every side by m = max(4, ceil(w / 4)) nodes, w the box's
width in x (the chord's extent for an airfoil); in a channel the x range is
clipped to [1, nx - 2] (the inlet and outlet columns stay outside); a range
that would reach a periodic edge becomes the whole period.  Each case below is
worked out by hand from that rule, with bodies chosen so that a margin taken
from the height, a wrong rounding, or a missing clip would give another box.
"""
import numpy as np

import oracle


def block(nx, ny, x0, x1, y0, y1):
    m = np.zeros((ny, nx), np.uint8)
    m[y0:y1 + 1, x0:x1 + 1] = 1
    return m


def test_small_body_gets_the_minimum_margin():
    # w = 8 -> ceil(8/4) = 2 < 4 -> m = 4
    m = block(100, 60, 40, 47, 25, 30)
    assert oracle.auto_cv(m).tolist() == [36, 51, 21, 34]


def test_margin_follows_the_width_not_the_height():
    # wide and short: w = 30 -> m = ceil(30/4) = 8 (the height 3 would give 4)
    m = block(200, 80, 50, 79, 39, 41)
    assert oracle.auto_cv(m).tolist() == [42, 87, 31, 49]
    # tall and narrow: w = 3 -> m = 4 (the height 30 would give 8)
    m = block(200, 80, 50, 52, 25, 54)
    assert oracle.auto_cv(m).tolist() == [46, 56, 21, 58]


def test_margin_rounds_up():
    # w = 33 -> 33/4 = 8.25 -> m = 9; w = 32 -> m = 8
    assert oracle.auto_cv(block(300, 100, 100, 132, 50, 50)).tolist() == [91, 141, 41, 59]
    assert oracle.auto_cv(block(300, 100, 100, 131, 50, 50)).tolist() == [92, 139, 42, 58]


def test_channel_clips_x_to_the_interior_columns():
    # near the inlet: 3 - 4 = -1 -> 1; near the outlet: 56 + 4 = 60 -> nx - 2 = 58
    assert oracle.auto_cv(block(60, 40, 3, 5, 18, 20)).tolist() == [1, 9, 14, 24]
    assert oracle.auto_cv(block(60, 40, 54, 56, 18, 20)).tolist() == [50, 58, 14, 24]


def test_periodic_edges_become_the_whole_period():
    # periodic x: a range reaching column 0 (or nx - 1) is the whole period
    assert oracle.auto_cv(block(60, 40, 3, 5, 18, 20), periodic_x=True).tolist() == [0, 59, 14, 24]
    assert oracle.auto_cv(block(60, 40, 54, 56, 18, 20), periodic_x=True).tolist() == [0, 59, 14, 24]
    # one node short of the edge in periodic x: x0 = 1 stays
    assert oracle.auto_cv(block(60, 40, 5, 7, 18, 20), periodic_x=True).tolist() == [1, 11, 14, 24]
    # y always wraps: 4 - 4 = 0 < 1 -> whole height; 36 + 4 = 40 > 38 -> whole height
    assert oracle.auto_cv(block(60, 40, 20, 22, 4, 6)).tolist() == [16, 26, 0, 39]
    assert oracle.auto_cv(block(60, 40, 20, 22, 33, 35)).tolist() == [16, 26, 0, 39]
    # y0 = 5 - 4 = 1 and y1 = 34 + 4 = 38 = ny - 2 both stay
    assert oracle.auto_cv(block(60, 40, 20, 22, 5, 34)).tolist() == [16, 26, 1, 38]


def test_empty_mask_takes_the_whole_interior():
    m = np.zeros((10, 30), np.uint8)
    assert oracle.auto_cv(m).tolist() == [1, 28, 0, 9]
    assert oracle.auto_cv(m, periodic_x=True).tolist() == [0, 29, 0, 9]


def test_scattered_solids_use_their_joint_bounding_box():
    m = np.zeros((90, 200), np.uint8)
    m[20, 60] = 1
    m[50, 75] = 1  # joint box x 60..75 (w = 16 -> m = 4), y 20..50
    assert oracle.auto_cv(m).tolist() == [56, 79, 16, 54]


def test_box_encloses_every_link_of_the_naca_workloads():
    # the property DRTT = B needs (Eqs. rtt2-rtt7): every link's fluid node and
    # its solid neighbour lie inside the box, away from its faces
    from paper_2210_10377_gb300 import inputs
    for w in (inputs.SMALL_F64, inputs.DIFF, inputs.scaled(inputs.LARGE_F32, 8)):
        m = oracle.naca_mask(w.nx, w.ny, w.chord, w.thickness, w.alpha_deg, w.xc, w.yc)
        x0, x1, y0, y1 = oracle.auto_cv(m).tolist()
        n = oracle.links(m) // 8
        xs, ys = n % w.nx, n // w.nx
        assert xs.min() > x0 and xs.max() < x1 and ys.min() > y0 and ys.max() < y1
