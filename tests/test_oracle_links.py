"""Pins of the oracle's fluid-solid link list.

A link is a pair (x_f, i) with x_f fluid and x_f + c_i solid (the halfway
bounce-back set-up of Section II and Fig. basicLadd).  Small cases are listed
by hand; larger random masks are checked against a solid-centred brute force,
which enumerates the same set from the other end of each link.
"""
import numpy as np
import pytest

from paper_2210_10377_gb300 import inputs

# direction order: 0 rest, 1 (1,0), 2 (0,1), 3 (-1,0), 4 (0,-1), 5 (1,1), 6 (-1,1), 7 (-1,-1), 8 (1,-1)
C = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]


def pack(x, y, i, nx):
    return (y * nx + x) * 8 + (i - 1)


def test_single_solid_node_hand_listed(oracle_mod):
    nx = ny = 8
    m = np.zeros((ny, nx), np.uint8)
    m[3, 3] = 1
    got = oracle_mod.links(m, periodic_x=True).tolist()
    # each of the 8 neighbours has exactly one link, pointing at (3, 3)
    want = sorted([
        pack(2, 3, 1, nx),  # west neighbour, direction (1,0)
        pack(3, 2, 2, nx),  # south neighbour, (0,1)
        pack(4, 3, 3, nx),  # east neighbour, (-1,0)
        pack(3, 4, 4, nx),  # north neighbour, (0,-1)
        pack(2, 2, 5, nx),  # south-west, (1,1)
        pack(4, 2, 6, nx),  # south-east, (-1,1)
        pack(4, 4, 7, nx),  # north-east, (-1,-1)
        pack(2, 4, 8, nx),  # north-west, (1,-1)
    ])
    assert got == want


def test_two_node_block_hand_listed(oracle_mod):
    nx, ny = 6, 5
    m = np.zeros((ny, nx), np.uint8)
    m[2, 2] = m[2, 3] = 1
    got = oracle_mod.links(m, periodic_x=False).tolist()
    want = sorted([
        pack(1, 1, 5, nx), pack(2, 1, 2, nx), pack(2, 1, 5, nx), pack(3, 1, 2, nx),
        pack(3, 1, 6, nx), pack(4, 1, 6, nx),
        pack(1, 2, 1, nx), pack(4, 2, 3, nx),
        pack(1, 3, 8, nx), pack(2, 3, 4, nx), pack(2, 3, 8, nx), pack(3, 3, 4, nx),
        pack(3, 3, 7, nx), pack(4, 3, 7, nx),
    ])
    assert got == want


def test_wrap_in_y_but_not_x_for_channel(oracle_mod):
    nx, ny = 5, 4
    m = np.zeros((ny, nx), np.uint8)
    m[0, 4] = 1  # bottom-right corner
    ch = set(oracle_mod.links(m, periodic_x=False).tolist())
    per = set(oracle_mod.links(m, periodic_x=True).tolist())
    # through the top boundary (y wraps): (4,3) direction (0,1) and (3,3) direction (1,1)
    assert pack(4, 3, 2, nx) in ch and pack(3, 3, 5, nx) in ch
    # through the right boundary only when x is periodic: (0,0) direction (-1,0)
    assert pack(0, 0, 3, nx) not in ch and pack(0, 0, 3, nx) in per
    assert len(ch) == 5 and len(per) == 8


def brute_links(mask, periodic_x):
    ny, nx = mask.shape
    out = set()
    for ys, xs in zip(*np.nonzero(mask)):
        for i in range(1, 9):
            xf, yf = xs - C[i][0], (ys - C[i][1]) % ny
            if not (0 <= xf < nx):
                if not periodic_x:
                    continue
                xf %= nx
            if not mask[yf, xf]:
                out.add(pack(xf, yf, i, nx))
    return sorted(out)


@pytest.mark.parametrize("seed,periodic", [(1, False), (2, True), (3, False)])
def test_random_masks_against_brute_force(oracle_mod, seed, periodic):
    m = inputs.random_blobs_mask(37, 23, 6, seed, max_radius=3.0, margin_x=0 if periodic else 2)
    got = oracle_mod.links(m, periodic_x=periodic)
    assert got.tolist() == brute_links(m, periodic)
    assert np.all(np.diff(got) > 0)


def test_closed_body_has_symmetric_link_counts(oracle_mod):
    # every lattice line through a closed body enters and leaves it: n_i = n_opp(i)
    m = oracle_mod.naca_mask(256, 128, 32.0, 0.12, 7.0, 80.0, 63.5)
    lk = oracle_mod.links(m)
    counts = np.bincount(lk % 8 + 1, minlength=9)
    for i, o in [(1, 3), (2, 4), (5, 7), (6, 8)]:
        assert counts[i] == counts[o]
