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


PREFIX = [("naca0012_4096x2048_c256_a4_re1000_f32", "naca0012_4096x2048_c256_a4_re1000_oracle_prefix5000.txt"),
          ("naca0012_8192x4096_c512_a6_re2000_f16dev", "naca0012_8192x4096_c512_a6_re2000_oracle_prefix1000.txt")]


@pytest.mark.parametrize("name,fixture", PREFIX, ids=["4096x2048", "8192x4096"])
def test_stored_prefix_series_obey_the_paper(name, fixture):
    # The stored full-size oracle series (written by make_prefix_series.py) hold
    # what the paper fixes: DRTT equals B every step (Eqs. rtt2-rtt7: the box
    # encloses the body, no body force), A' equals B at t = 0, A(0) = 0 for a
    # closed body, and B(0) = 2 sum_i n_i c_i feq_i from the link counts.
    from paper_2210_10377_gb300 import inputs
    rows = np.loadtxt(os.path.join(GOLDEN, fixture))
    assert rows.shape[1] == 11 and rows[0, 0] == 0
    scale = np.abs(rows[:, 1:]).max()
    ax, ay, bx, by, dx, dy, px, py = (rows[:, k] for k in range(1, 9))
    # to the round-off of J(t) - J(t+1): serial FP64 sums of ~1e5 momenta rho u
    # over the box, a few 1e-10 at most; a missing flux term would be O(1e-3)
    assert np.abs(dx - bx).max() <= 1e-8 * scale and np.abs(dy - by).max() <= 1e-8 * scale
    assert abs(px[0] - bx[0]) <= 1e-13 * scale and abs(py[0] - by[0]) <= 1e-13 * scale
    assert abs(ax[0]) <= 1e-13 * scale and abs(ay[0]) <= 1e-13 * scale
    w = inputs.WORKLOADS[name]
    m = oracle.naca_mask(w.nx, w.ny, w.chord, w.thickness, w.alpha_deg, w.xc, w.yc)
    n = np.bincount(oracle.links(m, periodic_x=False) % 8 + 1, minlength=9)
    cx = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    cy = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
    feq = oracle.feq(w.rho0, w.u_in, 0.0)
    # the file stores 13 significant digits (5e-13 relative)
    assert abs(bx[0] - 2 * (n * cx * feq).sum()) <= 1e-12 * scale
    assert abs(by[0] - 2 * (n * cy * feq).sum()) <= 1e-12 * scale


def test_prefix_series_generator_writes_the_oracle_series(tmp_path):
    # the generator of the stored series, run on the small differentiation
    # workload: its rows are the oracle's own series at the stored steps
    import subprocess
    import sys
    from paper_2210_10377_gb300 import inputs
    name = inputs.DIFF.name
    out = tmp_path / "series.txt"
    script = os.path.join(GOLDEN, "make_prefix_series.py")
    r = subprocess.run([sys.executable, script, name, "12", "4", str(out)], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    rows = np.loadtxt(out)
    assert rows[:, 0].tolist() == [0, 4, 8]
    w = inputs.DIFF
    sim = oracle.Sim(oracle.naca_mask(w.nx, w.ny, w.chord, w.thickness, w.alpha_deg, w.xc, w.yc), w.tau, w.u_in)
    sim.step(13)
    for j, k in enumerate((oracle.SCHEME_A, oracle.SCHEME_B, oracle.SCHEME_DRTT, oracle.SCHEME_A_RTT,
                           oracle.SCHEME_SI)):
        fx, fy = sim.force_series(k, 0, 12)
        np.testing.assert_allclose(rows[:, 1 + 2 * j], fx[[0, 4, 8]], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(rows[:, 2 + 2 * j], fy[[0, 4, 8]], rtol=1e-12, atol=1e-14)
