"""Flow past a circular cylinder (Section VI) on the GPU: the device mask is
bit-exact with the oracle's, the solver matches the FP64 oracle on the
smallest resolution of the convergence study for every force scheme, and the
batched convergence study produces finite drag coefficients with DRTT
tracking B (P11: DRTT equals B in exact arithmetic when the box encloses the
body)."""
import numpy as np
import pytest

import oracle
from paper_2210_10377_gb300 import inputs

pytestmark = pytest.mark.gpu

SCHEMES = ("A", "B", "DRTT", "A_RTT", "SI")
ORACLE_SCHEME = {"A": oracle.SCHEME_A, "B": oracle.SCHEME_B, "DRTT": oracle.SCHEME_DRTT,
                 "A_RTT": oracle.SCHEME_A_RTT, "SI": oracle.SCHEME_SI}


@pytest.fixture(scope="module")
def gb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_10377_gb300 import binding
    binding.lib()
    return binding


@pytest.mark.parametrize("nx,ny,xc,yc,d", [(600, 50, 150.0, 24.5, 10.0), (2400, 200, 600.0, 99.5, 40.0),
                                           (97, 61, 40.3, 29.7, 13.7), (33, 17, 0.0, 0.0, 9.0)])
def test_cylinder_mask_bit_exact(gb, nx, ny, xc, yc, d):
    assert np.array_equal(gb.cylinder_mask(nx, ny, xc, yc, d), oracle.cylinder_mask(nx, ny, xc, yc, d))


def test_smallest_resolution_matches_oracle_f64(gb):
    w = inputs.cylinder(10)
    m = oracle.cylinder_mask(w.nx, w.ny, w.xc, w.yc, w.chord)
    sim = oracle.Sim(m, w.tau, w.u_in)
    lat = gb.Lattice(m, w.tau, w.u_in, storage="f64")
    for n in (1, 15, 484):
        sim.step(n)
        lat.step(n)
    assert np.abs(lat.populations() - sim.populations()).max() <= 1e-12
    for s in SCHEMES:
        ox, oy = sim.force_series(ORACLE_SCHEME[s])
        gx, gy = lat.force_series(s)
        assert np.abs(gx - ox).max() <= 1e-11 and np.abs(gy - oy).max() <= 1e-11, s
    lat.close()


def test_convergence_study_runs_and_drtt_tracks_b(gb):
    from paper_2210_10377_gb300 import cylinder
    out = cylinder.cd_study(diameters=(10, 15, 20), flow_times=20.0, window_flow_times=5.0)
    assert out["unstable_domains"] == 0 and len(out["rows"]) == 3
    for row in out["rows"]:
        for s in cylinder.SCHEMES:
            assert np.isfinite(row["Cd_" + s]) and row["Cd_" + s] > 0, (row["D"], s)
        assert abs(row["Cd_DRTT"] - row["Cd_B"]) <= 1e-3 * row["Cd_B"], row


def test_cd_against_reynolds_number_runs(gb):
    from paper_2210_10377_gb300 import cylinder
    out = cylinder.cd_vs_re(d=10, res=(40.0, 100.0), flow_times=20.0, window_flow_times=5.0)
    assert out["unstable_domains"] == 0 and [r["Re"] for r in out["rows"]] == [40.0, 100.0]
    for row in out["rows"]:
        for s in cylinder.SCHEMES:
            assert np.isfinite(row["Cd_" + s]) and row["Cd_" + s] > 0, (row["Re"], s)
        assert abs(row["Cd_DRTT"] - row["Cd_B"]) <= 1e-3 * row["Cd_B"], row
    # drag falls as the Reynolds number grows (viscous drag dominates at low Re)
    assert out["rows"][0]["Cd_B"] > out["rows"][1]["Cd_B"]
