"""The seeded input recipes that both sides use (the only module the oracle and
the CUDA path share): deterministic, within their stated ranges, and with the
workload parameters the measurements quote."""
import numpy as np

from paper_2210_10377_gb300 import inputs


def test_named_workloads():
    small, large, prec, diff = (inputs.SMALL_F64, inputs.LARGE_F32, inputs.PRECISION, inputs.DIFF)
    assert (small.nx, small.ny, small.chord, small.alpha_deg, small.xc, small.re) == (256, 128, 32.0, 0.0, 80.0, 100.0)
    assert (large.nx, large.ny, large.chord, large.alpha_deg, large.re) == (4096, 2048, 256.0, 4.0, 1000.0)
    assert (prec.nx, prec.ny, prec.chord, prec.alpha_deg, prec.re) == (8192, 4096, 512.0, 6.0, 2000.0)
    assert (diff.nx, diff.ny, diff.chord, diff.alpha_deg, diff.re) == (512, 256, 64.0, 2.0, 200.0)
    # tau = 1/2 + 3 u_in C / Re; mid-chord 5 chords from the inlet on the mid-line
    for w, tau in ((small, 0.548), (large, 0.5384), (prec, 0.5384), (diff, 0.548)):
        assert abs(w.tau - tau) < 1e-12 and w.u_in == 0.05 and w.yc == (w.ny - 1) / 2
    assert large.xc == 0.3125 * large.nx and prec.xc == 0.3125 * prec.nx
    assert (small.storage, large.storage, prec.storage, diff.storage) == ("f64", "f32dev", "f16dev", "f32dev")


def test_batch_recipe_ranges_and_determinism():
    a = inputs.batch_instances(256)
    b = inputs.batch_instances(256)
    assert a == b and len(a) == 256
    assert inputs.batch_instances(256, seed=1) != a
    for w in a:
        assert 0.08 <= w.thickness <= 0.15 and 48 <= w.chord <= 128 and w.chord == int(w.chord)
        assert -8.0 <= w.alpha_deg <= 8.0 and 100.0 <= w.re <= 1000.0
        assert (w.nx, w.ny) == (8 * w.chord, 4 * w.chord) and w.xc == 2.5 * w.chord
        assert 0.5 < w.tau <= 0.5 + 3 * 0.05 * 128 / 100
    # the 66.9 M nodes the batch measurements quote
    assert sum(w.nodes for w in a) == 66901440
    # spread: the draws are not degenerate
    c = np.array([w.chord for w in a])
    assert c.min() < 56 and c.max() > 120


def test_seeded_draws_repeat():
    assert np.array_equal(inputs.random_populations(7, 5, seed=3), inputs.random_populations(7, 5, seed=3))
    assert np.array_equal(inputs.random_inlet(9, seed=4), inputs.random_inlet(9, seed=4))
    m = inputs.random_blobs_mask(40, 20, 5, seed=6, margin_x=3)
    assert m.dtype == np.uint8 and not m[:, :3].any() and not m[:, -3:].any()
    p = inputs.perturbation(6, 4)
    assert np.all(np.abs(p - 1) <= 1e-3)
