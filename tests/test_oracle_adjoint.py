"""Pins of the oracle's discrete adjoint against central finite differences of
the oracle's own forward solver (a separate code path: the forward step of the
solver versus the transposed, entry-by-entry Jacobians of the adjoint).

Objective: the window average of wx Fx + wy Fy, F the algorithm-B force
(Eq. rtt5 with bounce-back), after `steps` steps of the channel set-up from a
given initial state."""
import numpy as np
import pytest

from paper_2210_10377_gb300 import inputs


def case(seed):
    ny, nx = 18, 34
    m = np.zeros((ny, nx), np.uint8)
    m[6:11, 12:17] = inputs.random_blobs_mask(5, 5, 3, seed=seed, max_radius=2.0, margin_x=0)
    m[8, 14] = 1
    u = inputs.random_inlet(ny, seed=seed + 1)
    return m, u


def forward_J(oracle_mod, m, tau, u, f0, steps, window, wx, wy):
    s = oracle_mod.Sim(m, tau, u)
    s.set_populations(f0)
    s.step(steps)
    fx, fy = s.force_series(oracle_mod.SCHEME_B)
    return float((wx * fx[steps - window:] + wy * fy[steps - window:]).mean())


@pytest.mark.parametrize("seed,steps,window,wx,wy",
                         [(3, 61, 30, 1.0, 0.0), (7, 50, 50, 0.0, 1.0), (11, 37, 5, 0.6, -0.8)])
def test_adjoint_matches_central_differences(oracle_mod, seed, steps, window, wx, wy):
    m, u = case(seed)
    tau = 0.66
    base = oracle_mod.Sim(m, tau, u).populations()
    f0 = base * inputs.perturbation(m.shape[1], m.shape[0], seed=seed + 2, amp=1e-3)
    J, dtau, du, df0 = oracle_mod.adjoint(m, tau, u, f0, steps, window, wx, wy)
    fJ = lambda **kw: forward_J(oracle_mod, m, kw.get("tau", tau), kw.get("u", u),
                                kw.get("f0", f0), steps, window, wx, wy)
    assert J == pytest.approx(fJ(), rel=0, abs=1e-15)
    h = 1e-5
    fd = (fJ(tau=tau + h) - fJ(tau=tau - h)) / (2 * h)
    assert dtau == pytest.approx(fd, rel=1e-6, abs=1e-10)
    for r in (0, 5, 9, m.shape[0] - 1):
        up, um = u.copy(), u.copy()
        up[r] += h
        um[r] -= h
        assert du[r] == pytest.approx((fJ(u=up) - fJ(u=um)) / (2 * h), rel=1e-6, abs=1e-10)
    g = inputs.rng(seed + 5)
    fluid = np.argwhere(m == 0)
    for k in range(6):
        y, x = fluid[g.integers(0, len(fluid))]
        i = int(g.integers(0, 9))
        fp, fm = f0.copy(), f0.copy()
        fp[i, y, x] += h
        fm[i, y, x] -= h
        fd = (fJ(f0=fp) - fJ(f0=fm)) / (2 * h)
        assert df0[i, y, x] == pytest.approx(fd, rel=1e-5, abs=1e-9), (i, y, x)
    # the initial inlet column and solid nodes do not influence J
    assert np.all(df0[:, :, 0] == 0) and np.all(df0[:, m == 1] == 0)
