"""Pins of the oracle's stress integration (SI) force and boundary pressure
coefficient (Section IV, Eq. stress_int; Section VI, the C_p formula) against
closed forms that the mathematics fixes:

* a linear pressure field p = (rho0 + a x)/3 at rest has no deviatoric stress,
  and on the staircase faces of a rectangular block the pressure force is
  -(a/3) (w + 1) h along x (w + 1: the distance between the fluid nodes in
  front of and behind the block);
* steady Poiseuille flow between half-way bounce-back walls: the viscous stress
  at the first fluid rows, half a node from each wall, is rho nu du/dy of the
  exact parabola, so SI on the walls is g nx (H - 1) for H fluid rows.  This
  does not depend on tau, so it pins the factor (1 - omega/2) and its sign;
* at rest the force vanishes; C_p of the linear field is a x / (3 q).
"""
import numpy as np
import pytest

import oracle


def block_sim(nx=40, ny=24, box=(12, 20, 8, 14), tau=0.8):
    m = np.zeros((ny, nx), np.uint8)
    x0, x1, y0, y1 = box
    m[y0:y1 + 1, x0:x1 + 1] = 1
    return m, oracle.Sim(m, tau, 0.0, bc=oracle.BC_PERIODIC)


def linear_state(nx, ny, ax, ay, rho0=1.0):
    f = np.zeros((9, ny, nx))
    for y in range(ny):
        for x in range(nx):
            f[:, y, x] = oracle.feq(rho0 + ax * x + ay * y, 0.0, 0.0)
    return f


@pytest.mark.parametrize("ax,ay", [(1e-3, 0.0), (0.0, -2e-3), (7e-4, 3e-4)])
def test_linear_pressure_on_a_block(ax, ay):
    nx, ny, box = 40, 24, (12, 20, 8, 14)
    m, s = block_sim(nx, ny, box)
    s.set_populations(linear_state(nx, ny, ax, ay))
    s.step(1)
    fx, fy = s.force_series(oracle.SCHEME_SI)
    x0, x1, y0, y1 = box
    assert fx[0] == pytest.approx(-(ax / 3) * (x1 - x0 + 2) * (y1 - y0 + 1), rel=1e-12, abs=1e-15)
    assert fy[0] == pytest.approx(-(ay / 3) * (y1 - y0 + 2) * (x1 - x0 + 1), rel=1e-12, abs=1e-15)


def test_pressure_coefficient_of_a_linear_field():
    nx, ny, box = 40, 24, (12, 20, 8, 14)
    m, s = block_sim(nx, ny, box)
    a, q = 1e-3, 0.5 * 0.05 ** 2
    s.set_populations(linear_state(nx, ny, a, 0.0))
    nodes, cp = s.surface_pressure(1.0 / 3.0, q)
    # the boundary fluid nodes: fluid nodes with a solid neighbour in any direction
    expect = []
    for y in range(ny):
        for x in range(nx):
            if m[y, x]:
                continue
            if any(m[(y + dy) % ny, (x + dx) % nx] for dx in (-1, 0, 1) for dy in (-1, 0, 1)):
                expect.append(y * nx + x)
    assert nodes.tolist() == expect
    xs = nodes % nx
    assert np.allclose(cp, a * xs / (3 * q), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.4])
def test_steady_poiseuille_wall_shear(tau):
    H, nx, g = 20, 8, 1e-6
    ny = H + 2
    m = np.zeros((ny, nx), np.uint8)
    m[0] = 1
    m[-1] = 1
    s = oracle.Sim(m, tau, 0.0, bc=oracle.BC_PERIODIC, body_force=(g, 0.0),
                   cv=[0, nx - 1, 1, ny - 2])
    # relax to the steady state (the slowest mode decays like exp(-nu pi^2 t / H^2))
    nu = (tau - 0.5) / 3
    steps = int(40 * H * H / (np.pi ** 2 * nu))
    s.step(steps)
    fx, fy = s.force_series(oracle.SCHEME_SI, steps - 1, 1)
    assert fx[0] == pytest.approx(g * nx * (H - 1), rel=1e-8)
    # the walls' pressure forces cancel: round-off of 2 nx face terms of p ~ 1/3
    assert abs(fy[0]) <= 1e-14 * 2 * nx / 3


def test_zero_at_rest_around_a_naca_section():
    m = oracle.naca_mask(120, 60, 40.0, 0.12, 7.0, 50.0, 29.5)
    s = oracle.Sim(m, 0.7, 0.0, bc=oracle.BC_PERIODIC)
    s.step(30)
    fx, fy = s.force_series(oracle.SCHEME_SI)
    assert np.abs(fx).max() <= 1e-15 and np.abs(fy).max() <= 1e-15
