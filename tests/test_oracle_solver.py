"""Pins of the oracle's time step and force schemes.

What the paper and the mathematics fix, independently of the oracle's code:
  * conservation of mass and momentum by BGK collision and streaming (Sec. II),
  * the streaming map f(x + c_i, t+1) = ft_i(x, t) as an array shift, and the
    tau = 1 collision reducing to ft = feq (Eq. CollideAdv),
  * Taylor-Green decay exp(-2 nu k^2 t), nu = (tau - 1/2)/3, converging at
    second order,
  * steady Poiseuille flow between bounce-back walls: an exact parabola of
    curvature -g/nu, walls near the half-way points, and the wall force equal to
    the body force on the fluid (global momentum balance, Eq. rtt2),
  * DRTT (Eq. rtt7) equal to algorithm B (Eq. rtt5 with bounce-back) for any
    control volume enclosing the body, every step, in exact arithmetic,
  * B - A' equal to the collision increment on the links (Eq. lbb3 / rtt4),
  * step-0 closed forms and the mirror symmetry of an alpha = 0 section,
  * a pull-form brute force on tiny channels (inlet, outlet, bounce-back),
  * bit-exact checkpoint / resume.
"""
import math

import numpy as np
import pytest

from paper_2210_10377_gb300 import inputs

A, B, DRTT, AP = 0, 1, 2, 3


def lattice(oracle_mod):
    cx, cy, w, opp = oracle_mod.lattice()
    return cx.astype(np.int64), cy.astype(np.int64), w, opp


def feq_field(oracle_mod, rho, ux, uy):
    ny, nx = ux.shape
    f = np.zeros((9, ny, nx))
    for j in range(ny):
        for i in range(nx):
            f[:, j, i] = oracle_mod.feq(rho[j, i], ux[j, i], uy[j, i])
    return f


# ----------------------------------------------------------------------------- conservation

def test_mass_conserved_periodic_with_body(oracle_mod):
    # P4: bounce-back only swaps populations within a node, streaming permutes them
    m = inputs.random_blobs_mask(40, 30, 5, seed=11, margin_x=0)
    s = oracle_mod.Sim(m, 0.56, 0.0, bc=oracle_mod.BC_PERIODIC)
    f0 = inputs.random_populations(40, 30, seed=12) * (1 - m)[None]
    s.set_populations(f0)
    m0 = s.populations().sum()
    for _ in range(20):
        s.step(10)
        assert abs(s.populations().sum() - m0) < 1e-12 * m0


def test_momentum_conserved_without_body(oracle_mod):
    # P3: BGK collision conserves rho u per node; streaming conserves the total
    cx, cy, _, _ = lattice(oracle_mod)
    m = np.zeros((24, 32), np.uint8)
    s = oracle_mod.Sim(m, 0.7, 0.0, bc=oracle_mod.BC_PERIODIC)
    s.set_populations(inputs.random_populations(32, 24, seed=5))
    f = s.populations()
    j0 = np.array([(cx[:, None, None] * f).sum(), (cy[:, None, None] * f).sum()])
    s.step(50)
    f = s.populations()
    j1 = np.array([(cx[:, None, None] * f).sum(), (cy[:, None, None] * f).sum()])
    assert np.abs(j1 - j0).max() < 1e-12


def test_body_force_adds_momentum(oracle_mod):
    cx, cy, _, _ = lattice(oracle_mod)
    m = np.zeros((10, 12), np.uint8)
    g = np.array([2e-5, -1e-5])
    s = oracle_mod.Sim(m, 0.9, 0.0, bc=oracle_mod.BC_PERIODIC, body_force=g)
    s.set_populations(inputs.random_populations(12, 10, seed=6))
    mom = lambda f: np.array([(cx[:, None, None] * f).sum(), (cy[:, None, None] * f).sum()])
    j0 = mom(s.populations())
    s.step(7)
    np.testing.assert_allclose(mom(s.populations()) - j0, 7 * 120 * g, rtol=0, atol=1e-13)


# ----------------------------------------------------------------------------- stream / collide

def test_streaming_is_a_shift_and_tau1_collision_is_feq(oracle_mod):
    # f(x + c_i, t+1) = ft_i(x, t) with ft = feq(rho, u) when tau = 1 (omega = 1)
    cx, cy, _, _ = lattice(oracle_mod)
    nx, ny = 9, 7
    m = np.zeros((ny, nx), np.uint8)
    s = oracle_mod.Sim(m, 1.0, 0.0, bc=oracle_mod.BC_PERIODIC)
    f = inputs.random_populations(nx, ny, seed=3)
    s.set_populations(f)
    s.step(1)
    rho = f.sum(0)
    ux = (cx[:, None, None] * f).sum(0) / rho
    uy = (cy[:, None, None] * f).sum(0) / rho
    ft = feq_field(oracle_mod, rho, ux, uy)
    want = np.stack([np.roll(ft[i], shift=(cy[i], cx[i]), axis=(0, 1)) for i in range(9)])
    np.testing.assert_allclose(s.populations(), want, rtol=0, atol=1e-16)


def test_collide_then_stream_equals_stream_then_collide(oracle_mod):
    # Eqs. CollideAdv / AdvCollide: with no boundary the two orders give the same
    # trajectory; the stream-then-collide sequence is the post-collision states.
    cx, cy, _, _ = lattice(oracle_mod)
    nx, ny, tau = 8, 6, 0.73
    om = 1 / tau
    m = np.zeros((ny, nx), np.uint8)
    f0 = inputs.random_populations(nx, ny, seed=21)

    def collide(f):
        rho = f.sum(0)
        ux = (cx[:, None, None] * f).sum(0) / rho
        uy = (cy[:, None, None] * f).sum(0) / rho
        return f + om * (feq_field(oracle_mod, rho, ux, uy) - f)

    def stream(f):
        return np.stack([np.roll(f[i], shift=(cy[i], cx[i]), axis=(0, 1)) for i in range(9)])

    g = collide(f0)  # stream-then-collide sequence started from ft(0)
    s = oracle_mod.Sim(m, tau, 0.0, bc=oracle_mod.BC_PERIODIC)
    s.set_populations(f0)
    for _ in range(4):
        s.step(1)
        g = collide(stream(g))
        np.testing.assert_allclose(collide(s.populations()), g, rtol=0, atol=1e-15)


# ----------------------------------------------------------------------------- Taylor-Green

def taylor_green_rate_error(oracle_mod, N, tau, u0=1e-3):
    cx, cy, _, _ = lattice(oracle_mod)
    k = 2 * math.pi / N
    nu = (tau - 0.5) / 3
    y, x = np.mgrid[0:N, 0:N]
    ux = u0 * np.sin(k * x) * np.cos(k * y)
    uy = -u0 * np.cos(k * x) * np.sin(k * y)
    s = oracle_mod.Sim(np.zeros((N, N), np.uint8), tau, 0.0, bc=oracle_mod.BC_PERIODIC)
    s.set_populations(feq_field(oracle_mod, np.ones((N, N)), ux, uy))
    basis = np.sin(k * x) * np.cos(k * y)

    def amp():
        f = s.populations()
        u = (cx[:, None, None] * f).sum(0) / f.sum(0)
        return (u * basis).sum() / (basis * basis).sum()

    T = int(0.5 / (2 * nu * k * k))
    s.step(10)
    a1 = amp()
    s.step(T)
    a2 = amp()
    return -math.log(a2 / a1) / T / (2 * nu * k * k) - 1


@pytest.mark.parametrize("tau", [0.8, 1.2])
def test_taylor_green_decay_second_order(oracle_mod, tau):
    # P6: amplitude ~ exp(-2 nu k^2 t), error O(k^2)
    e32 = taylor_green_rate_error(oracle_mod, 32, tau)
    e64 = taylor_green_rate_error(oracle_mod, 64, tau)
    assert abs(e32) < 0.01
    assert 3.0 < e32 / e64 < 5.0


# ----------------------------------------------------------------------------- Poiseuille

@pytest.mark.parametrize("tau", [0.6, 1.0])
def test_poiseuille_between_bounce_back_walls(oracle_mod, tau):
    # P7 / P8: solid rows 0 and ny-1, periodic x, body force g along x
    cx, _, _, _ = lattice(oracle_mod)
    nx, ny, g = 3, 20, 1e-6
    nu = (tau - 0.5) / 3
    m = np.zeros((ny, nx), np.uint8)
    m[0] = m[-1] = 1
    s = oracle_mod.Sim(m, tau, 0.0, bc=oracle_mod.BC_PERIODIC, body_force=[g, 0.0],
                       cv=[0, nx - 1, 1, ny - 2])
    s.step(int(4 * (ny - 2) ** 2 / nu))
    f = s.populations()[:, 1:-1, 1]
    u = (cx[:, None] * f).sum(0) / f.sum(0)
    np.testing.assert_allclose(u, u[::-1], rtol=1e-10)
    d2 = u[2:] - 2 * u[1:-1] + u[:-2]
    np.testing.assert_allclose(d2, -g / nu, rtol=1e-7)  # exact parabola of the NS limit
    assert np.abs(np.diff(u, 3)).max() < 1e-9 * u.max()
    # walls where the parabola vanishes: near the half-way points y = 0.5, ny - 1.5
    y = np.arange(1, ny - 1)
    a = g / (2 * nu)
    S, P = np.linalg.lstsq(np.vstack([y, np.ones_like(y)]).T, u + a * y * y, rcond=None)[0]
    S, P = S / a, -P / a
    disc = math.sqrt(S * S - 4 * P)
    assert abs((S - disc) / 2 - 0.5) < 0.03 and abs((S + disc) / 2 - (ny - 1.5)) < 0.03
    # steady wall force = body force on all fluid nodes (algorithm B and DRTT + source)
    n_fluid = nx * (ny - 2)
    fx, fy = s.force(B)
    assert abs(fx / (g * n_fluid) - 1) < 1e-8 and abs(fy) < 1e-15
    dx, _ = s.force(DRTT)
    # the control volume holds every fluid node: DRTT misses exactly the source g N_V
    assert abs(dx + g * n_fluid - fx) < 1e-15
    # algorithm A does not give the wall force: it misses the collision increment
    assert abs(s.force(A)[0] / fx - 1) > 0.5


# ----------------------------------------------------------------------------- forces

def naca_small(oracle_mod, alpha=0.0):
    w = inputs.SMALL_F64
    return oracle_mod.naca_mask(w.nx, w.ny, w.chord, w.thickness, alpha, w.xc, w.yc), w


def test_drtt_equals_b_every_step_channel(oracle_mod):
    # P11 on the small NACA channel: J(t) - J(t+1) + gained - lost = 2 sum c ft
    m, w = naca_small(oracle_mod, 5.0)
    s = oracle_mod.Sim(m, w.tau, w.u_in)
    s.step(300)
    bx, by = s.force_series(B)
    dx, dy = s.force_series(DRTT)
    assert np.abs(dx - bx).max() < 1e-12 and np.abs(dy - by).max() < 1e-12
    assert np.abs(bx).max() > 1e-2


def test_drtt_equals_b_random_bodies_and_boxes(oracle_mod):
    nx, ny = 48, 30
    m = np.zeros((ny, nx), np.uint8)
    m[8:20, 14:30] = inputs.random_blobs_mask(16, 12, 4, seed=8, max_radius=3.0, margin_x=0)
    u_in = inputs.random_inlet(ny, seed=9)
    f0 = inputs.random_populations(nx, ny, seed=10, lo=0.05, hi=0.15)
    series = []
    for cv in ([10, 35, 4, 25], [12, 32, 6, 22], None):
        s = oracle_mod.Sim(m, 0.62, u_in, cv=cv)
        s.set_populations(f0)
        s.step(60)
        bx, by = s.force_series(B)
        dx, dy = s.force_series(DRTT)
        assert np.abs(dx - bx).max() < 1e-12 and np.abs(dy - by).max() < 1e-12
        series.append(dx)
    # and a box that cuts through the body does not balance
    s = oracle_mod.Sim(m, 0.62, u_in, cv=[10, 20, 4, 25])
    s.set_populations(f0)
    s.step(5)
    assert np.abs(s.force_series(DRTT)[0] - s.force_series(B)[0]).max() > 1e-4


def test_b_minus_a_prime_is_collision_increment(oracle_mod):
    # P10 (Eq. lbb3 / rtt4): B - A' = sum_links c_i (ft_i - f_i)(x_f, t)
    cx, cy, _, _ = lattice(oracle_mod)
    m, w = naca_small(oracle_mod, 3.0)
    s = oracle_mod.Sim(m, w.tau, w.u_in)
    s.step(40)
    f = s.populations().reshape(9, -1)
    rho = f.sum(0)
    ok = rho > 0
    ux = np.where(ok, (cx[:, None] * f).sum(0) / np.where(ok, rho, 1), 0)
    uy = np.where(ok, (cy[:, None] * f).sum(0) / np.where(ok, rho, 1), 0)
    lk = s.links()
    n, i = lk // 8, lk % 8 + 1
    inc = np.zeros(2)
    for nn, ii in zip(n, i):
        fe = oracle_mod.feq(rho[nn], ux[nn], uy[nn])[ii]
        d = (fe - f[ii, nn]) / w.tau
        inc += [cx[ii] * d, cy[ii] * d]
    s.step(1)
    b = np.array(s.force(B))
    ap = np.array(s.force(AP))
    np.testing.assert_allclose(b - ap, inc, rtol=0, atol=1e-14)


def test_step0_closed_forms_single_node(oracle_mod):
    # P12: uniform feq(rho0, u) around one solid node: 8 links, one per direction;
    # B(0) = 2 sum_i c_i feq_i = 2 rho0 u, A(0) = 0, A'(0) = B(0)
    m = np.zeros((9, 9), np.uint8)
    m[4, 4] = 1
    s = oracle_mod.Sim(m, 0.7, 0.05, bc=oracle_mod.BC_PERIODIC)
    s.step(1)
    assert s.nlinks == 8
    np.testing.assert_allclose(s.force(B), (0.1, 0.0), rtol=0, atol=1e-16)
    np.testing.assert_allclose(s.force(A), (0.0, 0.0), rtol=0, atol=1e-16)
    np.testing.assert_allclose(s.force(AP), s.force(B), rtol=0, atol=1e-16)


def test_step0_closed_forms_naca(oracle_mod):
    # closed body: n_i = n_opp(i), so A(0) = sum_i n_i c_i (feq_i + feq_opp) = 0 and
    # B(0) = 2 sum_i n_i c_i feq_i = 6 rho0 u sum_i n_i w_i c_ix^2 (x), 0 (y)
    cx, cy, wts, _ = lattice(oracle_mod)
    m, w = naca_small(oracle_mod, 0.0)
    s = oracle_mod.Sim(m, w.tau, w.u_in)
    s.step(1)
    counts = np.bincount(s.links() % 8 + 1, minlength=9)
    bx = 6 * w.u_in * (counts * wts * cx * cx).sum()
    np.testing.assert_allclose(s.force(B), (bx, 0.0), rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(s.force(A), (0.0, 0.0), atol=1e-15)


def test_body_at_rest_feels_no_force(oracle_mod):
    # P9: fluid at rest around a closed body in a periodic box
    m, _ = naca_small(oracle_mod, 9.0)
    s = oracle_mod.Sim(m, 0.6, 0.0, bc=oracle_mod.BC_PERIODIC)
    s.step(50)
    for k in (A, B, DRTT, AP):
        fx, fy = s.force_series(k)
        assert np.abs(fx).max() < 1e-14 and np.abs(fy).max() < 1e-14


def test_symmetric_section_has_no_lift_and_mirror_flips_it(oracle_mod):
    # P13
    m0, w = naca_small(oracle_mod, 0.0)
    s = oracle_mod.Sim(m0, w.tau, w.u_in)
    s.step(400)
    for k in (A, B, DRTT, AP):
        assert np.abs(s.force_series(k)[1]).max() < 1e-12
    mp, _ = naca_small(oracle_mod, 6.0)
    mn, _ = naca_small(oracle_mod, -6.0)
    sp = oracle_mod.Sim(mp, w.tau, w.u_in)
    sn = oracle_mod.Sim(mn, w.tau, w.u_in)
    sp.step(200)
    sn.step(200)
    for k in (A, B, DRTT, AP):
        fxp, fyp = sp.force_series(k)
        fxn, fyn = sn.force_series(k)
        np.testing.assert_allclose(fxn, fxp, rtol=0, atol=1e-12)
        np.testing.assert_allclose(fyn, -fyp, rtol=0, atol=1e-12)
    assert sp.force(B)[1] > 0  # nose-up section lifts


# ----------------------------------------------------------------------------- brute force

def brute_step(oracle_mod, f, mask, tau, u_in):
    """One channel step written in pull form: f_i(x, t+1) = ft_i(x - c_i, t), or the
    bounced ft_opp(x, t) when x - c_i is solid; inlet feq, outlet copy."""
    cx, cy, _, opp = lattice(oracle_mod)
    ny, nx = mask.shape
    ft = np.zeros_like(f)
    for y in range(ny):
        for x in range(nx):
            if mask[y, x]:
                continue
            if x == 0:
                ft[:, y, x] = oracle_mod.feq(1.0, u_in[y], 0.0)
                continue
            fi = f[:, y, x]
            rho = sum(fi[i] for i in range(9))
            jx = sum(cx[i] * fi[i] for i in range(9))
            jy = sum(cy[i] * fi[i] for i in range(9))
            fe = oracle_mod.feq(rho, jx / rho, jy / rho)
            ft[:, y, x] = [fi[i] + (fe[i] - fi[i]) / tau for i in range(9)]
    out = np.zeros_like(f)
    for y in range(ny):
        for x in range(nx):
            if mask[y, x]:
                continue
            for i in range(9):
                xs, ys = x - cx[i], (y - cy[i]) % ny
                if not 0 <= xs < nx:
                    continue
                out[i, y, x] = ft[opp[i], y, x] if mask[ys, xs] else ft[i, ys, xs]
    for y in range(ny):
        out[:, y, 0] = oracle_mod.feq(1.0, u_in[y], 0.0)
        out[:, y, nx - 1] = out[:, y, nx - 2]
    return out


def test_brute_force_tiny_channel(oracle_mod):
    # P14
    nx, ny, tau = 8, 6, 0.66
    m = np.zeros((ny, nx), np.uint8)
    m[2, 3] = m[3, 3] = m[3, 4] = 1
    u_in = inputs.random_inlet(ny, seed=4)
    f = inputs.random_populations(nx, ny, seed=7) * (1 - m)[None]
    s = oracle_mod.Sim(m, tau, u_in)
    s.set_populations(f)
    for _ in range(3):
        f = brute_step(oracle_mod, f, m, tau, u_in)
        s.step(1)
        np.testing.assert_allclose(s.populations(), f, rtol=0, atol=1e-15)


def test_inlet_and_outlet_columns(oracle_mod):
    m, w = naca_small(oracle_mod, 4.0)
    u_in = inputs.random_inlet(w.ny, seed=2)
    s = oracle_mod.Sim(m, w.tau, u_in)
    s.step(5)
    f = s.populations()
    for y in range(w.ny):
        np.testing.assert_array_equal(f[:, y, 0], oracle_mod.feq(1.0, u_in[y], 0.0))
    np.testing.assert_array_equal(f[:, :, -1], f[:, :, -2])


def test_checkpoint_resume_bitwise(oracle_mod):
    # P15
    m, w = naca_small(oracle_mod, 2.0)
    s1 = oracle_mod.Sim(m, w.tau, w.u_in)
    s1.step(40)
    s2 = oracle_mod.Sim(m, w.tau, w.u_in)
    s2.step(20)
    f = s2.populations()
    s3 = oracle_mod.Sim(m, w.tau, w.u_in)
    s3.set_populations(f)
    s3.step(20)
    np.testing.assert_array_equal(s1.populations(), s3.populations())


def test_threads_do_not_change_the_results():
    # the node loops may run on several host threads; every sum keeps its
    # single-threaded order, so the trajectory and every force are bitwise equal
    import oracle
    m = inputs.random_blobs_mask(97, 41, 8, seed=12, margin_x=3)
    f0 = inputs.random_populations(97, 41, seed=13, lo=0.05, hi=0.12) * (1 - m)[None]
    runs = []
    for th in (1, 4):
        oracle.set_threads(th)
        s = oracle.Sim(m, 0.6, inputs.random_inlet(41, seed=14))
        s.set_populations(f0)
        s.step(25)
        runs.append((s.populations(), [s.force_series(k) for k in range(5)]))
    oracle.set_threads(1)
    assert np.array_equal(runs[0][0], runs[1][0])
    for a, b in zip(runs[0][1], runs[1][1]):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
