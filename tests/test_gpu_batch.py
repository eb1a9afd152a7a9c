"""Batches of independent domains (lbm_batch_*, through the C ABI) against the
FP64 CPU oracle run on each domain alone, and against the single-domain GPU
handle.

A batch is a set of independent problems: each domain's populations and force
series must be those of the same problem solved alone.  The oracle therefore
pins a batch domain by domain.  The batched kernel runs the single-domain
kernel's per-node arithmetic, so populations agree bit for bit with
single-domain handles; the link sums of a domain run in one CTA instead of
several, so forces agree to round-off.
"""
import numpy as np
import pytest

import oracle
from bars import step_error
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


def naca_domain(w, **extra):
    m = oracle.naca_mask(w.nx, w.ny, w.chord, w.thickness, w.alpha_deg, w.xc, w.yc)
    d = {"mask": m, "tau": w.tau, "u_in": w.u_in}
    d.update(extra)
    return d


def small_domains(n=5, factor=4, seed=inputs.SEED):
    """The batching workload's instance recipe (NACA00xx, chord 48..128, 8 x 4
    chords) shrunk by `factor`: uneven domains of a few thousand nodes."""
    return [naca_domain(inputs.scaled(w, factor)) for w in inputs.batch_instances(n, seed)]


def oracle_run(d, chunks, f0=None):
    sim = oracle.Sim(d["mask"], d["tau"], d["u_in"], cv=d.get("cv"))
    if f0 is not None:
        sim.set_populations(f0)
    for n in chunks:
        sim.step(n)
    return sim


def scale_of(series):
    return max(max(np.abs(x).max(), np.abs(y).max()) for x, y in series.values()) or 1.0


def test_batch_f64_matches_oracle_per_domain(gb):
    doms = small_domains(4)
    # a ragged blob domain with a per-row inlet, an explicit box and random start
    ny, nx = 37, 150
    blob = inputs.random_blobs_mask(nx, ny, 9, seed=41, margin_x=3)
    doms.append({"mask": blob, "tau": 0.61, "u_in": inputs.random_inlet(ny, seed=42),
                 "cv": [20, 120, 3, 30]})
    f0 = inputs.random_populations(nx, ny, seed=43, lo=0.05, hi=0.15)
    chunks = [1, 16, 2, 131, 3, 47]  # graphs from both buffers, single steps
    b = gb.Batch(doms, storage="f64")
    b.set_populations(4, f0)
    for n in chunks:
        b.step(n)
    assert b.steps_done == sum(chunks)
    for k, d in enumerate(doms):
        sim = oracle_run(d, chunks, f0 if k == 4 else None)
        assert np.abs(b.populations(k) - sim.populations()).max() <= 1e-12, k
        for s in SCHEMES:
            ox, oy = sim.force_series(ORACLE_SCHEME[s])
            gx, gy = b.force_series(k, s)
            assert np.abs(gx - ox).max() <= 1e-11 and np.abs(gy - oy).max() <= 1e-11, (k, s)
    fx, fy = b.forces("B")
    for k, d in enumerate(doms):
        gx, gy = b.force_series(k, "B", b.steps_done - 1, 1)
        assert fx[k] == gx[0] and fy[k] == gy[0]
    flags, first = b.status()
    assert not flags.any() and (first == -1).all()
    b.close()


@pytest.mark.parametrize("storage,tol", [("f32dev", 1e-4), ("f32", 1e-2), ("f16dev", 1e-1)])
def test_batch_reduced_precision_matches_oracle(gb, storage, tol):
    # per domain, every scheme's per-step force against the oracle, relative
    # to the window's later forces (tests/bars.py), at the per-step bars of
    # the single-domain tests (test_gpu_parity.py)
    doms = small_domains(6, seed=7)
    steps = 400
    b = gb.Batch(doms, storage=storage)
    b.autotune(trials=2)
    b.step(steps)
    for k, d in enumerate(doms):
        sim = oracle_run(d, [steps])
        for s in SCHEMES:
            e = step_error(np.stack(b.force_series(k, s)), np.stack(sim.force_series(ORACLE_SCHEME[s])))
            assert e <= tol, (k, s, e)
    b.close()


@pytest.mark.parametrize("storage", ["f64", "f32", "f16dev"])
def test_batch_equals_single_domain_handles(gb, storage):
    doms = small_domains(5, seed=11)
    steps = 150
    b = gb.Batch(doms, storage=storage)
    b.step(steps)
    for k, d in enumerate(doms):
        lat = gb.Lattice(d["mask"], d["tau"], d["u_in"], storage=storage)
        lat.step(steps)
        assert np.array_equal(b.populations(k), lat.populations()), k
        q = 0.5 * 0.05 ** 2
        bn, bc = b.pressure_coefficient(k, 1.0 / 3.0, q)
        ln, lc = lat.pressure_coefficient(1.0 / 3.0, q)
        assert np.array_equal(bn, ln) and np.array_equal(bc, lc), k
        ser = {s: lat.force_series(s) for s in SCHEMES}
        sc = scale_of(ser)
        for s in SCHEMES:
            gx, gy = b.force_series(k, s)
            assert np.abs(gx - ser[s][0]).max() <= 1e-12 * sc, (k, s)
            assert np.abs(gy - ser[s][1]).max() <= 1e-12 * sc, (k, s)
        lat.close()
    b.close()


def test_batch_launch_configs_agree(gb):
    # every tile shape and grid computes the same populations and link forces
    # bit for bit; DRTT differs only by the grouping of the box sums
    doms = small_domains(5, seed=13)
    steps = 60
    ref = None
    b0 = gb.Batch(doms, storage="f32")
    configs = [(s, k) for s in range(b0.num_shapes) for k in (0, 1, 2)]
    b0.close()
    for shape, k in configs:
        b = gb.Batch(doms, storage="f32")
        try:
            b.set_launch(shape, k)
        except gb.LbmError as e:  # more CTAs per SM than this kernel fits
            assert k > 1 and e.code == 1 and "at most" in str(e)
            b.close()
            continue
        assert b.launch() == (shape, k)
        b.step(steps)
        got = ([b.populations(d) for d in range(len(doms))],
               {(d, s): b.force_series(d, s) for d in range(len(doms)) for s in SCHEMES})
        b.close()
        if ref is None:
            ref = got
            continue
        for d in range(len(doms)):
            assert np.array_equal(got[0][d], ref[0][d]), (shape, k, d)
            for s in ("A", "B", "A_RTT", "SI"):
                assert np.array_equal(got[1][(d, s)][0], ref[1][(d, s)][0]), (shape, k, d, s)
            sc = np.abs(ref[1][(d, "B")][0]).max()
            assert np.abs(got[1][(d, "DRTT")][0] - ref[1][(d, "DRTT")][0]).max() <= 1e-12 * sc


def test_batch_autotune_leaves_the_state_alone_and_splits_agree(gb):
    doms = small_domains(4, seed=17)
    a = gb.Batch(doms, storage="f32")
    a.step(2600)  # one call: the series grows twice (1024 -> 2048 -> 4096 rows)
    b = gb.Batch(doms, storage="f32")
    b.step(5)
    shape, k, ms = b.autotune(trials=2)
    assert 0 <= shape < b.num_shapes and k >= 0 and ms > 0
    assert b.launch() == (shape, k)
    chunks = [4] * 300 + [1, 2, 3, 17, 64] * 4
    chunks.append(2600 - 5 - sum(chunks))
    for n in chunks:
        b.step(n)
    assert a.steps_done == b.steps_done == 2600
    for d in range(len(doms)):
        assert np.array_equal(a.populations(d), b.populations(d)), d
        for s in ("A", "B", "A_RTT", "SI"):
            assert np.array_equal(a.force_series(d, s)[0], b.force_series(d, s)[0]), (d, s)
            assert np.array_equal(a.force_series(d, s)[1], b.force_series(d, s)[1]), (d, s)
    a.close()
    b.close()


def test_batch_instability_is_flagged_per_domain(gb):
    doms = small_domains(3, seed=19)
    ny, nx = 16, 64
    bad = {"mask": np.zeros((ny, nx), np.uint8), "tau": 0.5000001, "u_in": 0.45}
    b = gb.Batch(doms[:1] + [bad] + doms[1:], storage="f32")
    b.set_populations(1, inputs.random_populations(nx, ny, seed=5, lo=0.0, hi=0.6))
    with pytest.raises(gb.LbmError) as e:
        b.step(3000)
    assert e.value.code == 4
    flags, first = b.status()
    assert flags.tolist() == [0, 1, 0, 0] and first[1] >= 0 and (first[[0, 2, 3]] == -1).all()
    # the other domains are untouched by their neighbour's blow-up
    c = gb.Batch(doms, storage="f32")
    c.step(3000)
    for k_b, k_c in ((0, 0), (2, 1), (3, 2)):
        assert np.array_equal(b.populations(k_b), c.populations(k_c))
    b.close()
    c.close()


def test_batch_checkpoint_resume_bitwise(gb):
    doms = small_domains(3, seed=23)
    a = gb.Batch(doms, storage="f32")
    a.step(80)
    b = gb.Batch(doms, storage="f32")
    b.step(40)
    states = [b.populations(d) for d in range(3)]
    c = gb.Batch(doms, storage="f32")
    for d in range(3):
        c.set_populations(d, states[d])
    c.step(40)
    for d in range(3):
        assert np.array_equal(a.populations(d), c.populations(d))
        for s in ("A", "B", "A_RTT", "SI"):
            assert np.array_equal(a.force_series(d, s, 41, 39)[0], c.force_series(d, s, 1, 39)[0])
    with pytest.raises(gb.LbmError) as e:
        c.set_populations(0, states[0])
    assert e.value.code == 6
    a.close()
    b.close()
    c.close()


def test_batch_full_size_instances_sampled(gb):
    """The 256-instance batching workload at full size: every domain stays
    finite and unflagged; three domains are checked against the oracle over
    the first steps."""
    ws = inputs.batch_instances(256)
    doms = [naca_domain(w) for w in ws]
    b = gb.Batch(doms, storage=ws[0].storage)
    assert b.nodes == sum(w.nx * w.ny for w in ws)
    b.autotune(trials=2)
    steps = 120
    b.step(steps)
    flags, _ = b.status()
    assert not flags.any()
    fx, fy = b.forces("B")
    assert np.isfinite(fx).all() and np.isfinite(fy).all()
    order = np.argsort([w.nx * w.ny for w in ws])
    for k in order[:3]:
        sim = oracle_run(doms[k], [steps])
        for s in SCHEMES:
            e = step_error(np.stack(b.force_series(int(k), s)), np.stack(sim.force_series(ORACLE_SCHEME[s])))
            assert e <= 1e-4, (k, s, e)
    b.close()
