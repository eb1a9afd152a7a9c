"""Failure paths of the CUDA library that need a device, made without any GPU
fault: a bounded device wait that is told to give up at once, and the handle's
recovery afterwards.

The staged collide-stream kernel waits on an mbarrier for each tile's bulk
copy.  With the poll bound set to zero (a test hook of the library), every
CTA's first wait gives up immediately; the CTA raises the timeout status, waits
(within a bound of its own) for the copies it has already issued, and returns.
lbm_step then reports ETIMEOUT, and the same handle, once given back a state,
steps on with either kernel exactly like a fresh one.
"""
import numpy as np
import pytest

import oracle
from paper_2210_10377_gb300 import inputs

pytestmark = pytest.mark.gpu

ETIMEOUT = 5


@pytest.fixture(scope="module")
def gb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_10377_gb300 import binding
    binding.lib()
    return binding


@pytest.mark.parametrize("storage", ["f32", "f16dev"])
def test_staged_wait_timeout_is_reported_and_the_handle_recovers(gb, storage):
    w = inputs.SMALL_F64
    m = oracle.naca_mask(w.nx, w.ny, w.chord, w.thickness, 3.0, w.xc, w.yc)
    lat = gb.Lattice(m, w.tau, w.u_in, storage=storage, kernel="staged")
    lat.step(1)
    lat.step(6)
    f = lat.populations()
    lat.set_wait_limit(0)
    with pytest.raises(gb.LbmError) as e:
        lat.step(1)
    assert e.value.code == ETIMEOUT
    with pytest.raises(gb.LbmError) as e:
        lat.step(4)  # again, from a captured graph
    assert e.value.code == ETIMEOUT
    lat.set_wait_limit(-1)
    for kernel in ("direct", "staged"):
        lat.set_kernel(kernel)
        lat.set_populations(f)
        t0 = lat.steps_done
        lat.step(1)
        lat.step(20)
        ref = gb.Lattice(m, w.tau, w.u_in, storage=storage, kernel=kernel)
        ref.set_populations(f)
        ref.step(21)
        assert np.array_equal(lat.populations(), ref.populations()), kernel
        for s in ("A", "B", "A_RTT", "SI"):
            got = lat.force_series(s, t0, 21)
            want = ref.force_series(s, 0, 21)
            assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), (kernel, s)
        ref.close()
    lat.close()


def test_kernel_switch_needs_a_staged_handle(gb):
    w = inputs.SMALL_F64
    m = oracle.naca_mask(w.nx, w.ny, w.chord, w.thickness, 0.0, w.xc, w.yc)
    lat = gb.Lattice(m, w.tau, w.u_in, storage="f32")
    with pytest.raises(gb.LbmError) as e:
        lat.set_kernel("staged")
    assert e.value.code == 1
    lat.set_kernel("direct")
    lat.step(3)
    lat.close()
