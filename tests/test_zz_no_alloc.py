"""lbm_links_noalloc: the link list of a device-resident mask, built by the
library without allocating device memory.

Some callers cannot let a library allocate: a host application that owns a
fixed device-memory budget or its own pool, a plug-in whose host forbids
cudaMalloc, or a latency-bound loop that cannot absorb the synchronisation
cudaMalloc/cudaFree may trigger.  Such a caller hands in device buffers it
already owns; this entry point works in a fixed static scratch array instead.
Here the caller's buffers come from torch, and the result is checked against
the handle-based lbm_links() entry point, twice in a row, so that the second
call also shows that scratch contents left by the first do not leak through.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2210_10377_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_10377_gb300 import binding
    L = binding.lib()
    L.lbm_links_noalloc.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_long,
                                    C.POINTER(C.c_long), C.c_void_p]
    L.lbm_links_noalloc.restype = C.c_int
    return torch, binding, L


def noalloc_links(torch, L, mask, periodic, stream):
    ny, nx = mask.shape
    d_mask = torch.from_numpy(np.ascontiguousarray(mask, np.uint8)).to("cuda")
    cap = 9 * nx * ny // 8 + 16
    d_links = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    count = C.c_long(-1)
    torch.cuda.synchronize()
    rc = L.lbm_links_noalloc(d_mask.data_ptr(), nx, ny, int(periodic), d_links.data_ptr(), cap,
                             C.byref(count), stream.cuda_stream)
    assert rc == 0, L.lbm_last_error(None)
    assert count.value <= cap
    return d_links[:count.value].cpu().numpy()


def handle_links(binding, mask, periodic):
    lat = binding.Lattice(mask, 0.6, 0.05, kind=binding.PERIODIC if periodic else binding.CHANNEL,
                          storage="f32")
    out = lat.links()
    lat.close()
    return out


def test_noalloc_links_match_lbm_links_twice(env):
    torch, binding, L = env
    stream = torch.cuda.Stream()
    w = inputs.SMALL_F64
    cases = [
        (binding.naca_mask(w.nx, w.ny, w.chord, w.thickness, 5.0, w.xc, w.yc), False),
        (inputs.random_blobs_mask(301, 77, 25, seed=9, margin_x=0), True),
    ]
    for mask, periodic in cases:  # two calls in a row, different sizes
        got = noalloc_links(torch, L, mask, periodic, stream)
        want = handle_links(binding, mask, periodic)
        assert got.size > 0
        assert np.array_equal(got, want)


def test_noalloc_links_same_call_twice_and_full_size(env):
    torch, binding, L = env
    stream = torch.cuda.Stream()
    w = inputs.LARGE_F32
    mask = binding.naca_mask(w.nx, w.ny, w.chord, w.thickness, w.alpha_deg, w.xc, w.yc)
    want = handle_links(binding, mask, False)
    a = noalloc_links(torch, L, mask, False, stream)
    b = noalloc_links(torch, L, mask, False, stream)
    assert np.array_equal(a, want) and np.array_equal(b, want)


def test_noalloc_rejects_grids_beyond_its_scratch(env):
    torch, binding, L = env
    count = C.c_long(-7)
    dummy = torch.zeros(16, dtype=torch.uint8, device="cuda")
    rc = L.lbm_links_noalloc(dummy.data_ptr(), 1 << 14, (1 << 12) + 1, 0, None, 0, C.byref(count),
                             None)
    assert rc == 1 and b"scratch limit" in L.lbm_last_error(None)
    assert count.value == -7
