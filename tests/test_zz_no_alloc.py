"""lbm_links_noalloc: the link list of a device-resident mask, built by the
library without allocating device memory.

Some callers cannot let a library allocate: a host application that owns a
fixed device-memory budget or its own pool, a plug-in whose host forbids
cudaMalloc, or a latency-bound loop that cannot absorb the synchronisation
cudaMalloc/cudaFree may trigger.  Such a caller hands in device buffers it
already owns; this entry point works in a fixed static scratch array instead.
Here the caller's buffers come from torch.  The result is checked against the
oracle's link list (the definition of a link: a fluid node next to a solid
one, Section II) and against the handle-based lbm_links() entry point, twice in
a row, so that the second call also shows that scratch contents left by the
first do not leak through.  A short output buffer gets the first links and the
full count, and nothing past its end is written.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
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
        assert np.array_equal(got, oracle.links(mask, periodic_x=periodic))


def test_noalloc_short_buffer_gets_prefix_and_full_count(env):
    torch, binding, L = env
    stream = torch.cuda.Stream()
    mask = inputs.random_blobs_mask(257, 45, 12, seed=19, margin_x=2)
    want = oracle.links(mask)
    cap = want.size // 2
    assert cap > 0
    d_mask = torch.from_numpy(mask).to("cuda")
    d_links = torch.full((want.size + 64,), -1, dtype=torch.int32, device="cuda")
    for _ in range(2):
        d_links.fill_(-1)
        count = C.c_long(-1)
        torch.cuda.synchronize()
        rc = L.lbm_links_noalloc(d_mask.data_ptr(), mask.shape[1], mask.shape[0], 0,
                                 d_links.data_ptr(), cap, C.byref(count), stream.cuda_stream)
        assert rc == 0, L.lbm_last_error(None)
        assert count.value == want.size
        got = d_links.cpu().numpy()
        assert np.array_equal(got[:cap], want[:cap])
        assert (got[cap:] == -1).all()


def test_noalloc_refuses_a_capturing_stream(env):
    torch, binding, L = env
    mask = inputs.random_blobs_mask(64, 16, 3, seed=5, margin_x=2)
    d_mask = torch.from_numpy(mask).to("cuda")
    d_links = torch.full((256,), -1, dtype=torch.int32, device="cuda")
    x = torch.zeros(4, device="cuda")
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    count = C.c_long(-3)
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=stream):
        x.add_(1.0)
        rc = L.lbm_links_noalloc(d_mask.data_ptr(), mask.shape[1], mask.shape[0], 0,
                                 d_links.data_ptr(), 256, C.byref(count), stream.cuda_stream)
    assert rc == 1 and b"captured" in L.lbm_last_error(None)
    assert count.value == -3
    # the refused call queued nothing; the next plain call still works
    got = noalloc_links(torch, L, mask, False, torch.cuda.Stream())
    assert np.array_equal(got, oracle.links(mask))


def test_noalloc_links_same_call_twice_and_full_size(env):
    torch, binding, L = env
    stream = torch.cuda.Stream()
    w = inputs.LARGE_F32
    mask = binding.naca_mask(w.nx, w.ny, w.chord, w.thickness, w.alpha_deg, w.xc, w.yc)
    want = handle_links(binding, mask, False)
    a = noalloc_links(torch, L, mask, False, stream)
    b = noalloc_links(torch, L, mask, False, stream)
    assert np.array_equal(a, want) and np.array_equal(b, want)
    assert np.array_equal(a, oracle.links(mask))


def test_noalloc_rejects_grids_beyond_its_scratch(env):
    torch, binding, L = env
    count = C.c_long(-7)
    dummy = torch.zeros(16, dtype=torch.uint8, device="cuda")
    rc = L.lbm_links_noalloc(dummy.data_ptr(), 1 << 14, (1 << 12) + 1, 0, None, 0, C.byref(count),
                             None)
    assert rc == 1 and b"scratch limit" in L.lbm_last_error(None)
    assert count.value == -7
