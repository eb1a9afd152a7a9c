"""The C ABI on a machine without a GPU: the library builds, loads, exports every
function that include/gblbm.h declares, and rejects bad arguments on the host
before touching a device.  No compute call is made here."""
import ctypes as C

import numpy as np
import pytest

from paper_2210_10377_gb300 import binding as b


@pytest.fixture(scope="module")
def L():
    from paper_2210_10377_gb300 import build
    build.build()
    return b.lib()


def test_exports_every_declared_function(L):
    names = b.header_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(L, n)]
    assert missing == []


def create(L, mask, tau=0.6, u=(0.05,), **bc_fields):
    mask = np.ascontiguousarray(mask, np.uint8)
    ny, nx = mask.shape
    u = np.ascontiguousarray(u, np.float64)
    bc = b.lbm_bc()
    L.lbm_bc_default(C.byref(bc))
    for k, v in bc_fields.items():
        if k == "cv":
            for i in range(4):
                bc.cv[i] = v[i]
        elif k == "body_force":
            bc.body_force[0], bc.body_force[1] = v
        else:
            setattr(bc, k, v)
    h = C.c_void_p()
    rc = L.lbm_create(mask.ctypes.data_as(C.POINTER(C.c_uint8)), nx, ny, tau, b._dp(u), u.size,
                      C.byref(bc), C.byref(h))
    return rc, L.lbm_last_error(None).decode(), h


def test_defaults(L):
    bc = b.lbm_bc()
    L.lbm_bc_default(C.byref(bc))
    assert (bc.kind, bc.storage, bc.rho0, bc.cv[0], bc.record_series) == (0, 1, 1.0, -1, 1)


@pytest.mark.parametrize("kwargs,needle", [
    (dict(tau=0.5), "tau"),
    (dict(tau=float("nan")), "tau"),
    (dict(u=(0.05, 0.05)), "n_u_in"),
    (dict(u=(float("inf"),)), "u_in"),
    (dict(kind=7), "boundary kind"),
    (dict(storage=9), "storage"),
    (dict(rho0=0.0), "rho0"),
    (dict(body_force=(float("nan"), 0.0)), "body force"),
    (dict(cv=(0, 10, 2, 5)), "control volume"),       # touches the inlet column
    (dict(cv=(2, 19, 2, 5)), "control volume"),       # touches the outlet column
    (dict(cv=(2, 10, 0, 5)), "control volume"),       # straddles the periodic y edge
    (dict(cv=(5, 3, 2, 5)), "control volume"),        # empty
])
def test_rejects_bad_arguments(L, kwargs, needle):
    m = np.zeros((8, 20), np.uint8)
    rc, msg, h = create(L, m, **kwargs)
    assert rc == 1 and needle in msg and not h.value


@pytest.mark.parametrize("col", [0, 1, 18, 19])
def test_rejects_solid_in_boundary_columns(L, col):
    m = np.zeros((8, 20), np.uint8)
    m[3, col] = 1
    rc, msg, _ = create(L, m)
    assert rc == 1 and "columns" in msg
    # a fully periodic domain has no inlet or outlet
    rc, msg, _ = create(L, m, kind=1)
    assert rc != 1


def test_rejects_tiny_and_huge_grids(L):
    rc, msg, _ = create(L, np.zeros((2, 20), np.uint8))
    assert rc == 1 and "small" in msg
    rc, msg, _ = create(L, np.zeros((8, 3), np.uint8))
    assert rc == 1
    u = np.array([0.05])
    bc = b.lbm_bc()
    L.lbm_bc_default(C.byref(bc))
    h = C.c_void_p()
    dummy = np.zeros(1, np.uint8)
    rc = L.lbm_create(dummy.ctypes.data_as(C.POINTER(C.c_uint8)), 1 << 15, 1 << 14, 0.6, b._dp(u),
                      1, C.byref(bc), C.byref(h))
    assert rc == 1 and "int32" in L.lbm_last_error(None).decode()


def test_naca_mask_rejects_bad_arguments(L):
    out = np.zeros(16, np.uint8)
    p = out.ctypes.data_as(C.POINTER(C.c_uint8))
    assert L.lbm_naca_mask(4, 4, -1.0, 0.12, 0.0, 2.0, 2.0, 0, p) == 1
    assert L.lbm_naca_mask(4, 4, 2.0, 0.0, 0.0, 2.0, 2.0, 0, p) == 1
    assert L.lbm_naca_mask(0, 4, 2.0, 0.12, 0.0, 2.0, 2.0, 0, p) == 1


def test_null_handle_calls_fail_cleanly(L):
    fx, fy = C.c_double(), C.c_double()
    assert L.lbm_step(None, 1) == 1
    assert L.lbm_force(None, 0, C.byref(fx), C.byref(fy)) == 1
    assert L.lbm_steps_done(None) == -1
    assert L.lbm_set_adjoint_budget(None, 1.0) == 1
    L.lbm_destroy(None)


def test_no_device_is_an_error_not_a_fallback(L):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    rc, msg, h = create(L, np.zeros((8, 20), np.uint8))
    assert rc == 3 and not h.value


def test_binding_refuses_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(b, "_lib", None)
    monkeypatch.setattr(b._build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        b.lib()


def batch_create(L, domains, **bc_fields):
    keep = []
    arr = (b.lbm_domain * max(len(domains), 1))()
    for k, d in enumerate(domains):
        m = np.ascontiguousarray(d["mask"], np.uint8)
        u = np.ascontiguousarray(np.atleast_1d(d.get("u_in", 0.05)), np.float64)
        keep += [m, u]
        arr[k].mask = m.ctypes.data_as(C.POINTER(C.c_uint8))
        arr[k].ny, arr[k].nx = m.shape
        arr[k].tau = d.get("tau", 0.6)
        arr[k].u_in = b._dp(u)
        arr[k].n_u_in = u.size
        for i in range(4):
            arr[k].cv[i] = d.get("cv", (-1, 0, 0, 0))[i]
    bc = b.lbm_bc()
    L.lbm_bc_default(C.byref(bc))
    for k, v in bc_fields.items():
        if k == "body_force":
            bc.body_force[0], bc.body_force[1] = v
        else:
            setattr(bc, k, v)
    h = C.c_void_p()
    rc = L.lbm_batch_create(arr, len(domains), C.byref(bc), C.byref(h))
    return rc, L.lbm_batch_last_error(None).decode(), h


def test_batch_rejects_bad_arguments_on_the_host(L):
    ok = {"mask": np.zeros((8, 20), np.uint8)}
    wall = np.zeros((8, 20), np.uint8)
    wall[3, 1] = 1
    cases = [
        ([], {}, "n >= 1"),
        ([ok, {"mask": wall}], {}, "domain 1: solid node at (1, 3)"),
        ([ok, dict(ok, tau=0.5)], {}, "domain 1: tau"),
        ([dict(ok, u_in=[0.05, 0.05])], {}, "domain 0: n_u_in"),
        ([dict(ok, cv=(0, 19, 0, 7))], {}, "domain 0: control volume"),
        ([ok], dict(body_force=(1e-6, 0.0)), "body force"),
        ([ok], dict(kernel=1), "direct kernel"),
        ([ok], dict(storage=9), "storage"),
        ([ok], dict(rho0=-1.0), "rho0"),
    ]
    for doms, bc, needle in cases:
        rc, msg, h = batch_create(L, doms, **bc)
        assert rc == 1 and not h.value and needle in msg, (needle, msg)


def test_batch_null_handle_calls_fail_cleanly(L):
    fx, fy = C.c_double(), C.c_double()
    assert L.lbm_batch_step(None, 1) == 1
    assert L.lbm_batch_forces(None, 0, 0, C.byref(fx), C.byref(fy)) == 1
    assert L.lbm_batch_steps_done(None) == -1
    assert L.lbm_batch_nodes(None) == -1
    assert L.lbm_batch_num_shapes() == 3
    L.lbm_batch_destroy(None)


def test_batch_without_device_is_an_error(L):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    rc, msg, h = batch_create(L, [{"mask": np.zeros((8, 20), np.uint8)}])
    assert rc == 3 and not h.value
