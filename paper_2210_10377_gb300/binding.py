"""Python binding of libgblbm.so (ctypes): argument marshalling only.

Every step of the solver runs in the library's CUDA kernels.  PyTorch supplies
the CUDA stream and, through the allocator hook of ``lbm_bc``, device memory
from its caching allocator.  Importing this module raises if the library has
not been built; there is no fallback implementation.
"""
import ctypes as C
import os
import re

import numpy as np

from . import build as _build

CHANNEL, PERIODIC = 0, 1
F64, F32, F32_DEV, F16_DEV = 0, 1, 2, 3
STORAGE = {"f64": F64, "f32": F32, "f32dev": F32_DEV, "f16dev": F16_DEV}
MEA_A, MEA_B, DRTT, MEA_A_RTT, MOMENTUM_DEFECT, SI = 0, 1, 2, 3, 4, 5
SCHEMES = {"A": MEA_A, "B": MEA_B, "DRTT": DRTT, "A_RTT": MEA_A_RTT, "DEFECT": MOMENTUM_DEFECT,
           "SI": SI}
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EUNSTABLE", 5: "ETIMEOUT",
          6: "ESTATE"}
HEADER = os.path.join(_build.ROOT, "include", "gblbm.h")

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class LbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code


class lbm_bc(C.Structure):
    _fields_ = [("kind", C.c_int), ("storage", C.c_int), ("rho0", C.c_double),
                ("body_force", C.c_double * 2), ("cv", C.c_int * 4),
                ("record_series", C.c_int), ("cuda_stream", C.c_void_p),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p),
                ("kernel", C.c_int)]


class lbm_domain(C.Structure):
    _fields_ = [("mask", C.POINTER(C.c_uint8)), ("nx", C.c_int), ("ny", C.c_int),
                ("tau", C.c_double), ("u_in", C.POINTER(C.c_double)), ("n_u_in", C.c_int),
                ("cv", C.c_int * 4)]


_lib = None


def lib():
    """Load libgblbm.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libgblbm.so is not built (%s); run __graft_entry__.build() or "
                           "python -m paper_2210_10377_gb300.build" % _build.LIB)
    L = C.CDLL(_build.LIB)
    vp, dp, ip, lp = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_long)
    L.lbm_bc_default.argtypes = [C.POINTER(lbm_bc)]
    L.lbm_bc_default.restype = None
    L.lbm_create.argtypes = [C.POINTER(C.c_uint8), C.c_int, C.c_int, C.c_double, dp, C.c_int,
                             C.POINTER(lbm_bc), C.POINTER(vp)]
    L.lbm_step.argtypes = [vp, C.c_int]
    L.lbm_force.argtypes = [vp, C.c_int, dp, dp]
    L.lbm_force_series.argtypes = [vp, C.c_int, C.c_long, C.c_long, dp, dp]
    L.lbm_populations.argtypes = [vp, dp]
    L.lbm_set_populations.argtypes = [vp, dp]
    L.lbm_links.argtypes = [vp, C.POINTER(C.c_int32), C.c_long, lp]
    L.lbm_control_volume.argtypes = [vp, ip]
    L.lbm_naca_mask.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                C.c_double, C.c_double, C.c_int, C.POINTER(C.c_uint8)]
    L.lbm_adjoint.argtypes = [vp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, dp, dp, dp, dp]
    L.lbm_steps_done.argtypes = [vp]
    L.lbm_steps_done.restype = C.c_long
    L.lbm_num_links.argtypes = [vp]
    L.lbm_num_links.restype = C.c_long
    L.lbm_set_kernel_timing.argtypes = [vp, C.c_int]
    L.lbm_kernel_times.argtypes = [vp, dp, lp, C.c_int]
    L.lbm_launch_count.argtypes = [vp]
    L.lbm_launch_count.restype = C.c_long
    L.lbm_last_error.argtypes = [vp]
    L.lbm_last_error.restype = C.c_char_p
    L.lbm_destroy.argtypes = [vp]
    L.lbm_destroy.restype = None
    L.lbm_prepare.argtypes = [vp, C.c_long]
    L.lbm_step_async.argtypes = [vp, C.c_int]
    L.lbm_sync.argtypes = [vp]
    L.lbm_set_kernel.argtypes = [vp, C.c_int]
    L.lbm_set_wait_limit.argtypes = [vp, C.c_long]
    L.lbm_coefficients.argtypes = [vp, C.c_int, C.c_long, C.c_long, C.c_double, C.c_double, dp, dp, dp]
    L.lbm_set_adjoint_budget.argtypes = [vp, C.c_double]
    for name in ("lbm_create", "lbm_step", "lbm_force", "lbm_force_series", "lbm_populations",
                 "lbm_set_populations", "lbm_links", "lbm_control_volume", "lbm_naca_mask",
                 "lbm_set_kernel_timing", "lbm_kernel_times", "lbm_adjoint", "lbm_prepare",
                 "lbm_coefficients", "lbm_set_kernel", "lbm_set_wait_limit", "lbm_step_async", "lbm_sync",
                 "lbm_set_adjoint_budget"):
        getattr(L, name).restype = C.c_int
    # batches
    L.lbm_batch_create.argtypes = [C.POINTER(lbm_domain), C.c_int, C.POINTER(lbm_bc), C.POINTER(vp)]
    L.lbm_batch_step.argtypes = [vp, C.c_int]
    L.lbm_batch_forces.argtypes = [vp, C.c_int, C.c_long, dp, dp]
    L.lbm_batch_force_series.argtypes = [vp, C.c_int, C.c_int, C.c_long, C.c_long, dp, dp]
    L.lbm_batch_populations.argtypes = [vp, C.c_int, dp]
    L.lbm_batch_set_populations.argtypes = [vp, C.c_int, dp]
    L.lbm_batch_status.argtypes = [vp, ip, lp]
    L.lbm_batch_set_launch.argtypes = [vp, C.c_int, C.c_int]
    L.lbm_batch_get_launch.argtypes = [vp, ip, ip]
    L.lbm_batch_num_shapes.argtypes = []
    L.lbm_batch_num_shapes.restype = C.c_int
    L.lbm_batch_shape.argtypes = [vp, C.c_int, ip, ip]
    L.lbm_batch_autotune.argtypes = [vp, C.c_int, ip, ip, dp]
    L.lbm_batch_steps_done.argtypes = [vp]
    L.lbm_batch_steps_done.restype = C.c_long
    L.lbm_batch_num_domains.argtypes = [vp]
    L.lbm_batch_num_domains.restype = C.c_int
    L.lbm_batch_nodes.argtypes = [vp]
    L.lbm_batch_nodes.restype = C.c_longlong
    L.lbm_batch_launch_count.argtypes = [vp]
    L.lbm_batch_launch_count.restype = C.c_longlong
    L.lbm_batch_last_error.argtypes = [vp]
    L.lbm_batch_last_error.restype = C.c_char_p
    L.lbm_cylinder_mask.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.POINTER(C.c_uint8)]
    L.lbm_cylinder_mask.restype = C.c_int
    L.lbm_pressure_coefficient.argtypes = [vp, C.c_double, C.c_double, C.POINTER(C.c_int32), dp, C.c_long, lp]
    L.lbm_pressure_coefficient.restype = C.c_int
    L.lbm_batch_pressure_coefficient.argtypes = [vp, C.c_int, C.c_double, C.c_double, C.POINTER(C.c_int32), dp,
                                                 C.c_long, lp]
    L.lbm_batch_pressure_coefficient.restype = C.c_int
    L.lbm_batch_destroy.argtypes = [vp]
    L.lbm_batch_destroy.restype = None
    L.lbm_batch_prepare.argtypes = [vp, C.c_long]
    L.lbm_batch_coefficients.argtypes = [vp, C.c_int, C.c_int, C.c_long, C.c_long, C.c_double, C.c_double,
                                         dp, dp, dp]
    for name in ("lbm_batch_create", "lbm_batch_step", "lbm_batch_forces", "lbm_batch_force_series",
                 "lbm_batch_populations", "lbm_batch_set_populations", "lbm_batch_status",
                 "lbm_batch_set_launch", "lbm_batch_get_launch", "lbm_batch_shape",
                 "lbm_batch_autotune", "lbm_batch_prepare", "lbm_batch_coefficients"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def header_functions(path=HEADER):
    """Names of the functions declared in include/gblbm.h."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text)) - {"lbm_alloc_fn", "lbm_free_fn"})


def _check(rc, h=None):
    if rc != 0:
        msg = lib().lbm_last_error(h)
        raise LbmError(rc, msg.decode() if msg else "")


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def naca_mask(nx, ny, chord, thickness, alpha_deg, xc, yc, closed_te=False):
    """NACA 4-digit section voxelised on the device; uint8 [ny][nx], 1 = solid."""
    out = np.zeros((ny, nx), np.uint8)
    _check(lib().lbm_naca_mask(int(nx), int(ny), float(chord), float(thickness),
                               float(alpha_deg), float(xc), float(yc), int(closed_te),
                               out.ctypes.data_as(C.POINTER(C.c_uint8))))
    return out


def cylinder_mask(nx, ny, xc, yc, diameter):
    """Circular cylinder voxelised on the device; uint8 [ny][nx], 1 = solid."""
    out = np.zeros((ny, nx), np.uint8)
    _check(lib().lbm_cylinder_mask(int(nx), int(ny), float(xc), float(yc), float(diameter),
                                   out.ctypes.data_as(C.POINTER(C.c_uint8))))
    return out


def body_mask(w):
    """The mask of a workload: its NACA section, or its cylinder."""
    if w.extra.get("body") == "cylinder":
        return cylinder_mask(w.nx, w.ny, w.xc, w.yc, w.chord)
    return naca_mask(w.nx, w.ny, w.chord, w.thickness, w.alpha_deg, w.xc, w.yc)


_STREAMS = {}


def default_stream(device=0):
    """The stream handles use when none is given: one per device, so that the
    memory one handle returns to torch's caching allocator (which reuses a
    block on the stream it was freed on) serves the next handle.  The library
    frees memory only after its stream is idle."""
    import torch
    s = _STREAMS.get(device)
    if s is None:
        s = _STREAMS[device] = torch.cuda.Stream(device)
    return s


class _TorchAllocator:
    """Device memory for the library from torch's caching allocator."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device
        self.live = {}
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, nbytes, stream, user):
        try:
            p = self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream or 0)
        except Exception:
            return None
        self.live[p] = nbytes
        return p

    def _free(self, ptr, user):
        if ptr in self.live:
            del self.live[ptr]
            self.torch.cuda.caching_allocator_delete(ptr)


class Lattice:
    """One solver handle (lbm_create ... lbm_destroy)."""

    def __init__(self, mask, tau, u_in, *, kind=CHANNEL, storage="f32", rho0=1.0,
                 body_force=(0.0, 0.0), cv=None, record_series=True, stream=None,
                 torch_alloc=True, device=0, kernel="direct"):
        import torch
        L = lib()
        self.mask = np.ascontiguousarray(mask, np.uint8)
        self.ny, self.nx = self.mask.shape
        self.device = device
        self.stream = stream if stream is not None else default_stream(device)
        u = np.ascontiguousarray(np.atleast_1d(np.asarray(u_in, np.float64)))
        bc = lbm_bc()
        L.lbm_bc_default(C.byref(bc))
        bc.kind = int(kind)
        bc.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        bc.rho0 = float(rho0)
        bc.body_force[0], bc.body_force[1] = float(body_force[0]), float(body_force[1])
        if cv is not None:
            for k in range(4):
                bc.cv[k] = int(cv[k])
        bc.record_series = int(bool(record_series))
        bc.kernel = {"direct": 0, "staged": 1}[kernel]
        bc.cuda_stream = self.stream.cuda_stream
        self._alloc = _TorchAllocator(device) if torch_alloc else None
        if self._alloc is not None:
            bc.alloc = self._alloc.alloc
            bc.free = self._alloc.free
        self.storage = bc.storage
        self.rho0 = float(rho0)
        self.u_ref = float(np.mean(u))
        h = C.c_void_p()
        with torch.cuda.device(device):
            _check(L.lbm_create(self.mask.ctypes.data_as(C.POINTER(C.c_uint8)), self.nx, self.ny,
                                float(tau), _dp(u), int(u.size), C.byref(bc), C.byref(h)))
        self._h = h

    # -- life cycle
    def close(self):
        if getattr(self, "_h", None):
            lib().lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- stepping and forces
    def step(self, n=1):
        _check(lib().lbm_step(self._h, int(n)), self._h)

    def step_async(self, n=1):
        """Queue n steps without waiting (lbm_step_async); sync() or any call
        that reads results waits for them and reports their status."""
        _check(lib().lbm_step_async(self._h, int(n)), self._h)

    def sync(self):
        _check(lib().lbm_sync(self._h), self._h)

    def force(self, scheme):
        fx, fy = C.c_double(), C.c_double()
        _check(lib().lbm_force(self._h, SCHEMES.get(scheme, scheme), C.byref(fx), C.byref(fy)),
               self._h)
        return fx.value, fy.value

    def force_series(self, scheme, first=0, count=None):
        if count is None:
            count = self.steps_done - first
        fx = np.zeros(max(count, 1))
        fy = np.zeros(max(count, 1))
        _check(lib().lbm_force_series(self._h, SCHEMES.get(scheme, scheme), int(first),
                                      int(count), _dp(fx), _dp(fy)), self._h)
        return fx[:count], fy[:count]

    def prepare(self, n):
        """Grow the series for n more steps and build every captured step graph
        (lbm_prepare), so that stepping afterwards only launches."""
        _check(lib().lbm_prepare(self._h, int(n)), self._h)

    def set_kernel(self, kernel):
        """'direct' or 'staged' for later steps (lbm_set_kernel)."""
        _check(lib().lbm_set_kernel(self._h, {"direct": 0, "staged": 1}.get(kernel, kernel)), self._h)

    def set_wait_limit(self, polls):
        """Poll bound of the staged kernel's pipeline waits (lbm_set_wait_limit;
        negative: the default).  Only for testing the timeout path."""
        _check(lib().lbm_set_wait_limit(self._h, int(polls)), self._h)

    def coefficients(self, scheme, length, u_ref, first=0, count=None, per_step=True):
        """Drag and lift coefficients of one scheme over steps [first,
        first+count) (lbm_coefficients): (cd[count], cl[count], stats) with
        stats = (mean C_d, mean C_l, std C_d, std C_l); cd and cl are None
        when per_step is false."""
        if count is None:
            count = self.steps_done - first
        cd = np.zeros(max(count, 1)) if per_step else None
        cl = np.zeros(max(count, 1)) if per_step else None
        st = np.zeros(4)
        _check(lib().lbm_coefficients(self._h, SCHEMES.get(scheme, scheme), int(first), int(count),
                                      float(length), float(u_ref), _dp(cd) if per_step else None,
                                      _dp(cl) if per_step else None, _dp(st)), self._h)
        return (cd[:count] if per_step else None), (cl[:count] if per_step else None), tuple(st)

    # -- state
    def populations(self, out=None):
        if out is None:
            out = np.empty((9, self.ny, self.nx), np.float64)
        _check(lib().lbm_populations(self._h, _dp(out)), self._h)
        return out

    def set_populations(self, f):
        f = np.ascontiguousarray(f, np.float64).reshape(9, self.ny, self.nx)
        _check(lib().lbm_set_populations(self._h, _dp(f)), self._h)

    def links(self):
        n = self.num_links
        out = np.zeros(max(n, 1), np.int32)
        cnt = C.c_long()
        _check(lib().lbm_links(self._h, out.ctypes.data_as(C.POINTER(C.c_int32)), n,
                               C.byref(cnt)), self._h)
        return out[:cnt.value]

    def control_volume(self):
        cv = (C.c_int * 4)()
        _check(lib().lbm_control_volume(self._h, cv), self._h)
        return list(cv)

    def set_adjoint_budget(self, nbytes):
        """Device memory lbm_adjoint may fill with kept states (lbm_set_adjoint_budget;
        0: 60 % of the free memory).  adjoint() sets it from torch's view of the
        memory unless keep_budget=True is passed."""
        _check(lib().lbm_set_adjoint_budget(self._h, float(nbytes)), self._h)

    def adjoint(self, steps, window, wx=1.0, wy=0.0, checkpoint_every=0, want_df0=True, df0_device=False,
                keep_budget=False):
        """Run `steps` steps and return (J, dJ/dtau, dJ/du_in[ny], dJ/df0[9][ny][nx] or
        None) for J = the window-averaged wx Fx + wy Fy of algorithm B.
        df0_device: dJ/df0 as a float64 CUDA tensor on the handle's device,
        written there by the library (no copy to the host); else a numpy array."""
        J, dtau = C.c_double(), C.c_double()
        du = np.zeros(self.ny)
        df0, ptr = None, None
        if checkpoint_every <= 0 and self._alloc is not None and not keep_budget:
            # what torch can provide: the free memory and its own unused cache
            import torch
            free, _ = torch.cuda.mem_get_info(self.device)
            cached = torch.cuda.memory_reserved(self.device) - torch.cuda.memory_allocated(self.device)
            _check(lib().lbm_set_adjoint_budget(self._h, 0.6 * float(free + cached)), self._h)
        if want_df0 and df0_device:
            import torch
            df0 = torch.empty((9, self.ny, self.nx), dtype=torch.float64, device=self.device)
            # the handle's stream writes the block torch allocated on its current stream
            self.stream.wait_stream(torch.cuda.current_stream(self.device))
            ptr = C.cast(C.c_void_p(df0.data_ptr()), C.POINTER(C.c_double))
        elif want_df0:
            df0 = np.empty((9, self.ny, self.nx))
            ptr = _dp(df0)
        _check(lib().lbm_adjoint(self._h, int(steps), int(window), float(wx), float(wy),
                                 int(checkpoint_every), C.byref(J), C.byref(dtau), _dp(du), ptr), self._h)
        return J.value, dtau.value, du, df0

    def pressure_coefficient(self, p_inf=None, q=None):
        """(nodes, cp) at the boundary fluid nodes.  Defaults: p_inf = rho0/3 and
        q = rho0 U^2/2, U the mean of the inlet velocity given at creation."""
        p_inf = self.rho0 / 3.0 if p_inf is None else p_inf
        q = 0.5 * self.rho0 * self.u_ref ** 2 if q is None else q
        cnt = C.c_long()
        _check(lib().lbm_pressure_coefficient(self._h, float(p_inf), float(q), None, None, 0, C.byref(cnt)),
               self._h)
        nodes = np.zeros(max(cnt.value, 1), np.int32)
        cp = np.zeros(max(cnt.value, 1))
        _check(lib().lbm_pressure_coefficient(self._h, float(p_inf), float(q),
                                              nodes.ctypes.data_as(C.POINTER(C.c_int32)), _dp(cp), cnt.value,
                                              C.byref(cnt)), self._h)
        return nodes[:cnt.value], cp[:cnt.value]

    @property
    def steps_done(self):
        return lib().lbm_steps_done(self._h)

    @property
    def num_links(self):
        return lib().lbm_num_links(self._h)

    @property
    def launch_count(self):
        return lib().lbm_launch_count(self._h)

    # -- measurement support
    def set_kernel_timing(self, on):
        _check(lib().lbm_set_kernel_timing(self._h, int(bool(on))), self._h)

    def kernel_times(self, reset=False):
        ms = (C.c_double * 2)()
        n = (C.c_long * 2)()
        _check(lib().lbm_kernel_times(self._h, ms, n, int(bool(reset))), self._h)
        return {"collide_stream": (ms[0], n[0]), "link_force": (ms[1], n[1])}


def _bcheck(rc, b=None):
    if rc != 0:
        msg = lib().lbm_batch_last_error(b)
        raise LbmError(rc, msg.decode() if msg else "")


class Batch:
    """Many independent domains stepped together (lbm_batch_create ... destroy).

    domains: a list of dicts with keys mask (uint8 [ny][nx]), tau, u_in (scalar
    or ny values) and optionally cv (4 ints)."""

    def __init__(self, domains, *, kind=CHANNEL, storage="f32", rho0=1.0, record_series=True,
                 stream=None, torch_alloc=True, device=0):
        import torch
        L = lib()
        self.device = device
        self.stream = stream if stream is not None else default_stream(device)
        self._keep = []
        arr = (lbm_domain * len(domains))()
        self.shapes = []
        for k, d in enumerate(domains):
            m = np.ascontiguousarray(d["mask"], np.uint8)
            u = np.ascontiguousarray(np.atleast_1d(np.asarray(d["u_in"], np.float64)))
            self._keep += [m, u]
            arr[k].mask = m.ctypes.data_as(C.POINTER(C.c_uint8))
            arr[k].ny, arr[k].nx = m.shape
            arr[k].tau = float(d["tau"])
            arr[k].u_in = _dp(u)
            arr[k].n_u_in = int(u.size)
            cv = d.get("cv")
            for j in range(4):
                arr[k].cv[j] = int(cv[j]) if cv is not None else -1
            self.shapes.append(m.shape)
        bc = lbm_bc()
        L.lbm_bc_default(C.byref(bc))
        bc.kind = int(kind)
        bc.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        bc.rho0 = float(rho0)
        bc.record_series = int(bool(record_series))
        bc.cuda_stream = self.stream.cuda_stream
        self._alloc = _TorchAllocator(device) if torch_alloc else None
        if self._alloc is not None:
            bc.alloc = self._alloc.alloc
            bc.free = self._alloc.free
        self.storage = bc.storage
        h = C.c_void_p()
        with torch.cuda.device(device):
            _bcheck(L.lbm_batch_create(arr, len(domains), C.byref(bc), C.byref(h)))
        self._h = h
        self._keep = []

    def close(self):
        if getattr(self, "_h", None):
            lib().lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        _bcheck(lib().lbm_batch_step(self._h, int(n)), self._h)

    def forces(self, scheme, step=None):
        """(fx[n], fy[n]) of every domain at one step (default: the last)."""
        n = self.num_domains
        step = self.steps_done - 1 if step is None else int(step)
        fx, fy = np.zeros(n), np.zeros(n)
        sc = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
        _bcheck(lib().lbm_batch_forces(self._h, sc, step, _dp(fx), _dp(fy)), self._h)
        return fx, fy

    def force_series(self, domain, scheme, first=0, count=None):
        if count is None:
            count = self.steps_done - first
        fx, fy = np.zeros(count), np.zeros(count)
        sc = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
        _bcheck(lib().lbm_batch_force_series(self._h, int(domain), sc, int(first), int(count),
                                             _dp(fx), _dp(fy)), self._h)
        return fx, fy

    def prepare(self, n):
        """Grow the series for n more steps and build the captured step graphs
        of the current launch configuration (lbm_batch_prepare)."""
        _bcheck(lib().lbm_batch_prepare(self._h, int(n)), self._h)

    def coefficients(self, domain, scheme, length, u_ref, first=0, count=None, per_step=False):
        """Drag and lift coefficients of one domain (lbm_batch_coefficients):
        (cd, cl, stats) as Lattice.coefficients."""
        if count is None:
            count = self.steps_done - first
        cd = np.zeros(max(count, 1)) if per_step else None
        cl = np.zeros(max(count, 1)) if per_step else None
        st = np.zeros(4)
        sc = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
        _bcheck(lib().lbm_batch_coefficients(self._h, int(domain), sc, int(first), int(count), float(length),
                                             float(u_ref), _dp(cd) if per_step else None,
                                             _dp(cl) if per_step else None, _dp(st)), self._h)
        return (cd[:count] if per_step else None), (cl[:count] if per_step else None), tuple(st)

    def populations(self, domain):
        ny, nx = self.shapes[domain]
        out = np.zeros((9, ny, nx))
        _bcheck(lib().lbm_batch_populations(self._h, int(domain), _dp(out)), self._h)
        return out

    def set_populations(self, domain, f):
        f = np.ascontiguousarray(f, np.float64)
        _bcheck(lib().lbm_batch_set_populations(self._h, int(domain), _dp(f)), self._h)

    def pressure_coefficient(self, domain, p_inf, q):
        """(nodes, cp) at the boundary fluid nodes of one domain."""
        cnt = C.c_long()
        _bcheck(lib().lbm_batch_pressure_coefficient(self._h, int(domain), float(p_inf), float(q), None, None, 0,
                                                     C.byref(cnt)), self._h)
        nodes = np.zeros(max(cnt.value, 1), np.int32)
        cp = np.zeros(max(cnt.value, 1))
        _bcheck(lib().lbm_batch_pressure_coefficient(self._h, int(domain), float(p_inf), float(q),
                                                     nodes.ctypes.data_as(C.POINTER(C.c_int32)), _dp(cp),
                                                     cnt.value, C.byref(cnt)), self._h)
        return nodes[:cnt.value], cp[:cnt.value]

    def status(self):
        n = self.num_domains
        flags = (C.c_int * n)()
        first = (C.c_long * n)()
        _bcheck(lib().lbm_batch_status(self._h, flags, first), self._h)
        return np.array(flags[:], np.int32), np.array(first[:], np.int64)

    def set_launch(self, shape, ctas_per_sm):
        _bcheck(lib().lbm_batch_set_launch(self._h, int(shape), int(ctas_per_sm)), self._h)

    def launch(self):
        s, k = C.c_int(), C.c_int()
        _bcheck(lib().lbm_batch_get_launch(self._h, C.byref(s), C.byref(k)), self._h)
        return s.value, k.value

    def shape(self, k):
        w, h = C.c_int(), C.c_int()
        _bcheck(lib().lbm_batch_shape(self._h, int(k), C.byref(w), C.byref(h)), self._h)
        return w.value, h.value

    def autotune(self, trials=5):
        """Time every (tile shape, grid) and keep the fastest: (shape, ctas_per_sm, ms)."""
        s, k, ms = C.c_int(), C.c_int(), C.c_double()
        _bcheck(lib().lbm_batch_autotune(self._h, int(trials), C.byref(s), C.byref(k), C.byref(ms)),
                self._h)
        return s.value, k.value, ms.value

    @property
    def num_shapes(self):
        return lib().lbm_batch_num_shapes()

    @property
    def steps_done(self):
        return lib().lbm_batch_steps_done(self._h)

    @property
    def num_domains(self):
        return lib().lbm_batch_num_domains(self._h)

    @property
    def nodes(self):
        return lib().lbm_batch_nodes(self._h)

    @property
    def launch_count(self):
        return lib().lbm_batch_launch_count(self._h)
