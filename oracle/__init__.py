"""FP64 CPU oracle for the D2Q9 bounce-back solver and its force schemes.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library; see ``lbm_oracle.c`` for what each function follows in
arXiv:2210.10377 (Section II for the update, Eq. MEA / rtt4 / rtt5 for the
momentum-exchange orders, Eq. rtt7 and the Appendix for DRTT).

This module only marshals arguments between numpy and the C library.
"""
import ctypes as C

import numpy as np

from .build import build_oracle

SCHEME_A, SCHEME_B, SCHEME_DRTT, SCHEME_A_RTT, SCHEME_SI = 0, 1, 2, 3, 4
BC_CHANNEL, BC_PERIODIC = 0, 1

_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build_oracle())
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        up = C.POINTER(C.c_ubyte)
        L.oracle_lattice.argtypes = [ip, ip, dp, ip]
        L.oracle_feq.argtypes = [C.c_double, C.c_double, C.c_double, dp]
        L.oracle_naca_mask.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                       C.c_double, C.c_double, C.c_int, up]
        L.oracle_naca_mask.restype = C.c_int
        L.oracle_cylinder_mask.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, up]
        L.oracle_cylinder_mask.restype = C.c_int
        L.oracle_naca_thickness.argtypes = [C.c_double, C.c_double, C.c_int]
        L.oracle_naca_thickness.restype = C.c_double
        L.oracle_links.argtypes = [up, C.c_int, C.c_int, C.c_int, ip, C.c_long]
        L.oracle_links.restype = C.c_long
        L.oracle_auto_cv.argtypes = [up, C.c_int, C.c_int, C.c_int, ip]
        L.oracle_create.argtypes = [up, C.c_int, C.c_int, C.c_double, dp, C.c_int, C.c_int,
                                    C.c_double, dp, ip]
        L.oracle_create.restype = C.c_void_p
        L.oracle_destroy.argtypes = [C.c_void_p]
        L.oracle_nlinks.argtypes = [C.c_void_p]
        L.oracle_nlinks.restype = C.c_long
        L.oracle_steps_done.argtypes = [C.c_void_p]
        L.oracle_steps_done.restype = C.c_long
        L.oracle_cv.argtypes = [C.c_void_p, ip]
        L.oracle_get_links.argtypes = [C.c_void_p, ip]
        L.oracle_get_populations.argtypes = [C.c_void_p, dp]
        L.oracle_set_populations.argtypes = [C.c_void_p, dp]
        L.oracle_step.argtypes = [C.c_void_p, C.c_int]
        L.oracle_step.restype = C.c_int
        L.oracle_force_series.argtypes = [C.c_void_p, C.c_int, C.c_long, C.c_long, dp, dp]
        L.oracle_force_series.restype = C.c_int
        L.oracle_surface_pressure.argtypes = [C.c_void_p, C.c_double, C.c_double, ip, dp, C.c_long,
                                              C.POINTER(C.c_long)]
        L.oracle_surface_pressure.restype = None
        L.oracle_drtt_parts.argtypes = [C.c_void_p, C.c_long, dp]
        L.oracle_drtt_parts.restype = C.c_int
        L.oracle_adjoint.argtypes = [up, C.c_int, C.c_int, C.c_double, dp, dp, C.c_int, C.c_int,
                                     C.c_double, C.c_double, dp, dp, dp, dp]
        L.oracle_adjoint.restype = C.c_int
        L.oracle_set_threads.argtypes = [C.c_int]
        L.oracle_set_threads.restype = C.c_int
        L.oracle_set_threads(1)
        _lib = L
    return _lib


def set_threads(n):
    """Host threads for the oracle's node loops; returns the count in use.
    The results are the same for any count."""
    return lib().oracle_set_threads(int(n))


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _up(a):
    return a.ctypes.data_as(C.POINTER(C.c_ubyte))


def lattice():
    """(cx, cy, w, opp) of the D2Q9 set, Table tabD2Q9."""
    cx = np.zeros(9, np.int32)
    cy = np.zeros(9, np.int32)
    w = np.zeros(9, np.float64)
    opp = np.zeros(9, np.int32)
    lib().oracle_lattice(_ip(cx), _ip(cy), _dp(w), _ip(opp))
    return cx, cy, w, opp


def feq(rho, ux, uy):
    out = np.zeros(9, np.float64)
    lib().oracle_feq(float(rho), float(ux), float(uy), _dp(out))
    return out


def cylinder_mask(nx, ny, xc, yc, diameter):
    """uint8 [ny][nx], 1 where (x - xc)^2 + (y - yc)^2 <= (diameter/2)^2."""
    out = np.zeros((ny, nx), np.uint8)
    rc = lib().oracle_cylinder_mask(int(nx), int(ny), float(xc), float(yc), 0.5 * float(diameter),
                                    out.ctypes.data_as(C.POINTER(C.c_ubyte)))
    if rc != 0:
        raise ValueError("bad cylinder arguments")
    return out


def naca_mask(nx, ny, chord, thickness, alpha_deg, xc, yc, closed_te=False):
    out = np.zeros((ny, nx), np.uint8)
    rc = lib().oracle_naca_mask(nx, ny, chord, thickness, alpha_deg, xc, yc, int(closed_te),
                                _up(out))
    if rc != 0:
        raise ValueError("bad NACA parameters")
    return out


def naca_thickness(s, thickness, closed_te=False):
    """Half-thickness y_t / C at s = xi / C."""
    return lib().oracle_naca_thickness(float(s), float(thickness), int(closed_te))


def links(mask, periodic_x=False):
    mask = np.ascontiguousarray(mask, np.uint8)
    ny, nx = mask.shape
    n = lib().oracle_links(_up(mask), nx, ny, int(periodic_x), None, 0)
    out = np.zeros(max(n, 1), np.int32)
    lib().oracle_links(_up(mask), nx, ny, int(periodic_x), _ip(out), n)
    return out[:n]


def auto_cv(mask, periodic_x=False):
    mask = np.ascontiguousarray(mask, np.uint8)
    ny, nx = mask.shape
    cv = np.zeros(4, np.int32)
    lib().oracle_auto_cv(_up(mask), nx, ny, int(periodic_x), _ip(cv))
    return cv


class Sim:
    """The oracle's solver state.  Populations are pre-collision f(x, t)."""

    def __init__(self, mask, tau, u_in, bc=BC_CHANNEL, rho0=1.0, body_force=None, cv=None):
        self.mask = np.ascontiguousarray(mask, np.uint8)
        self.ny, self.nx = self.mask.shape
        u = np.ascontiguousarray(np.atleast_1d(np.asarray(u_in, np.float64)))
        g = None if body_force is None else np.ascontiguousarray(body_force, np.float64)
        cva = None if cv is None else np.ascontiguousarray(cv, np.int32)
        self._h = lib().oracle_create(_up(self.mask), self.nx, self.ny, float(tau), _dp(u),
                                      int(u.size), int(bc), float(rho0),
                                      None if g is None else _dp(g),
                                      None if cva is None else _ip(cva))
        if not self._h:
            raise ValueError("oracle_create rejected its arguments")

    def close(self):
        if self._h:
            lib().oracle_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        if lib().oracle_step(self._h, int(n)) != 0:
            raise RuntimeError("oracle_step failed")

    @property
    def t(self):
        return lib().oracle_steps_done(self._h)

    @property
    def nlinks(self):
        return lib().oracle_nlinks(self._h)

    def links(self):
        out = np.zeros(max(self.nlinks, 1), np.int32)
        lib().oracle_get_links(self._h, _ip(out))
        return out[:self.nlinks]

    def cv(self):
        cv = np.zeros(4, np.int32)
        lib().oracle_cv(self._h, _ip(cv))
        return cv

    def populations(self):
        out = np.zeros((9, self.ny, self.nx), np.float64)
        lib().oracle_get_populations(self._h, _dp(out))
        return out

    def set_populations(self, f):
        f = np.ascontiguousarray(f, np.float64).reshape(9, self.ny, self.nx)
        lib().oracle_set_populations(self._h, _dp(f))

    def force_series(self, scheme, first=0, count=None):
        if count is None:
            count = self.t - first
        fx = np.zeros(max(count, 1), np.float64)
        fy = np.zeros(max(count, 1), np.float64)
        if lib().oracle_force_series(self._h, int(scheme), int(first), int(count), _dp(fx),
                                     _dp(fy)) != 0:
            raise IndexError("force series out of range")
        return fx[:count], fy[:count]

    def force(self, scheme):
        fx, fy = self.force_series(scheme, self.t - 1, 1)
        return float(fx[0]), float(fy[0])

    def surface_pressure(self, p_inf, q):
        """(nodes, cp): the boundary fluid nodes (ascending node index y*nx + x) and
        C_p = (p - p_inf)/q with p = rho/3 on the current pre-collision state."""
        cnt = C.c_long()
        lib().oracle_surface_pressure(self._h, float(p_inf), float(q), None, None, 0, C.byref(cnt))
        nodes = np.zeros(max(cnt.value, 1), np.int32)
        cp = np.zeros(max(cnt.value, 1), np.float64)
        lib().oracle_surface_pressure(self._h, float(p_inf), float(q), _ip(nodes), _dp(cp), cnt.value,
                                      C.byref(cnt))
        return nodes[:cnt.value], cp[:cnt.value]

    def drtt_parts(self, t):
        out = np.zeros(6, np.float64)
        if lib().oracle_drtt_parts(self._h, int(t), _dp(out)) != 0:
            raise IndexError("step out of range")
        return out


def adjoint(mask, tau, u_in, f0, steps, window, wx=1.0, wy=0.0):
    """J = window-average of wx Fx + wy Fy (algorithm B) after `steps` steps from
    f0, and dJ/dtau, dJ/du_in[ny], dJ/df0[9][ny][nx] (channel set-up)."""
    mask = np.ascontiguousarray(mask, np.uint8)
    ny, nx = mask.shape
    u = np.ascontiguousarray(np.broadcast_to(np.asarray(u_in, np.float64), (ny,)))
    f0 = np.ascontiguousarray(f0, np.float64).reshape(9, ny, nx)
    J = np.zeros(1)
    dtau = np.zeros(1)
    du = np.zeros(ny)
    df0 = np.zeros((9, ny, nx))
    rc = lib().oracle_adjoint(_up(mask), nx, ny, float(tau), _dp(u), _dp(f0), int(steps),
                              int(window), float(wx), float(wy), _dp(J), _dp(dtau), _dp(du),
                              _dp(df0))
    if rc != 0:
        raise ValueError("oracle_adjoint rejected its arguments")
    return float(J[0]), float(dtau[0]), du, df0
