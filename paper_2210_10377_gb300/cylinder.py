"""Flow past a circular cylinder (Section VI): the drag coefficient against
grid resolution and against the Reynolds number for every force scheme, and
the pressure coefficient on the cylinder's boundary nodes.

The resolutions run together as one batch of uneven domains (lbm_batch_*), so
a whole convergence study is one sequence of batched launches.  Each domain is
60 D x 5 D with the cylinder centre 15 D from the inlet on the mid-line,
Re = u_in D / nu = 100 by default, u_in = 0.05, rho0 = 1.

  C_d = 2 |F_x| / (rho0 u_in^2 D)        (Section VI)
  C_p = (p - p_inf) / (rho0 u_in^2 / 2),  p = rho / 3,  p_inf = rho0 / 3

Cd is averaged over the last `window` steps; the lift's standard deviation
over the same window tells whether vortex shedding has set in.  Both come
from the library (lbm_batch_coefficients: signed window mean and standard
deviation, computed on the device); the studies only quote |mean C_d| as the
paper does.
"""
import numpy as np

from . import binding, inputs

SCHEMES = ("A", "B", "DRTT", "SI")


def domains(diameters, re=100.0):
    ws = [inputs.cylinder(int(d), re) for d in diameters]
    doms = [{"mask": binding.body_mask(w), "tau": w.tau, "u_in": w.u_in} for w in ws]
    return ws, doms


def cd_study(diameters=(10, 15, 20, 30, 40), re=100.0, flow_times=100.0, window_flow_times=40.0,
             storage="f32", autotune=True, device=0):
    """Cd of every scheme per diameter.  The run lasts `flow_times` convective
    times D_max / u_in of the largest cylinder (all domains take the same
    number of steps); Cd is averaged over the last `window_flow_times` of them.
    Returns a dict with the steps, the window and one row per diameter."""
    ws, doms = domains(diameters, re)
    u = ws[0].u_in
    dmax = max(diameters)
    steps = int(round(flow_times * dmax / u))
    window = int(round(window_flow_times * dmax / u))
    b = binding.Batch(doms, storage=storage, device=device)
    if autotune:
        b.autotune(trials=3)
    b.step(steps)
    rows = []
    for k, (w, d) in enumerate(zip(ws, diameters)):
        row = {"D": int(d), "nx": w.nx, "ny": w.ny, "tau": round(w.tau, 6)}
        for s in SCHEMES:
            _, _, (cd, cl, cd_std, cl_std) = b.coefficients(k, s, float(d), u, steps - window, window)
            row["Cd_" + s] = abs(cd)
            row["Cl_std_" + s] = cl_std
        rows.append(row)
    flags, _ = b.status()
    out = {"re": re, "steps": steps, "window": window, "storage": storage, "rows": rows,
           "unstable_domains": int(flags.sum()), "nodes": b.nodes}
    b.close()
    return out


def cd_vs_re(d=20, res=(20.0, 40.0, 60.0, 100.0, 150.0, 200.0), flow_times=100.0, window_flow_times=40.0,
             storage="f32", device=0):
    """Cd of every scheme against the Reynolds number at one resolution
    (Section VI's second cylinder study): the same 60 d x 5 d geometry at each
    Re, tau = 1/2 + 3 u_in d / Re, all run as one batch."""
    ws = [inputs.cylinder(int(d), re) for re in res]
    mask = binding.body_mask(ws[0])
    doms = [{"mask": mask, "tau": w.tau, "u_in": w.u_in} for w in ws]
    u = ws[0].u_in
    steps = int(round(flow_times * d / u))
    window = int(round(window_flow_times * d / u))
    b = binding.Batch(doms, storage=storage, device=device)
    b.autotune(trials=3)
    b.step(steps)
    rows = []
    for k, (w, re) in enumerate(zip(ws, res)):
        row = {"Re": float(re), "tau": round(w.tau, 6)}
        for s_ in SCHEMES:
            _, _, (cd, cl, cd_std, cl_std) = b.coefficients(k, s_, float(d), u, steps - window, window)
            row["Cd_" + s_] = abs(cd)
            row["Cl_std_" + s_] = cl_std
        rows.append(row)
    flags, _ = b.status()
    out = {"D": int(d), "steps": steps, "window": window, "storage": storage, "rows": rows,
           "unstable_domains": int(flags.sum())}
    b.close()
    return out


def pressure_profile(d=40, re=100.0, flow_times=100.0, storage="f32", device=0):
    """C_p against the angle theta (degrees, 0 = the front stagnation point,
    measured from the upstream direction) at the boundary fluid nodes of one
    cylinder at the end of the run."""
    w = inputs.cylinder(int(d), re)
    lat = binding.Lattice(binding.body_mask(w), w.tau, w.u_in, storage=storage, device=device)
    lat.step(int(round(flow_times * d / w.u_in)))
    nodes, cp = lat.pressure_coefficient(w.rho0 / 3.0, 0.5 * w.rho0 * w.u_in ** 2)
    x, y = nodes % w.nx, nodes // w.nx
    theta = np.degrees(np.arctan2(y - w.yc, -(x - w.xc)))
    lat.close()
    order = np.argsort(theta)
    return theta[order], cp[order]
