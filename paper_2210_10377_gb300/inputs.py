"""Seeded synthetic inputs and named workloads.

This module holds no arithmetic of the method: it only names workload
parameters and draws seeded random numbers.  Both the CUDA path and the CPU
oracle are fed from here, and neither is imported by it.

Workloads follow the 2-D NACA0012 family of the paper's Section V (flow past a
2-D NACA0012 at Re = 1000, drag and lift by momentum exchange and by DRTT):
a NACA 00xx section in a channel with an equilibrium inlet, a zero-gradient
outlet and periodic top/bottom, inflow u_in = 0.05, rho0 = 1, uniform initial
equilibrium.  The relaxation time follows the lattice-unit relation
nu = (tau - 1/2)/3 with nu = u_in * chord / Re.
"""
from dataclasses import dataclass, field

import numpy as np

SEED = 2210


@dataclass(frozen=True)
class Workload:
    name: str
    nx: int
    ny: int
    chord: float
    thickness: float
    alpha_deg: float
    xc: float
    re: float
    steps: int
    storage: str
    u_in: float = 0.05
    rho0: float = 1.0
    extra: dict = field(default_factory=dict, compare=False, hash=False)

    @property
    def yc(self) -> float:
        # mid-chord on the domain's mid-line, so an alpha = 0 section is mirror-exact
        return (self.ny - 1) / 2.0

    @property
    def tau(self) -> float:
        return 0.5 + 3.0 * self.u_in * self.chord / self.re

    @property
    def nodes(self) -> int:
        return self.nx * self.ny


# The small FP64 case: 256 x 128, chord 32 at 0 deg centred at x = 80, Re = 100.
SMALL_F64 = Workload("naca0012_256x128_c32_a0_re100_f64", 256, 128, 32.0, 0.12, 0.0, 80.0,
                     100.0, 2000, "f64")
# The throughput case: 4096 x 2048, chord 256 at 4 deg, Re = 1000, FP32
# storage, as deviations f_i - w_i rho0 (the same 72 bytes a node update as
# plain FP32 values, and the one of the two that keeps the drag and lift
# within 1e-4 of the FP64 trajectory).
LARGE_F32 = Workload("naca0012_4096x2048_c256_a4_re1000_f32", 4096, 2048, 256.0, 0.12, 4.0,
                     1280.0, 1000.0, 50000, "f32dev")
# The precision case: 8192 x 4096, chord 512 at 6 deg, Re = 2000, FP16 / FP32 deviations.
PRECISION = Workload("naca0012_8192x4096_c512_a6_re2000_f16dev", 8192, 4096, 512.0, 0.12, 6.0,
                     2560.0, 2000.0, 20000, "f16dev")
# The differentiation case: 512 x 256, chord 64 at 2 deg, Re = 200, FP32
# deviations (FP32 forward, FP32 adjoint).
DIFF = Workload("naca0012_512x256_c64_a2_re200_f32", 512, 256, 64.0, 0.12, 2.0, 160.0, 200.0,
                4000, "f32dev")

WORKLOADS = {w.name: w for w in (SMALL_F64, LARGE_F32, PRECISION, DIFF)}


def cylinder(d: int, re: float = 100.0, storage: str = "f32", steps: int = 0) -> Workload:
    """Section VI: flow past a circular cylinder of diameter d (the `chord`
    field) at Re = u_in d / nu; domain 60 d x 5 d, centre 15 d from the inlet
    on the mid-line y = (ny - 1)/2 (Section VI's 12:1 aspect ratio)."""
    return Workload("cylinder_d%d_re%g" % (d, re), 60 * d, 5 * d, float(d), 0.0, 0.0, 15.0 * d, re,
                    steps, storage, extra={"body": "cylinder"})


def scaled(w: Workload, factor: int, storage: str = None) -> Workload:
    """The same geometry shrunk by an integer factor (for oracle-sized cases)."""
    return Workload(w.name + "_div%d" % factor, w.nx // factor, w.ny // factor,
                    w.chord / factor, w.thickness, w.alpha_deg, w.xc / factor,
                    w.re / factor, w.steps, storage or w.storage, w.u_in, w.rho0)


def rng(seed: int = SEED) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_blobs_mask(nx: int, ny: int, n_blobs: int, seed: int, max_radius: float = 4.0,
                      margin_x: int = 3) -> np.ndarray:
    """A uint8 [ny][nx] mask of random discs (1 = solid), kept off the first and
    last margin_x columns; discs may wrap through the top/bottom boundary."""
    g = rng(seed)
    mask = np.zeros((ny, nx), np.uint8)
    yy, xx = np.mgrid[0:ny, 0:nx]
    for _ in range(n_blobs):
        r = g.uniform(0.6, max_radius)
        cx = g.uniform(margin_x + r, nx - 1 - margin_x - r)
        cy = g.uniform(0, ny)
        dy = np.abs(yy - cy)
        dy = np.minimum(dy, ny - dy)
        mask[(xx - cx) ** 2 + dy ** 2 <= r * r] = 1
    mask[:, :margin_x] = 0
    mask[:, nx - margin_x:] = 0
    return mask


def random_populations(nx: int, ny: int, seed: int, lo: float = 0.02,
                       hi: float = 0.2) -> np.ndarray:
    """Random positive populations [9][ny][nx], uniform in [lo, hi)."""
    return rng(seed).uniform(lo, hi, size=(9, ny, nx))


def perturbation(nx: int, ny: int, seed: int = SEED, amp: float = 1e-3) -> np.ndarray:
    """Multiplicative factors 1 + U[-amp, amp], shape [9][ny][nx]."""
    return 1.0 + rng(seed).uniform(-amp, amp, size=(9, ny, nx))


def random_inlet(ny: int, seed: int, mean: float = 0.05, amp: float = 0.01) -> np.ndarray:
    """A per-row inlet velocity profile, mean +- amp, uniform random."""
    return mean + rng(seed).uniform(-amp, amp, size=ny)


def batch_instances(n: int = 256, seed: int = SEED):
    """Parameters of n independent NACA00xx instances: thickness U[0.08, 0.15],
    chord round(U[48, 128]), alpha U[-8, 8] deg, Re = 10**U[2, 3]; each domain
    8 chords x 4 chords with the mid-chord 2.5 chords from the inlet."""
    g = rng(seed)
    out = []
    for _ in range(n):
        t = g.uniform(0.08, 0.15)
        cb = int(round(g.uniform(48, 128)))
        a = g.uniform(-8.0, 8.0)
        re = 10.0 ** g.uniform(2.0, 3.0)
        out.append(Workload("naca00%02d_c%d" % (round(100 * t), cb), 8 * cb, 4 * cb, float(cb),
                            t, a, 2.5 * cb, re, 10000, "f32dev"))
    return out
