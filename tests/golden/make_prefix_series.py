"""Writes the stored FP64 oracle force series of a full-size workload's first
steps (a golden fixture for the GPU parity tests).  It runs only the oracle.

    python tests/golden/make_prefix_series.py WORKLOAD STEPS STRIDE OUT

WORKLOAD is a named workload, or one with the suffix _divK: the same geometry
shrunk K times (inputs.scaled).

Every STRIDE-th step t = 0, STRIDE, ... < STEPS gets one row: t, then F_x and
F_y of algorithm A (Eq. MEA on the pre-collision state), algorithm B (Eq.
rtt5), DRTT (Eq. rtt7), A' (Eq. rtt4) and stress integration (Eq.
stress_int), each the force of the transition t -> t+1.
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2210_10377_gb300 import inputs  # noqa: E402

SCHEMES = (("A", oracle.SCHEME_A), ("B", oracle.SCHEME_B), ("DRTT", oracle.SCHEME_DRTT),
           ("A_RTT", oracle.SCHEME_A_RTT), ("SI", oracle.SCHEME_SI))


def main():
    name, steps, stride, out = sys.argv[1], int(sys.argv[2]), int(sys.argv[3]), sys.argv[4]
    base, _, div = name.rpartition("_div")
    w = inputs.scaled(inputs.WORKLOADS[base], int(div)) if base and div.isdigit() else inputs.WORKLOADS[name]
    m = oracle.naca_mask(w.nx, w.ny, w.chord, w.thickness, w.alpha_deg, w.xc, w.yc)
    sim = oracle.Sim(m, w.tau, w.u_in)
    t0 = time.time()
    # one step past the window, so that DRTT of its last step is complete
    sim.step(steps + 1)
    series = {s: sim.force_series(k, 0, steps) for s, k in SCHEMES}
    with open(out, "w") as f:
        f.write("# FP64 oracle force series of workload %s (%dx%d, chord %g, alpha %g deg, Re %g,\n"
                "# tau %.10g, u_in %g), steps 0..%d, every %d-th step; written by\n"
                "# tests/golden/make_prefix_series.py from the oracle alone (%.0f s).\n"
                "# columns: t  A_x A_y  B_x B_y  DRTT_x DRTT_y  A'_x A'_y  SI_x SI_y\n"
                % (name, w.nx, w.ny, w.chord, w.alpha_deg, w.re, w.tau, w.u_in, steps - 1, stride,
                   time.time() - t0))
        for t in range(0, steps, stride):
            vals = []
            for s, _ in SCHEMES:
                fx, fy = series[s]
                vals += [fx[t], fy[t]]
            f.write("%d %s\n" % (t, " ".join("%.12e" % v for v in vals)))


if __name__ == "__main__":
    main()
