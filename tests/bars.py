"""Relative error measures of a force series against the FP64 oracle's,
shared by the GPU parity tests (not a test module).

Drag and lift coefficients C = 2F/(rho0 U^2 L) (Section V) differ from the
forces by one constant factor, so their relative errors are the forces'.  A
series F(t) = (F_x(t), F_y(t)) is judged:

- step by step, on the scale S(t) = max over the window's steps s >= min(t,
  n/2) of max(|F_x(s)|, |F_y(s)|) of the oracle (n steps in the window).
  Steps of the back half are judged against the largest force of the back
  half, and an earlier step against the largest force from itself onwards, so
  the force of the impulsive start (t = 0, tens of times the later forces)
  judges only itself and the steps of its own decay.  A component near zero
  (the lift of a symmetric section) is judged on the scale of the other one.
- as window means, over the window's back half (after the start-up
  transient), relative to max(|mean F_x|, |mean F_y|) of the oracle.
"""
import numpy as np


def envelope(o):
    """S(t) = max over s >= min(t, n/2) of max(|F_x(s)|, |F_y(s)|)."""
    mag = np.abs(np.asarray(o, dtype=np.float64)).max(axis=0)
    env = np.maximum.accumulate(mag[::-1])[::-1]
    h = mag.size // 2
    env[h:] = env[h]
    return env


def step_error(g, o):
    """max over steps of max(|dF_x|, |dF_y|)(t) / S(t)."""
    g, o = np.asarray(g, dtype=np.float64), np.asarray(o, dtype=np.float64)
    return float((np.abs(g - o).max(axis=0) / np.maximum(envelope(o), 1e-300)).max())


def mean_error(g, o):
    """|mean(F_gpu) - mean(F_oracle)| over the back half, relative to the
    larger oracle mean component."""
    g, o = np.asarray(g, dtype=np.float64), np.asarray(o, dtype=np.float64)
    h = o.shape[1] // 2
    mo, mg = o[:, h:].mean(axis=1), g[:, h:].mean(axis=1)
    return float(np.abs(mg - mo).max() / max(np.abs(mo).max(), 1e-300))
