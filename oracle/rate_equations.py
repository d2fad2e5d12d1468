"""Rate equations of the paper, for validating kinetics (TEST INFRASTRUCTURE).

* Chain growth, Sec. II.A: with [P*] constant the monomers decay as
  [M](t) = [M0] exp(-k_c [P*] t) and the polymer fraction is Eq. 10,
  phi(t) = 1 - (1 - phi0) exp(-k_c [P*] t), where k_c = k <N_P*M> / rho and
  [P*] = rho phi0, so k_c [P*] = k <N_P*M> phi0.
* Step growth, Sec. II.B, Eq. 12: crosslinker populations X_s (s = bonds
  formed, X_0 the fresh crosslinkers, x_0(0) = 1) obey
      dX_0/dt = -k_0 X_0,
      dX_s/dt = -k_s X_s + k_{s-1} X_{s-1}   (0 < s < f),
      dX_f/dt =  k_{f-1} X_{f-1},
  with k_s = <N_{X^s E^0}> k (Eq. 13).  The paper integrates it with SciPy's
  odeint; here a classical fourth-order Runge-Kutta integrator written out
  step by step does the same job.
"""
from __future__ import annotations

import numpy as np


def chain_fraction(t, k: float, n_avg: float, phi0: float, approximate: bool = False):
    """Eq. 10.  `approximate` drops the (1 - phi0) prefactor (last line of Eq. 10)."""
    t = np.asarray(t, dtype=np.float64)
    rate = k * n_avg * phi0
    if approximate:
        return 1.0 - np.exp(-rate * t)
    return 1.0 - (1.0 - phi0) * np.exp(-rate * t)


def step_rhs(x: np.ndarray, ks: np.ndarray) -> np.ndarray:
    """Right-hand side of Eq. 12 for fractions x[0..f]; ks[s] for s = 0..f-1."""
    f = len(x) - 1
    d = np.zeros_like(x)
    if f == 0:
        return d
    d[0] = -ks[0] * x[0]
    for s in range(1, f):
        d[s] = -ks[s] * x[s] + ks[s - 1] * x[s - 1]
    d[f] = ks[f - 1] * x[f - 1]
    return d


def step_kinetics(t_out, ks, f: int, dt: float = 1e-3):
    """x_s(t) (Eq. 14) at the times t_out, from x_0 = 1, by RK4 with step <= dt."""
    ks = np.asarray(ks, dtype=np.float64)
    if len(ks) < f:
        raise ValueError("need k_s for s = 0..f-1")
    t_out = np.asarray(t_out, dtype=np.float64)
    x = np.zeros(f + 1)
    x[0] = 1.0
    out = np.zeros((len(t_out), f + 1))
    t = 0.0
    for i, te in enumerate(t_out):
        while t < te:
            h = min(dt, te - t)
            k1 = step_rhs(x, ks)
            k2 = step_rhs(x + 0.5 * h * k1, ks)
            k3 = step_rhs(x + 0.5 * h * k2, ks)
            k4 = step_rhs(x + h * k3, ks)
            x = x + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
            t += h
        out[i] = x
    return out
