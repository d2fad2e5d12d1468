"""From pair histograms to the rate-equation predictions of the paper.

* g_ab(r) and <N_ab> (Secs. V-VI): the mean number of available partners of
  class b around a particle of class a within the reaction cutoff is the
  integral of rho_b g_ab(r) 4 pi r^2 up to the cutoff, i.e. the pair count
  per a-particle; prx_pair_histogram supplies the counts on the device.
* Chain growth (Sec. II.A): with a constant number of active ends the
  polymer fraction is phi(t) = 1 - (1 - phi0) exp(-k_c [P*] t), and
  k_c [P*] = k <N_P*M> phi0 (k_c = k <N> / rho, [P*] = rho phi0).
* Step growth (Sec. II.B, Eq. step-kin): the crosslinker populations obey a
  linear chain X_0 -> X_1 -> ... -> X_f with rates k_s = k <N_X^s E^0>,
  indexed here by the number of bonds formed s; solved exactly with a
  matrix exponential.

Plain host arithmetic on a few numbers per call; every simulation step stays
in the library's kernels.
"""
from __future__ import annotations

import numpy as np


def radial_distribution(counts, n_a: int, n_b: int, volume: float, r_max: float,
                        samples: int = 1, same_class: bool = False):
    """(r of the bin centres, g(r)) from summed pair counts: the counts over
    the ideal-gas expectation n_a rho_b V_shell per sample."""
    counts = np.asarray(counts, dtype=np.float64)
    nbins = len(counts)
    edges = r_max * np.arange(nbins + 1) / nbins
    shell = 4.0 / 3.0 * np.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
    rho_b = (n_b - 1 if same_class else n_b) / volume
    ideal = samples * n_a * rho_b * shell
    with np.errstate(divide="ignore", invalid="ignore"):
        g = np.where(ideal > 0, counts / ideal, 0.0)
    return 0.5 * (edges[1:] + edges[:-1]), g


def mean_partners(counts, n_a: int, samples: int = 1) -> float:
    """<N_ab> = rho_b int_0^r_max g_ab(r) 4 pi r^2 dr = pairs per a-particle."""
    return float(np.sum(counts)) / (samples * n_a) if n_a else 0.0


def polymer_fraction(t, k: float, n_mean: float, phi0: float):
    """Chain growth, Sec. II.A: phi(t) = 1 - (1 - phi0) exp(-k <N> phi0 t)."""
    t = np.asarray(t, dtype=np.float64)
    return 1.0 - (1.0 - phi0) * np.exp(-k * n_mean * phi0 * t)


def crosslinker_fractions(t, k: float, n_s, f: int):
    """Step growth: x_s(t), s = bonds formed (0..f), from x_0(0) = 1, for the
    linear chain with rates k n_s[s] (s = 0..f-1); exact, by the matrix
    exponential of the rate matrix."""
    from scipy.linalg import expm
    rates = k * np.asarray(n_s, dtype=np.float64)[:f]
    A = np.zeros((f + 1, f + 1))
    for s in range(f):
        A[s, s] -= rates[s]
        A[s + 1, s] += rates[s]
    x0 = np.zeros(f + 1)
    x0[0] = 1.0
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    return np.stack([expm(A * tt) @ x0 for tt in t])
