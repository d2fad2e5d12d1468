"""The host-side kinetics module of the package against the oracle's rate
equations (two independent writings: a closed form and a matrix exponential
here, a written-out Runge-Kutta integration there) and against closed forms."""
import numpy as np

from oracle import rate_equations as req
from paper_1409_7498_gb300 import kinetics as kin


def test_polymer_fraction_matches_the_oracle_and_limits():
    t = np.linspace(0, 200, 41)
    a = kin.polymer_fraction(t, k=0.01, n_mean=3.25, phi0=0.0099)
    b = req.chain_fraction(t, k=0.01, n_avg=3.25, phi0=0.0099)
    assert np.allclose(a, b, rtol=0, atol=1e-14)
    assert abs(a[0] - 0.0099) < 1e-15 and np.all(np.diff(a) > 0)


def test_crosslinker_fractions_match_runge_kutta():
    t = np.array([0.0, 1.0, 5.0, 20.0, 80.0])
    n_s = [1.30, 0.890, 0.572, 0.327, 0.137, 0.0128]
    for f in (1, 2, 4, 6):
        a = kin.crosslinker_fractions(t, 0.1, n_s, f)
        b = req.step_kinetics(t, 0.1 * np.asarray(n_s[:f]), f, dt=1e-3)
        assert np.allclose(a, b, rtol=0, atol=1e-9)
        assert np.allclose(a.sum(1), 1.0)
    # f = 1: x_0 = exp(-k0 t)
    a = kin.crosslinker_fractions(t, 0.1, [2.0], 1)
    assert np.allclose(a[:, 0], np.exp(-0.2 * t), rtol=1e-12)


def test_rdf_normalisation_and_mean_partners():
    # an ideal gas histogram gives g = 1 and <N> = rho V_sphere
    n_a, n_b, V, r_max, nb = 1000, 2000, 1000.0, 1.5, 30
    edges = r_max * np.arange(nb + 1) / nb
    counts = n_a * n_b / V * 4 / 3 * np.pi * np.diff(edges ** 3)
    r, g = kin.radial_distribution(counts, n_a, n_b, V, r_max)
    assert np.allclose(g, 1.0)
    assert abs(kin.mean_partners(counts, n_a) - n_b / V * 4 / 3 * np.pi * r_max ** 3) < 1e-9
