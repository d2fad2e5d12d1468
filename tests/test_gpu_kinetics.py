"""Kinetics on the GPU against the FP64 oracle and the paper's rate equations.

* Step growth (config 1: 1,000 B + 250 A of functionality 4, k = 0.1):
  conversion and crosslinker populations x_s(t), averaged over 32 seeds on
  each side, agree within the combined standard error (criterion below).
  Trajectories decorrelate, so this parity is statistical.
* g(r) -> <N> -> rate equation: the GPU pair histogram equals the oracle's,
  count for count; chain growth (config 2, k = 0.01) then follows the
  polymer fraction of Sec. II.A with the <N_P*M> measured on the same runs,
  and the LAMMPS nearest-partner rule does not (Fig. 2 of the paper).
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle as orc
import synth
from helpers import gpu, gpu_reaction, gpu_system, md_params, oracle_system
from paper_1409_7498_gb300 import kinetics as kin

pytestmark = pytest.mark.gpu

SEEDS = 32
NSTEPS = 2000
WARMUP = 2000  # MD steps without reactions before a chain-growth run
A, B = synth.TYPE_A, synth.TYPE_B


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return gpu()


def cfg1(seed):
    return synth.step_growth(1000, 250, 4, seed)


def curves_from_counts(bonds, countsA):
    """conversion (bonds over 4 x 250 sites) and x_s (s = bonds formed)."""
    conv = bonds / 1000.0
    xs = countsA[..., 4::-1] / 250.0  # state 4 - s -> s bonds formed
    return np.concatenate([conv[..., None], xs], axis=-1)


def oracle_run(seed):
    inp = cfg1(seed)
    o = orc.System(inp.x, inp.v, inp.type, inp.state, cap=4)
    md = orc.MDParams(L=(inp.L,) * 3, seed=seed)
    obs = orc.run(o, md, orc.Reaction(**synth.step_growth_scheme(4, k=0.1)), NSTEPS)
    bonds = np.array([ob["bonds"] for ob in obs], np.float64)
    cA = np.array([ob["counts"][A][:5] for ob in obs], np.float64)
    return curves_from_counts(bonds, cA)


def test_step_growth_kinetics_32_seeds_match_the_oracle(P):
    seeds = [synth.BASE_SEED + s for s in range(SEEDS)]
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        pending = pool.map_async(oracle_run, seeds)
        # GPU: the 32 replicas advance together in one batch
        systems = []
        for seed in seeds:
            inp = cfg1(seed)
            g = gpu_system(P, inp.L, inp.x, inp.v, inp.type, inp.state, cap=4, seed=seed)
            g.set_reaction(gpu_reaction(P, synth.step_growth_scheme(4, k=0.1)))
            systems.append(g)
        with P.Batch() as b:
            for g in systems:
                b.add(g)
            b.run(NSTEPS)
            b.sync()
        gpu_curves = []
        for g in systems:
            h = g.history()
            gpu_curves.append(curves_from_counts(h["bonds"].astype(np.float64),
                                                 h["counts"][:, A, :5].astype(np.float64)))
            g.close()
        orc_curves = np.array(pending.get())
    gpu_curves = np.array(gpu_curves)
    assert gpu_curves.shape == orc_curves.shape == (SEEDS, NSTEPS // 10, 6)
    idx = np.arange(19, NSTEPS // 10, 20)  # ten sample times
    mg, mo = gpu_curves[:, idx].mean(0), orc_curves[:, idx].mean(0)
    se = np.sqrt(gpu_curves[:, idx].var(0, ddof=1) / SEEDS + orc_curves[:, idx].var(0, ddof=1) / SEEDS)
    z = np.abs(mg - mo) / np.maximum(se, 1e-12)
    # within 2 combined standard errors at (nearly) every point, none beyond 3.5
    assert (z <= 2.0).mean() >= 0.9 and z.max() <= 3.5, z
    assert mg[-1, 0] > 0.3  # the runs went far enough to test something


def test_pair_histogram_matches_the_oracle(P):
    inp = synth.step_growth_sites(6000, 4, 21, jitter=0.5)
    o = oracle_system(inp.x, inp.v, inp.type, inp.state, 4)
    md = md_params(inp.L, 21)
    with gpu_system(P, inp.L, inp.x, inp.v, inp.type, inp.state, cap=4, seed=21) as g:
        for a, b in [((1 << A, 1, 4), (1 << B, 0, 1)), ((1 << B, 0, 1), (1 << B, 0, 1)),
                     ((0xFF, -128, 127), (1 << A, 4, 4))]:
            cg, nag, nbg = g.pair_histogram(a, b, 1.1, 22)
            co, nao, nbo = orc.pair_histogram(o, md, a, b, 1.1, 22)
            assert nag == nao and nbg == nbo
            assert np.array_equal(cg, co)
            assert cg.sum() > 100
        with pytest.raises(P.PolyrxError):
            g.pair_histogram((1, 0, 0), (1, 0, 0), 2.0, 10)  # beyond the guaranteed cutoff


def chain_runs(P, selection, seeds, nsteps, k):
    """phi(t) per seed (from the reaction history) and <N_P*M> sampled every
    2,000 steps from the pair histogram."""
    P_star, M = ((1 << A) | (1 << B), 2, 2), (1 << B, 0, 0)
    systems = []
    for seed in seeds:
        inp = synth.chain_growth(32768, 328, seed)
        g = gpu_system(P, inp.L, inp.x, inp.v, inp.type, inp.state, cap=2, seed=seed)
        g.run(WARMUP)  # melt the initial lattice before the reaction starts
        g.set_reaction(gpu_reaction(P, synth.chain_growth_scheme(k=k, selection=selection)))
        systems.append(g)
    pairs = na = 0
    with P.Batch() as b:
        for g in systems:
            b.add(g)
        for _ in range(nsteps // 2000):
            b.run(2000)
            b.sync()
            for g in systems:
                c, a_, _ = P.prx_pair_histogram(g.h, P_star, M, 1.1, 11)
                pairs += int(c.sum())
                na += a_
    phis = []
    for g in systems:
        h = g.history()
        n = 33096
        phis.append((n - h["counts"][:, B, 0]) / n)  # everything but free monomers
        g.close()
    return np.array(phis), pairs / na


def test_chain_growth_follows_the_rate_equation_and_nearest_does_not(P):
    seeds = [synth.BASE_SEED + 100 + s for s in range(8)]
    k, nsteps, phi0 = 0.01, 20000, 328 / 33096
    t = 0.005 * 10 * np.arange(1, nsteps // 10 + 1)
    phi_r, n_r = chain_runs(P, 0, seeds, nsteps, k)
    phi_n, _ = chain_runs(P, 1, seeds, nsteps, k)
    theory = kin.polymer_fraction(t, k, n_r, phi0)
    grown_sim = phi_r.mean(0)[-1] - phi0
    grown_th = theory[-1] - phi0
    se = phi_r[:, -1].std(ddof=1) / np.sqrt(len(seeds))
    # Sec. V: at k = 0.01 simulation and theory are indistinguishable
    assert abs(grown_sim - grown_th) <= max(3 * se, 0.05 * grown_th), (grown_sim, grown_th, se)
    # Fig. 2: the nearest-partner rule grows the chains at another rate
    grown_near = phi_n.mean(0)[-1] - phi0
    se_n = phi_n[:, -1].std(ddof=1) / np.sqrt(len(seeds))
    assert abs(grown_near - grown_sim) > 4 * np.hypot(se, se_n), (grown_near, grown_sim)
    assert 2.0 < n_r < 5.0  # <N_P*M> near the paper's 3.25
