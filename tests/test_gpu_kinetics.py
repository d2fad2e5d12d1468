"""Kinetics on the GPU against the FP64 oracle and the paper's rate equations.

* Step growth (config 1: 1,000 B + 250 A of functionality 4, k = 0.1):
  conversion and crosslinker populations x_s(t), averaged over 32 seeds on
  each side, agree within the combined standard error (criterion below).
  Trajectories decorrelate, so this parity is statistical.
* Chain growth (2,970 M + 30 initiators, k = 0.5): the polymer fraction and
  the fraction of initiators that reacted, 32 seeds on each side, agree
  within the combined standard error (same criterion).
* g(r) -> <N> -> rate equation: the GPU pair histogram equals the oracle's,
  count for count; chain growth (config 2, k = 0.01) then follows the rate
  law of Sec. II.A (Eq. 10: monomers consumed at k <N_P*M> per active end)
  window by window, with <N_P*M> measured in the same window, within two
  standard errors of the bond counts, and the LAMMPS nearest-partner rule
  does not (Fig. 2 of the paper).
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle as orc
import synth
from helpers import gpu, gpu_reaction, gpu_system, md_params, oracle_system

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


def chain_small(seed):
    return synth.chain_growth(2970, 30, seed)


def chain_curves(counts):
    """polymer fraction (all but free monomers) and the fraction of the 30
    initiators that reacted, from per-reaction populations counts[..., type, state]."""
    phi = (3000.0 - counts[..., B, 0]) / 3000.0
    init = counts[..., A, 1] / 30.0
    return np.stack([phi, init], axis=-1)


def oracle_chain_run(seed):
    inp = chain_small(seed)
    o = orc.System(inp.x, inp.v, inp.type, inp.state, cap=2)
    md = orc.MDParams(L=(inp.L,) * 3, seed=seed)
    obs = orc.run(o, md, orc.Reaction(**synth.chain_growth_scheme(k=0.5)), NSTEPS)
    return chain_curves(np.array([ob["counts"] for ob in obs], np.float64))


def test_chain_growth_kinetics_32_seeds_match_the_oracle(P):
    seeds = [synth.BASE_SEED + 700 + s for s in range(SEEDS)]
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        pending = pool.map_async(oracle_chain_run, seeds)
        systems = []
        for seed in seeds:
            inp = chain_small(seed)
            g = gpu_system(P, inp.L, inp.x, inp.v, inp.type, inp.state, cap=2, seed=seed)
            g.set_reaction(gpu_reaction(P, synth.chain_growth_scheme(k=0.5)))
            systems.append(g)
        with P.Batch() as b:
            for g in systems:
                b.add(g)
            b.run(NSTEPS)
            b.sync()
        gpu_curves = []
        for g in systems:
            gpu_curves.append(chain_curves(g.history()["counts"].astype(np.float64)))
            g.close()
        orc_curves = np.array(pending.get())
    gpu_curves = np.array(gpu_curves)
    assert gpu_curves.shape == orc_curves.shape == (SEEDS, NSTEPS // 10, 2)
    idx = np.arange(19, NSTEPS // 10, 20)  # ten sample times
    mg, mo = gpu_curves[:, idx].mean(0), orc_curves[:, idx].mean(0)
    se = np.sqrt(gpu_curves[:, idx].var(0, ddof=1) / SEEDS + orc_curves[:, idx].var(0, ddof=1) / SEEDS)
    z = np.abs(mg - mo) / np.maximum(se, 1e-12)
    print("chain growth 32 seeds, |z| of (polymer fraction, initiators reacted) at ten times:",
          np.round(z, 2).tolist())
    assert (z <= 2.0).mean() >= 0.9 and z.max() <= 3.5, z
    assert mg[-1, 0] > 0.1 and mg[-1, 1] > 0.8  # the chains grew


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


SAMPLE = 500  # MD steps between samples of <N_P*M>


def chain_runs(P, selection, seeds, nsteps, k):
    """Per seed: bonds at every reaction step (from the reaction history) and
    <N_P*M> (monomers within r_react per active end, from the pair
    histogram) every SAMPLE steps from t = 0."""
    P_star, M = ((1 << A) | (1 << B), 2, 2), (1 << B, 0, 0)
    systems = []
    for seed in seeds:
        inp = synth.chain_growth(32768, 328, seed)
        g = gpu_system(P, inp.L, inp.x, inp.v, inp.type, inp.state, cap=2, seed=seed)
        g.run(WARMUP)  # melt the initial lattice before the reaction starts
        g.set_reaction(gpu_reaction(P, synth.chain_growth_scheme(k=k, selection=selection)))
        systems.append(g)
    nsamp = nsteps // SAMPLE + 1
    n_t = np.zeros((len(seeds), nsamp))
    with P.Batch() as b:
        for g in systems:
            b.add(g)
        for q in range(nsamp):
            if q:
                b.run(SAMPLE)
                b.sync()
            for r, g in enumerate(systems):
                c, a_, _ = P.prx_pair_histogram(g.h, P_star, M, 1.1, 11)
                n_t[r, q] = c.sum() / a_
    bonds = []
    for g in systems:
        bonds.append(g.history()["bonds"].astype(np.float64))
        g.close()
    return np.array(bonds), n_t


def test_chain_growth_follows_the_rate_equation_and_nearest_does_not(P):
    """Eq. 10's rate law: an active end consumes monomers at k per monomer in
    range, so the bonds formed at a reaction step have the mean
    p n_P* <N_P*M> (p = k dt Theta; selection conflicts are O(p) rarer at
    k = 0.01).  Over each window of 2,000 steps the bonds formed (8 seeds
    pooled) must agree with the prediction from the <N_P*M> measured in that
    window (sampled every 500 steps, linear in between) within 2 standard
    errors of the (Poisson) bond count at nine of ten windows or more, none
    beyond 3.5, and in total within 2."""
    seeds = [synth.BASE_SEED + 100 + s for s in range(8)]
    k, nsteps, n_init, theta, dt = 0.01, 20000, 328, 10, 0.005
    p = k * dt * theta
    bonds_r, n_r = chain_runs(P, 0, seeds, nsteps, k)
    steps = theta * np.arange(1, nsteps // theta + 1)
    samples = SAMPLE * np.arange(n_r.shape[1])
    n_at = np.array([np.interp(steps, samples, n_r[r]) for r in range(len(seeds))])
    expected = p * n_init * n_at  # mean bonds formed at each reaction step, per seed
    formed = np.diff(np.concatenate([np.zeros((len(seeds), 1)), bonds_r], axis=1), axis=1)
    win = 2000 // theta
    e_w = expected.sum(0).reshape(-1, win).sum(1)
    f_w = formed.sum(0).reshape(-1, win).sum(1)
    z = (f_w - e_w) / np.sqrt(e_w)
    assert (np.abs(z) <= 2.0).mean() >= 0.9 and np.abs(z).max() <= 3.5, (z, f_w, e_w)
    z_tot = (f_w.sum() - e_w.sum()) / np.sqrt(e_w.sum())
    print(f"chain growth k = 0.01, 8 seeds: <N_P*M> {n_r[:, 0].mean():.3f} -> "
          f"{n_r[:, -1].mean():.3f}; bonds per 2,000-step window formed / predicted "
          f"{np.round(f_w).astype(int).tolist()} / {np.round(e_w, 1).tolist()}; "
          f"z {np.round(z, 2).tolist()}, total z {z_tot:.2f}")
    assert abs(z_tot) <= 2.0, (z_tot, f_w.sum(), e_w.sum())
    assert 2.0 < n_r[:, 0].mean() < 5.0  # <N_P*M> near the paper's 3.25 at the start
    assert n_r[:, -1].mean() < n_r[:, 0].mean()  # the monomers around the ends deplete
    # Fig. 2: the nearest-partner rule grows the chains at another rate
    bonds_n, _ = chain_runs(P, 1, seeds, nsteps, k)
    grown_r, grown_n = bonds_r[:, -1], bonds_n[:, -1]
    se = np.hypot(grown_r.std(ddof=1), grown_n.std(ddof=1)) / np.sqrt(len(seeds))
    assert abs(grown_n.mean() - grown_r.mean()) > 4 * se, (grown_n.mean(), grown_r.mean())
