"""Precision of the FP32-force path against the FP64 oracle, per workload
family:

* energy: without a thermostat (gamma = 0), the total energy
  E = KE(stored velocities) + PE drifts no more on the GPU (FP32 forces, FP64
  integration; and the FP64 force mode) than in the FP64 oracle, up to the
  bounds written below;
* end-to-end distance: chain growth with reactions and the Langevin
  thermostat gives the same mean squared end-to-end distance of the chains
  on both sides (8 seeds each, within 3 standard errors).
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle as orc
import synth
from helpers import chain_ree2, gpu, gpu_reaction, gpu_system

pytestmark = pytest.mark.gpu
A, B = synth.TYPE_A, synth.TYPE_B
NVE_STEPS = 1000


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return gpu()


def oracle_energy_track(seed):
    inp = synth.step_growth(1000, 250, 4, seed)
    o = orc.System(inp.x, inp.v, inp.type, inp.state, cap=4)
    md = orc.MDParams(L=(inp.L,) * 3, seed=seed, gamma=0.0)
    e = []
    for _ in range(NVE_STEPS // 100):
        for _ in range(100):
            orc.step(o, md)
        e.append(0.5 * (o.v ** 2).sum() + orc.forces(o, md, use_cells=True)[1])
    return np.array(e)


def gpu_energy_track(P, seed, fp64):
    inp = synth.step_growth(1000, 250, 4, seed)
    with gpu_system(P, inp.L, inp.x, inp.v, inp.type, inp.state, cap=4, seed=seed, gamma=0.0,
                    fp64=fp64) as g:
        e = []
        for _ in range(NVE_STEPS // 100):
            g.run(100)
            e.append(g.observables()["ke_half"] + g.forces()[1])
        return np.array(e)


def test_nve_energy_drift_against_the_oracle(P):
    seed = 77
    e_o = oracle_energy_track(seed)
    e_64 = gpu_energy_track(P, seed, True)
    e_32 = gpu_energy_track(P, seed, False)
    d = {k: float(np.abs(v - v[0]).max() / abs(v[0])) for k, v in
         (("oracle", e_o), ("gpu_fp64", e_64), ("gpu_fp32", e_32))}
    assert d["gpu_fp64"] <= 2.0 * d["oracle"] + 1e-6, d
    assert d["gpu_fp32"] <= 5.0 * d["oracle"] + 2e-5, d


def oracle_chains(seed):
    inp = synth.chain_growth(2970, 30, seed)
    o = orc.System(inp.x, inp.v, inp.type, inp.state, cap=2)
    md = orc.MDParams(L=(inp.L,) * 3, seed=seed)
    orc.run(o, md, orc.Reaction(**synth.chain_growth_scheme(k=1.0)), 2000)
    b = o.bonds()
    return chain_ree2(o.x, b[:, 1:3], o.type, o.state, inp.L)


def test_end_to_end_distance_against_the_oracle(P):
    seeds = [synth.BASE_SEED + 500 + s for s in range(8)]
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        pending = pool.map_async(oracle_chains, seeds)
        r_g = []
        for seed in seeds:
            inp = synth.chain_growth(2970, 30, seed)
            with gpu_system(P, inp.L, inp.x, inp.v, inp.type, inp.state, cap=2, seed=seed) as g:
                g.set_reaction(gpu_reaction(P, synth.chain_growth_scheme(k=1.0)))
                g.run(2000)
                b = g.bonds()
                r_g.append(np.mean(chain_ree2(g.positions(), np.stack([b["a"], b["t"]], 1),
                                              g.types(), g.states(), inp.L)))
        r_o = [np.mean(v) for v in pending.get()]
    mg, mo = np.mean(r_g), np.mean(r_o)
    se = np.hypot(np.std(r_g, ddof=1), np.std(r_o, ddof=1)) / np.sqrt(len(seeds))
    assert abs(mg - mo) <= 3 * se, (mg, mo, se)
    assert mg > 5.0  # chains of a few bonds at least
