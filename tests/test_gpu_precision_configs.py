"""Precision against the FP64 oracle at the sizes of the benchmark workloads,
from their warmed-liquid starts (uniform placement relaxed by the capped-force
warm-up, the workloads' recipe):

* 33,096-bead chain growth (FP32 forces, FP64 integration): without a
  thermostat, the relative excursion of the total energy over 1,000 steps on
  the GPU (FP32 forces, and the FP64 force mode) against the oracle's on the
  same start; with reactions (k = 1) and the thermostat, the mean squared
  end-to-end distance of the chains after 1,000 steps, four seeds on each
  side, within 3 standard errors (chains pooled);
* 1,048,576-bead step growth (FP32 forces): the energy excursion over a
  200-step slice against the oracle's on the same start.

The excursion of the FP32-force path must stay within 5x the oracle's plus
2e-5 (and the FP64 mode within 2x plus 1e-6); the measured values are
printed for the record.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle as orc
import synth
from helpers import chain_ree2, gpu

pytestmark = pytest.mark.gpu
A, B = synth.TYPE_A, synth.TYPE_B


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return gpu()


def excursion(e):
    e = np.asarray(e)
    return float(np.abs(e - e[0]).max() / abs(e[0]))


def gpu_energy(P, inp, x, v, cap, seed, fp64, steps, every):
    desc = P.make_desc(inp.n, inp.L, adj_cap=cap, seed=seed, gamma=0.0, fp64=fp64)
    with P.System(desc, x, v, inp.type, inp.state) as g:
        e = [g.observables()["ke_half"] + g.forces()[1]]
        for _ in range(steps // every):
            g.run(every)
            e.append(g.observables()["ke_half"] + g.forces()[1])
    return e


def oracle_energy(inp, x, v, cap, seed, steps, every):
    o = orc.System(x, v, inp.type, inp.state, cap=cap)
    md = orc.MDParams(L=(inp.L,) * 3, seed=seed, gamma=0.0)
    threads = 0 if orc.omp_lib() is not None else None
    e = [0.5 * (o.v ** 2).sum() + orc.forces(o, md, use_cells=True)[1]]
    for _ in range(steps // every):
        if threads is None:
            orc.run(o, md, None, every)
        else:
            orc.run_omp(o, md, None, every, threads)
        e.append(0.5 * (o.v ** 2).sum() + orc.forces(o, md, use_cells=True)[1])
    return e


def oracle_chain_ree(args):
    x, v, types, states, L, seed, steps = args
    o = orc.System(x, v, types, states, cap=2)
    md = orc.MDParams(L=(L,) * 3, seed=seed)
    rx = orc.Reaction(**synth.chain_growth_scheme(k=1.0))
    if orc.omp_lib() is not None:
        orc.run_omp(o, md, rx, steps, 4)
    else:
        orc.run(o, md, rx, steps)
    b = o.bonds()
    return chain_ree2(o.x, b[:, 1:3], o.type, o.state, L)


def test_chain_growth_33096_energy_and_end_to_end(P):
    from paper_1409_7498_gb300.warmup import warmed_liquid
    seed = synth.BASE_SEED + 900
    inp = synth.chain_growth(32768, 328, seed, placement="uniform")
    x, v = warmed_liquid(P, inp, 2, seed)
    e_o = oracle_energy(inp, x, v, 2, seed, 1000, 100)
    e_32 = gpu_energy(P, inp, x, v, 2, seed, False, 1000, 100)
    e_64 = gpu_energy(P, inp, x, v, 2, seed, True, 1000, 100)
    d = {"oracle": excursion(e_o), "gpu_fp32": excursion(e_32), "gpu_fp64": excursion(e_64)}
    print("chain_growth_33096 NVE relative energy excursion over 1,000 steps:", d)
    assert d["gpu_fp64"] <= 2.0 * d["oracle"] + 1e-6, d
    assert d["gpu_fp32"] <= 5.0 * d["oracle"] + 2e-5, d

    # end-to-end distance with reactions and the thermostat, four seeds a side
    starts = []
    for q in range(4):
        s = synth.BASE_SEED + 910 + q
        i2 = synth.chain_growth(32768, 328, s, placement="uniform")
        starts.append((i2, *warmed_liquid(P, i2, 2, s), s))
    with mp.get_context("spawn").Pool(4) as pool:
        pending = pool.map_async(oracle_chain_ree, [(x2, v2, i2.type, i2.state, i2.L, s, 1000)
                                                    for i2, x2, v2, s in starts])
        r_g = []
        for i2, x2, v2, s in starts:
            desc = P.make_desc(i2.n, i2.L, adj_cap=2, seed=s)
            with P.System(desc, x2, v2, i2.type, i2.state) as g:
                g.set_reaction(P.make_reaction(**synth.chain_growth_scheme(k=1.0)))
                g.run(1000)
                b = g.bonds()
                r_g += chain_ree2(g.positions(), np.stack([b["a"], b["t"]], 1), g.types(),
                                  g.states(), i2.L)
        r_o = [r for v in pending.get() for r in v]
    mg, mo = np.mean(r_g), np.mean(r_o)
    se = np.hypot(np.std(r_g, ddof=1) / np.sqrt(len(r_g)), np.std(r_o, ddof=1) / np.sqrt(len(r_o)))
    print(f"chain_growth_33096 <R_ee^2> after 1,000 steps: GPU {mg:.2f} ({len(r_g)} chains), "
          f"oracle {mo:.2f} ({len(r_o)} chains), combined SE {se:.2f}")
    assert abs(mg - mo) <= 3 * se, (mg, mo, se)
    assert len(r_g) > 500 and mg > 5.0


def test_step_growth_1m_energy_slice(P):
    from paper_1409_7498_gb300.warmup import warmed_liquid
    seed = synth.BASE_SEED + 950
    inp = synth.step_growth_sites(1_048_576, 4, seed, placement="uniform")
    x, v = warmed_liquid(P, inp, 4, seed)
    e_32 = gpu_energy(P, inp, x, v, 4, seed, False, 200, 100)
    e_o = oracle_energy(inp, x, v, 4, seed, 200, 100)
    d = {"oracle": excursion(e_o), "gpu_fp32": excursion(e_32)}
    print("step_growth_1m NVE relative energy excursion over 200 steps:", d)
    assert d["gpu_fp32"] <= 5.0 * d["oracle"] + 2e-5, d
    # the same start on both sides: the first energies agree to the force tolerance
    assert abs(e_32[0] - e_o[0]) / abs(e_o[0]) < 1e-5
