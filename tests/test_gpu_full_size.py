"""The 1M-bead step-growth workload the bench times (f = 4, k = 0.1,
Theta = 10, skin 0.4, 32-bit lists, the same kernels and launch shapes), on
the GPU against the oracle.

Both sides start from the same seeded synthetic input (plus, for the
reaction test, bonds the oracle made); nothing flows from the GPU to the
oracle.  Checked at full size:
  * FP32 forces on every bead within 1e-5 of the oracle's FP64 forces;
  * one reaction step bit-exact (bonds, states, Table I counts);
  * a run of reaction cycles in the bench's CUDA-graph path keeps the
    bookkeeping invariants that hold at any size.
"""
import numpy as np
import pytest

import oracle as orc
import synth
from helpers import (bonds_of_oracle, canonical, force_errors, gpu, md_params, oracle_system,
                     orc_reaction)

pytestmark = pytest.mark.gpu

N = 1_048_576
F = 4
SKIN = 0.4


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return gpu()


@pytest.fixture(scope="module")
def workload():
    inp = synth.step_growth_sites(N, F, synth.BASE_SEED)
    return inp, synth.step_growth_scheme(F, k=0.1, theta=10)


def gpu_of(P, inp, x, v, types, states, bonds=None):
    desc = P.make_desc(inp.n, inp.L, adj_cap=F, seed=synth.BASE_SEED, skin=SKIN)
    return P.System(desc, x, v, types, states, bonds=bonds)


def test_forces_at_full_size(P, workload):
    inp, _ = workload
    o = oracle_system(inp.x, inp.v, inp.type, inp.state, F)
    f_ref, e_ref = orc.forces(o, md_params(inp.L, synth.BASE_SEED), use_cells=True)
    with gpu_of(P, inp, inp.x, inp.v, inp.type, inp.state) as g:
        f, e = g.forces()
    err = force_errors(f, f_ref)
    assert err["max_over_rms"] < 1e-5, err
    assert err["rms_rel"] < 1e-5, err
    assert e == pytest.approx(e_ref, rel=1e-5)


def test_reaction_steps_bit_exact_at_full_size(P, workload):
    inp, sch = workload
    o = oracle_system(inp.x, inp.v, inp.type, inp.state, F)
    md = md_params(inp.L, synth.BASE_SEED)
    # bonds made by the oracle first (k = 2: a few percent conversion)
    orc.react(o, md, orc_reaction(dict(sch, k=2.0)), step=1000, use_cells=True)
    with gpu_of(P, inp, o.x, o.v, o.type, o.state, bonds=bonds_of_oracle(o)) as g:
        g.set_reaction(P.make_reaction(**sch))
        for step in (1010, 1020):
            tr_o = orc.react(o, md, orc_reaction(sch), step=step, use_cells=True)
            tr_g = g.react_once(step)
            assert tr_g == tr_o, (step, tr_g, tr_o)
            assert (g.states() == o.state).all()
            assert np.array_equal(canonical(g.bonds()), canonical(bonds_of_oracle(o)))
    assert tr_o["formed"] > 1000


def test_graph_run_invariants_at_full_size(P, workload):
    """Ten reaction cycles in the bench's path (CUDA graphs, rebuilds by the
    displacement trigger): step growth keeps, at any size, f - state bonds
    per crosslinker, state = bonds per target (at most two), bonds only
    between a crosslinker and a target, each pair once, and at most one new
    bond per bead per reaction step; the observables agree with the states."""
    inp, sch = workload
    with gpu_of(P, inp, inp.x, inp.v, inp.type, inp.state) as g:
        g.set_reaction(P.make_reaction(**sch))
        g.run(100)
        ob = g.observables()
        st = g.states()
        b = canonical(g.bonds())
        x = g.positions()
        stats = g.stats()
    assert stats["steps"] == 100 and stats["reactions"] == 10 and stats["rebins"] >= 5
    assert np.isfinite(x).all()
    ty = inp.type
    A = ty == synth.TYPE_A
    assert len(b) > 1000 and ob["bonds"] == len(b)
    a, t = b[:, 1], b[:, 2]
    assert (ty[a] == synth.TYPE_A).all() and (ty[t] != synth.TYPE_A).all()
    assert len(np.unique(a * N + t)) == len(b)
    deg = np.bincount(np.concatenate([a, t]), minlength=N)
    assert (deg[A] == F - st[A]).all()
    assert (deg[~A] == st[~A]).all() and deg[~A].max() <= 2
    for s in np.unique(b[:, 0]):
        ends = b[b[:, 0] == s][:, 1:3].ravel()
        assert len(ends) == len(np.unique(ends))
    counts = np.zeros((8, 16), np.int64)
    np.add.at(counts, (ty, st), 1)
    assert (ob["counts"] == counts).all()
