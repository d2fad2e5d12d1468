"""Concurrent reactions on the GPU against the oracle (orc_react_set), the
extension of Secs. III.B and VII.  The reaction step is integer and
FP64-decision work, so bonds (with the reaction that formed each), states
and Table I counts must be identical; the FP64 trajectory must follow the
oracle's to round-off (1e-9 in positions) with identical bonds."""
import numpy as np
import pytest

import oracle as orc
import synth
from helpers import canonical, gpu, gpu_system, md_params, oracle_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return gpu()


def schemes(k=(4.0, 1.0, 2.0)):
    return synth.concurrent_schemes(*k)


def with_reactions(bonds):
    """(step, a, t, reaction) rows in canonical order."""
    if len(bonds) == 0:
        return np.zeros((0, 4), np.int64)
    b = np.stack([bonds["step"].astype(np.int64), bonds["a"].astype(np.int64),
                  bonds["t"].astype(np.int64), bonds["reaction"].astype(np.int64)], axis=1)
    return b[np.lexsort((b[:, 2], b[:, 1], b[:, 0]))]


def min_image_diff(a, b, L):
    d = a - b
    return np.abs(d - L * np.round(d / L)).max()


@pytest.mark.parametrize("n_B,n_A,n_X6", [(1600, 200, 100), (30000, 2500, 1200)])
def test_reaction_steps_bit_exact(P, n_B, n_A, n_X6):
    seed = 31
    inp = synth.step_growth_mixed(n_B, n_A, n_X6, seed, jitter=0.5)
    sch = schemes()
    o = oracle_system(inp.x, inp.v, inp.type, inp.state, 6)
    md = md_params(inp.L, seed)
    with gpu_system(P, inp.L, inp.x, inp.v, inp.type, inp.state, cap=6, seed=seed) as g:
        g.set_reactions([P.make_reaction(**s) for s in sch])
        for step in (10, 20, 30, 40):
            tr = g.react_once(step)
            tr_o, per = orc.react_set(o, md, [orc.Reaction(**s) for s in sch], step,
                                      use_cells=True)
            assert tr == tr_o
        gb = with_reactions(g.bonds())
        assert np.array_equal(gb, o.bond_reactions())
        assert np.array_equal(g.states(), o.state)
        counts = np.bincount(gb[:, 3], minlength=3)
        assert (counts > 10).all(), counts  # every reaction formed bonds


def test_fp64_trajectory_with_concurrent_reactions(P):
    seed = 7
    inp = synth.step_growth_mixed(1000, 160, 80, seed)
    sch = schemes((2.0, 0.5, 1.0))
    rxo = [orc.Reaction(**s) for s in sch]
    o = oracle_system(inp.x, inp.v, inp.type, inp.state, 6)
    md = md_params(inp.L, seed)
    with gpu_system(P, inp.L, inp.x, inp.v, inp.type, inp.state, cap=6, fp64=True,
                    seed=seed) as g:
        g.set_reactions([P.make_reaction(**s) for s in sch])
        for chunk in range(3):
            orc.run_set(o, md, rxo, 100)
            g.run(100)
            assert g.step() == o.step
            assert min_image_diff(g.positions(), o.x, inp.L) < 1e-9
            assert np.array_equal(with_reactions(g.bonds()), o.bond_reactions())
            assert np.array_equal(g.states(), o.state)
        assert o.nb > 50


def test_fp32_graph_run_invariants_and_checkpoint(P, tmp_path):
    """FP32 mode in the CUDA graph: one new bond per particle per step, each
    crosslinker's first bond from reaction 0 and later ones from reaction 1,
    X6 bonds from reaction 2, states = functionality - bonds; a checkpoint
    with the three reactions continues bit for bit; a batch member with
    them matches its run alone."""
    seed = 17
    inp = synth.step_growth_mixed(8000, 800, 400, seed)
    sch = schemes((1.0, 0.3, 0.6))
    rxs = [P.make_reaction(**s) for s in sch]
    path = str(tmp_path / "multi.ckpt")
    with gpu_system(P, inp.L, inp.x, inp.v, inp.type, inp.state, cap=6, seed=seed) as g:
        g.set_reactions(rxs)
        g.run(300)
        g.save(path)
        g.run(200)
        b = with_reactions(g.bonds())
        st = g.states()
        pos = g.positions()
        # the reaction records' populations, kept by the reaction kernel one
        # bond at a time, equal a full count of the states
        last = g.history()[-1]
        ty = g.types()
        for t in (synth.TYPE_B, synth.TYPE_A, synth.TYPE_X6):
            assert np.array_equal(np.bincount(st[ty == t], minlength=16)[:16], last["counts"][t])
        assert last["bonds"] == len(b)
    ends = b[:, 1:3]
    for s_ in np.unique(b[:, 0]):
        e = ends[b[:, 0] == s_].ravel()
        assert len(np.unique(e)) == len(e)
    deg = np.bincount(ends.ravel(), minlength=inp.n)
    A = inp.type == synth.TYPE_A
    X6 = inp.type == synth.TYPE_X6
    assert np.array_equal(st[A], 4 - deg[A]) and np.array_equal(st[X6], 6 - deg[X6])
    for a in np.flatnonzero(A)[:300]:
        rows = b[b[:, 1] == a]
        if len(rows):
            assert rows[0, 3] == 0 and (rows[1:, 3] == 1).all()
    assert set(b[np.isin(b[:, 1], np.flatnonzero(X6)), 3].tolist()) == {2}
    g2 = P.System.load(path)
    with g2:
        g2.run(200)
        assert np.array_equal(with_reactions(g2.bonds()), b)
        assert np.array_equal(g2.positions(), pos)
    # batch member against its run alone
    with gpu_system(P, inp.L, inp.x, inp.v, inp.type, inp.state, cap=6, seed=seed) as a, \
            gpu_system(P, inp.L, inp.x, inp.v, inp.type, inp.state, cap=6, seed=seed) as m:
        a.set_reactions(rxs)
        m.set_reactions(rxs)
        a.run(200)
        with P.Batch() as bt:
            bt.add(m)
            bt.run(200)
            bt.sync()
            bt.remove(m)
        assert np.array_equal(with_reactions(a.bonds()), with_reactions(m.bonds()))
        assert np.array_equal(a.positions(), m.positions())


def test_invalid_sets_are_rejected(P):
    inp = synth.step_growth(500, 100, 4, 3)
    sch = schemes()
    with gpu_system(P, inp.L, inp.x, inp.v, inp.type, inp.state, cap=6) as g:
        bad = dict(sch[0], mask_A=1 << synth.TYPE_B, a_lo=0, a_hi=1, mask_T=1 << synth.TYPE_A,
                   t_lo=1, t_hi=4)
        with pytest.raises(P.PolyrxError):
            g.set_reactions([P.make_reaction(**sch[0]), P.make_reaction(**bad)])
        with pytest.raises(P.PolyrxError):
            g.set_reactions([P.make_reaction(**sch[0]), P.make_reaction(**dict(sch[1], theta=5))])
        with pytest.raises(P.PolyrxError):
            g.set_reactions([P.make_reaction(**sch[0])] * 5)
        g.set_reactions([P.make_reaction(**s) for s in sch])
        g.set_reactions([])  # clears
