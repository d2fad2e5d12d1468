"""The E-P_n-E step-growth input (Sec. II.B) and the oracle on it (CPU).

The seeded generator must give what the section describes: chains whose
two end units E are the only targets, crosslinkers X of functionality f in
the stoichiometric ratio f n_X = 2 n_chains, chain bonds within the FENE
range, no overlapping beads; the oracle's reactions on it must keep the
section's rules (only X-E bonds, each E at most once, each X at most f
times, chain bonds kept).
"""
import numpy as np

import oracle as orc
import synth
from helpers import oracle_system, orc_reaction

F = 4


def test_generator_matches_the_section():
    inp, dims, cb = synth.ep_chains(400, 3, F, 5)
    ty, st = inp.type, inp.state
    assert (ty == synth.TYPE_E).sum() == 2 * 400 and (ty == synth.TYPE_P).sum() == 3 * 400
    assert F * (ty == synth.TYPE_A).sum() >= 2 * 400
    assert (st[ty == synth.TYPE_A] == F).all() and (st[ty != synth.TYPE_A] == 0).all()
    assert abs(inp.n / np.prod(dims) - synth.DENSITY) < 1e-9
    # every chain is E-P-P-P-E: four bonds, ends of type E
    assert len(cb) == 4 * 400
    deg = np.bincount(cb.ravel(), minlength=inp.n)
    assert (deg[ty == synth.TYPE_E] == 1).all() and (deg[ty == synth.TYPE_P] == 2).all()
    assert (deg[ty == synth.TYPE_A] == 0).all()
    d = inp.x[cb[:, 1]] - inp.x[cb[:, 0]]
    d -= np.array(dims) * np.round(d / np.array(dims))
    r = np.linalg.norm(d, axis=1)
    assert r.max() < 1.2 and r.min() > 0.9  # inside the FENE range (R0 = 1.5)
    # no two beads closer than 0.9 sigma (brute force over all pairs)
    x = inp.x
    for i0 in range(0, inp.n, 512):
        dd = x[i0:i0 + 512, None, :] - x[None, :, :]
        dd -= np.array(dims) * np.round(dd / np.array(dims))
        r2 = (dd ** 2).sum(-1)
        r2[np.arange(len(r2)), np.arange(i0, i0 + len(r2))] = np.inf
        assert r2.min() > 0.81


def test_oracle_reactions_keep_the_rules():
    inp, dims, cb = synth.ep_chains(400, 3, F, 6)
    bonds = np.zeros(len(cb), [("a", "<u4"), ("t", "<u4"), ("step", "<i8"), ("style", "<u4")])
    bonds["a"], bonds["t"] = cb[:, 0], cb[:, 1]
    o = oracle_system(inp.x, inp.v, inp.type, inp.state, F, bonds)
    sch = synth.ep_scheme(F, k=5.0)
    orc.run(o, orc.MDParams(L=dims, seed=6), orc_reaction(sch), 200)
    b = o.bonds()  # (step, a, t, style)
    new = b[b[:, 0] > 0]
    assert len(b) - len(new) == len(cb) and len(new) > 20
    ty, st = inp.type, o.state
    assert (ty[new[:, 1]] == synth.TYPE_A).all() and (ty[new[:, 2]] == synth.TYPE_E).all()
    e_deg = np.bincount(new[:, 2], minlength=inp.n)
    x_deg = np.bincount(new[:, 1], minlength=inp.n)
    assert e_deg.max() <= 1 and (e_deg == np.where(ty == synth.TYPE_E, st, 0)).all()
    assert (x_deg[ty == synth.TYPE_A] == F - st[ty == synth.TYPE_A]).all()
    assert len(np.unique(new[:, 1] * inp.n + new[:, 2])) == len(new)
