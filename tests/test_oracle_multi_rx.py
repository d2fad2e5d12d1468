"""Pins of the oracle's concurrent reactions (orc_react_set), the extension
the paper names in Secs. III.B and VII without giving its algorithm.

What fixes it independently of its own code:
  * one reaction is the single-reaction step of Table I, bit for bit (the
    pinned orc_react and orc_run);
  * hand-built frozen systems whose outcome is forced (p = 1, isolated pairs,
    per-reaction cutoffs) and whose bonds carry each reaction's increments,
    style and valence limit;
  * the shared acceptance draw: a pair eligible for reactions with p_0 and
    p_1 takes reaction 0, reaction 1 or none with probabilities p_0, p_1,
    1 - p_0 - p_1 (chi-square over keyed draws); isolated pairs of each
    reaction bond after m reaction steps with probability 1 - (1 - p_r)^m;
  * a T that two A's of different reactions both retain takes each with
    probability 1/2 (one A per T, Table I step 7);
  * invariants of runs with three reactions: at most one new bond per
    particle per step, valence limits, state windows, no duplicate bonds,
    state = initial state + the increments of the reactions of its bonds.
"""
import numpy as np
import pytest

import oracle as orc
import synth

TYPE_B, TYPE_A = synth.TYPE_B, synth.TYPE_A
TYPE_A2 = 2  # a second crosslinker type


def rx(mask_A, mask_T, a_lo, a_hi, t_lo, t_hi, dA, dT, k, r_react=1.1, style=0, mv=None,
       theta=10):
    return orc.Reaction(mask_A=mask_A, mask_T=mask_T, a_lo=a_lo, a_hi=a_hi, t_lo=t_lo, t_hi=t_hi,
                        dA=dA, dT=dT, k=k, theta=theta, r_react=r_react, bond_style=style,
                        max_valence=mv or (8,) * 8)


def k_of(p, dt=0.005, theta=10):
    """The rate k whose acceptance probability k dt Theta is p."""
    return p / (dt * theta)


def tiny(pos, types, states, L=30.0, cap=8, seed=1):
    pos = np.asarray(pos, float)
    s = orc.System(pos, np.zeros_like(pos), np.asarray(types, np.uint8),
                   np.asarray(states, np.int8), cap=cap)
    return s, orc.MDParams(L=(L,) * 3, seed=seed)


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("k", [0.1, 2.0, 40.0])
@pytest.mark.parametrize("seed", [3, 4])
def test_one_reaction_is_the_single_reaction_step(k, seed):
    inp = synth.step_growth(1000, 250, 4, seed, jitter=0.5)
    r = orc.Reaction(**synth.step_growth_scheme(4, k=k))
    md = orc.MDParams(L=(inp.L,) * 3, seed=seed)
    a = orc.System(inp.x, inp.v, inp.type, inp.state, cap=4)
    b = orc.System(inp.x, inp.v, inp.type, inp.state, cap=4)
    for step in (10, 20, 30):
        tr_a = orc.react(a, md, r, step, use_cells=True)
        tr_b, per = orc.react_set(b, md, [r], step, use_cells=True)
        assert tr_a == tr_b and per == [tr_a["formed"]]
    assert np.array_equal(a.bonds(), b.bonds()) and np.array_equal(a.state, b.state)
    assert np.array_equal(a.nadj, b.nadj) and np.array_equal(a.adj, b.adj)


def test_one_reaction_run_is_the_single_reaction_run():
    inp = synth.chain_growth(900, 30, 5)
    r = orc.Reaction(**synth.chain_growth_scheme(k=5.0))
    md = orc.MDParams(L=(inp.L,) * 3, seed=5)
    a = orc.System(inp.x, inp.v, inp.type, inp.state, cap=2)
    b = orc.System(inp.x, inp.v, inp.type, inp.state, cap=2)
    orc.run(a, md, r, 60)
    orc.run_set(b, md, [r], 60)
    assert a.nb > 20
    assert np.array_equal(a.x, b.x) and np.array_equal(a.v, b.v)
    assert np.array_equal(a.bonds(), b.bonds()) and np.array_equal(a.state, b.state)


def test_invalid_sets_are_rejected():
    r0 = rx(1 << TYPE_A, 1 << TYPE_B, 1, 4, 0, 1, -1, 1, 0.1)
    assert orc.check_reactions([r0]) == orc.OK
    assert orc.check_reactions([r0] * 4) == orc.OK
    assert orc.check_reactions([r0] * 5) == orc.EINVAL
    # a (type, state) that is an A of one reaction and a T of another
    r_bad = rx(1 << TYPE_B, 1 << TYPE_A, 0, 1, 1, 4, 1, -1, 0.1)
    assert orc.check_reactions([r0, r_bad]) == orc.EINVAL
    # ... but disjoint states of the same type are fine
    r_ok = rx(1 << TYPE_B, 1 << TYPE_A2, 2, 2, 0, 0, -1, 1, 0.1)
    assert orc.check_reactions([r0, r_ok]) == orc.OK
    # another Theta, or the nearest rule with several reactions
    assert orc.check_reactions([r0, rx(1 << TYPE_A2, 1 << TYPE_B, 1, 6, 0, 1, -1, 1, 0.1,
                                       theta=5)]) == orc.EINVAL
    near = orc.Reaction(**synth.step_growth_scheme(4, k=0.1, selection=orc.SELECT_NEAREST))
    assert orc.check_reactions([near]) == orc.OK
    assert orc.check_reactions([near, r_ok]) == orc.EINVAL


def test_two_isolated_pairs_bond_with_their_own_reaction():
    """Crosslinker A (type 1) next to a B and crosslinker A2 (type 2) next to
    another B, far apart; both reactions certain.  Each bond takes its own
    reaction's increments and style."""
    pos = [[5, 5, 5], [6, 5, 5], [20, 20, 20], [21, 20, 20]]
    s, md = tiny(pos, [TYPE_A, TYPE_B, TYPE_A2, TYPE_B], [4, 0, 6, 0])
    r0 = rx(1 << TYPE_A, 1 << TYPE_B, 1, 4, 0, 1, -1, +1, k_of(1.0), style=0)
    r1 = rx(1 << TYPE_A2, 1 << TYPE_B, 1, 6, 0, 1, -2, +3, k_of(1.0), style=1)
    tr, per = orc.react_set(s, md, [r0, r1], step=10)
    assert tr == dict(candidates=2, retained=2, a_winners=2, formed=2) and per == [1, 1]
    assert s.bond_reactions()[:, 1:].tolist() == [[0, 1, 0], [2, 3, 1]]
    assert s.bonds()[:, 3].tolist() == [0, 1]  # styles
    assert s.state.tolist() == [3, 1, 4, 3]
    assert s.adj_style[0, 0] == 0 and s.adj_style[2, 0] == 1


def test_each_reaction_has_its_own_cutoff():
    """A pair at r = 1.1 is inside reaction 1's cutoff (1.2) and outside
    reaction 0's (1.0): only reaction 1 can bond it."""
    pos = [[5, 5, 5], [6.1, 5, 5]]
    for p1, expect in ((1.0, [[0, 1, 1]]), (0.0, [])):
        s, md = tiny(pos, [TYPE_A, TYPE_B], [4, 0])
        r0 = rx(1 << TYPE_A, 1 << TYPE_B, 1, 4, 0, 1, -1, 1, k_of(1.0), r_react=1.0)
        r1 = rx(1 << TYPE_A, 1 << TYPE_B, 1, 4, 0, 1, -1, 1, k_of(p1), r_react=1.2)
        orc.react_set(s, md, [r0, r1], step=10)
        assert s.bond_reactions()[:, 1:].tolist() == expect


def test_each_reaction_has_its_own_valence_limit():
    """Reaction 0 allows the crosslinker one bond, reaction 1 four: with
    the crosslinker already holding one bond, a pair taken by reaction 0 is
    refused (capacity) and one taken by reaction 1 forms."""
    pos = [[5, 5, 5], [6, 5, 5], [4, 5, 5]]
    mv0 = [8] * 8
    mv0[TYPE_A] = 1
    for p0, p1, formed in ((1.0, 0.0, False), (0.0, 1.0, True)):
        s, md = tiny(pos, [TYPE_A, TYPE_B, TYPE_B], [3, 0, 1])
        s.add_bond(0, 2)
        r0 = rx(1 << TYPE_A, 1 << TYPE_B, 1, 4, 0, 0, -1, 1, k_of(p0), mv=mv0)
        r1 = rx(1 << TYPE_A, 1 << TYPE_B, 1, 4, 0, 0, -1, 1, k_of(p1))
        if formed:
            orc.react_set(s, md, [r0, r1], step=10)
            assert s.nb == 2 and s.state[0] == 2
        else:
            with pytest.raises(orc.OracleError) as e:
                orc.react_set(s, md, [r0, r1], step=10)
            assert e.value.code == orc.ECAPACITY and s.nb == 1 and s.state[0] == 3


def _chi2(counts, probs):
    counts = np.asarray(counts, float)
    exp = counts.sum() * np.asarray(probs)
    return float(((counts - exp) ** 2 / exp).sum())


def test_shared_draw_splits_a_pair_between_reactions():
    """One A and one T eligible for both reactions: reaction 0 with p_0,
    reaction 1 with p_1, none with 1 - p_0 - p_1 (chi-square, 2 degrees of
    freedom, 99.9% quantile 13.8)."""
    p0, p1 = 0.2, 0.3
    counts = [0, 0, 0]
    for trial in range(4000):
        s, md = tiny([[5, 5, 5], [6, 5, 5]], [TYPE_A, TYPE_B], [4, 0], seed=1000 + trial)
        r0 = rx(1 << TYPE_A, 1 << TYPE_B, 1, 4, 0, 1, -1, 1, k_of(p0))
        r1 = rx(1 << TYPE_A, 1 << TYPE_B, 1, 4, 0, 1, -1, 1, k_of(p1))
        _, per = orc.react_set(s, md, [r0, r1], step=10)
        counts[0 if per[0] else (1 if per[1] else 2)] += 1
    assert _chi2(counts, [p0, p1, 1 - p0 - p1]) < 13.8, counts


def test_per_reaction_binomial_rate():
    """Isolated pairs of two reactions (different crosslinker types) with
    p_0 = 0.05 and p_1 = 0.2: after m reaction steps, the fraction of bonded
    pairs of reaction r is 1 - (1 - p_r)^m (within 4 standard errors)."""
    npairs, m = 400, 5
    p = (0.05, 0.2)
    pos, types, states = [], [], []
    g = 10  # pairs on a 10 x 10 x 10 grid of spacing 4 (1,000 sites)
    for q in range(2 * npairs):
        x, y, z = (q % g) * 4.0 + 1, ((q // g) % g) * 4.0 + 1, (q // (g * g)) * 4.0 + 1
        pos += [[x, y, z], [x + 1.0, y, z]]
        types += [TYPE_A if q < npairs else TYPE_A2, TYPE_B]
        states += [4, 0]
    L = 4.0 * g
    assert 2 * npairs <= g ** 3
    s, md = tiny(pos, types, states, L=L, seed=99)
    r0 = rx(1 << TYPE_A, 1 << TYPE_B, 1, 4, 0, 0, -1, 1, k_of(p[0]))
    r1 = rx(1 << TYPE_A2, 1 << TYPE_B, 1, 4, 0, 0, -1, 1, k_of(p[1]))
    for step in range(10, 10 * (m + 1), 10):
        orc.react_set(s, md, [r0, r1], step=step, use_cells=True)
    br = s.bond_reactions()
    for r in (0, 1):
        got = (br[:, 3] == r).sum() / npairs
        want = 1 - (1 - p[r]) ** m
        se = np.sqrt(want * (1 - want) / npairs)
        assert abs(got - want) < 4 * se, (r, got, want)


def test_a_t_that_two_reactions_retain_takes_one_a_at_random():
    """A T with an A of reaction 0 on one side and an A of reaction 1 on the
    other, both certain: exactly one bond forms, each A winning about half
    the time (Table I step 7; chi-square, 1 degree of freedom)."""
    wins = [0, 0]
    for trial in range(2000):
        s, md = tiny([[4, 5, 5], [5, 5, 5], [6, 5, 5]], [TYPE_A, TYPE_B, TYPE_A2], [4, 0, 6],
                     seed=5000 + trial)
        r0 = rx(1 << TYPE_A, 1 << TYPE_B, 1, 4, 0, 1, -1, 1, k_of(1.0))
        r1 = rx(1 << TYPE_A2, 1 << TYPE_B, 1, 6, 0, 1, -1, 1, k_of(1.0))
        tr, per = orc.react_set(s, md, [r0, r1], step=10)
        assert tr["formed"] == 1 and sum(per) == 1 and s.nb == 1
        wins[0 if per[0] else 1] += 1
    assert _chi2(wins, [0.5, 0.5]) < 10.8, wins


def test_invariants_of_a_three_reaction_run():
    """Step growth with a substitution effect (a crosslinker's first bond at
    k_1, later ones at k_2) and a second crosslinker type of functionality 6
    at k_3, all on the same difunctional B's."""
    rng = np.random.default_rng(21)
    inp = synth.step_growth(1600, 300, 4, 21, jitter=0.5)
    types = inp.type.copy()
    states = inp.state.copy()
    a_ids = np.flatnonzero(types == TYPE_A)
    x6 = rng.permutation(a_ids)[: len(a_ids) // 3]
    types[x6] = TYPE_A2
    states[x6] = 6
    mv = [0] * 8
    mv[TYPE_B], mv[TYPE_A], mv[TYPE_A2] = 2, 4, 6
    rs = [rx(1 << TYPE_A, 1 << TYPE_B, 4, 4, 0, 1, -1, 1, 4.0, mv=tuple(mv)),
          rx(1 << TYPE_A, 1 << TYPE_B, 1, 3, 0, 1, -1, 1, 1.0, mv=tuple(mv)),
          rx(1 << TYPE_A2, 1 << TYPE_B, 1, 6, 0, 1, -1, 1, 2.0, r_react=1.05, mv=tuple(mv))]
    s = orc.System(inp.x, inp.v, types, states, cap=6)
    md = orc.MDParams(L=(inp.L,) * 3, seed=21)
    assert orc.check_reactions(rs) == orc.OK
    counts = np.zeros(3, int)
    for step in range(10, 410, 10):
        nb0 = s.nb
        _, per = orc.react_set(s, md, rs, step=step, use_cells=True)
        counts += per
        new = s.bond_reactions()
        new = new[new[:, 0] == step]
        ends = np.concatenate([new[:, 1], new[:, 2]])
        assert len(np.unique(ends)) == len(ends)  # one new bond per particle per step
        assert s.nb - nb0 == len(new) == sum(per)
    assert (counts > 20).all()
    br = s.bond_reactions()
    pairs = {(int(a), int(t)) for _, a, t, _ in br}
    assert len(pairs) == len(br)  # no duplicate bonds
    # crosslinkers: state = functionality - bonds; B: state = bonds <= 2
    deg = np.bincount(np.concatenate([br[:, 1], br[:, 2]]), minlength=s.n)
    assert np.array_equal(s.state[types == TYPE_A], 4 - deg[types == TYPE_A])
    assert np.array_equal(s.state[types == TYPE_A2], 6 - deg[types == TYPE_A2])
    assert np.array_equal(s.state[types == TYPE_B], deg[types == TYPE_B])
    assert deg[types == TYPE_B].max() <= 2
    # a crosslinker's first bond comes from reaction 0, its later ones from reaction 1
    for a in np.flatnonzero(types == TYPE_A):
        rows = br[br[:, 1] == a]
        if len(rows):
            assert rows[0, 3] == 0 and (rows[1:, 3] == 1).all()
    assert set(br[np.isin(br[:, 1], x6), 3].tolist()) <= {2}
