"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each checks it against a
published known answer, a closed form worked by hand, a conservation law,
an exact discrete-time property of the integrator, a combinatorial property
of the reaction rule, or an independent enumeration.
"""
import math
import os

import numpy as np
import pytest

import oracle as orc
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def two_particles(r, L=10.0):
    x = np.array([[2.0, 3.0, 4.0], [2.0 + r, 3.0, 4.0]])
    return orc.System(x, np.zeros((2, 3)), np.zeros(2, np.uint8), np.zeros(2, np.int8), cap=4)


# --------------------------------------------------------------------------
# Philox4x32-10
# --------------------------------------------------------------------------
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        assert orc.philox4x32_10(v[0:4], v[4:6]) == v[6:10]


def test_uniform_conversions_exact():
    assert orc.u53(0, 0) == 0.0
    assert orc.u53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert orc.u53(0x80000000, 0) == 0.5
    assert orc.u24(0) == 0.0
    assert orc.u24(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert orc.u24(0x80000000) == 0.5
    # the low 11 (resp. 8) bits do not matter
    assert orc.u53(0x12345678, 0x9ABCDEF0) == orc.u53(0x12345678, 0x9ABCD800)
    assert orc.u24(0x123456FF) == orc.u24(0x12345600)


def test_philox_uniform_statistics():
    # chi-square of 64 bins over 2^16 draws of u53 keyed like the acceptance draw
    n, nb = 1 << 16, 64
    u = np.empty(n)
    for i in range(n):
        w = orc.philox4x32_10([i & 0xFFFFFFFF, 7, 11, 2], [123, 456])
        u[i] = orc.u53(w[0], w[1])
    h, _ = np.histogram(u, bins=nb, range=(0, 1))
    chi2 = ((h - n / nb) ** 2 / (n / nb)).sum()
    assert chi2 < 120  # 63 dof: P(chi2 > 120) ~ 2e-5
    # lag-1 serial correlation
    c = np.corrcoef(u[:-1], u[1:])[0, 1]
    assert abs(c) < 5.0 / math.sqrt(n)


# --------------------------------------------------------------------------
# Potentials: closed forms worked by hand, energy/force consistency
# --------------------------------------------------------------------------
def golden_potentials():
    rows = []
    for l in open(os.path.join(GOLDEN, "potentials.txt")):
        if l.strip() and not l.startswith("#"):
            name, r, V, F = l.split()
            rows.append((name, float(r), float(V), float(F)))
    return rows


@pytest.mark.parametrize("row", golden_potentials(), ids=lambda r: f"{r[0]}@{r[1]}")
def test_potential_closed_forms(row):
    name, r, V, F = row
    s = two_particles(r)
    md = orc.MDParams(L=(10.0, 10.0, 10.0))
    if name == "fene":
        md.eps = 0.0  # isolate the bond
        s.add_bond(0, 1, orc.BOND_FENE)
    elif name == "mirror_lj":
        s.add_bond(0, 1, orc.BOND_MIRROR_LJ)
    f, e = orc.forces(s, md)
    # particle 1 sits at +r along x: a repulsive force pushes it to +x
    assert e == pytest.approx(V, abs=1e-12, rel=1e-12)
    assert f[1, 0] == pytest.approx(F, abs=1e-10, rel=1e-12)
    assert f[0, 0] == -f[1, 0]
    assert f[0, 1] == f[0, 2] == 0.0


@pytest.mark.parametrize("style,eps,rs", [
    (None, 1.0, [0.85, 0.95, 1.05, 1.12]),
    (orc.BOND_FENE, 0.0, [0.6, 0.9, 1.2, 1.45]),
    (orc.BOND_MIRROR_LJ, 0.0, [1.13, 1.2, 1.3, 1.5, 1.7]),
])
def test_force_is_minus_energy_gradient(style, eps, rs):
    md = orc.MDParams(L=(10.0, 10.0, 10.0), eps=eps)
    h = 1e-6
    for r in rs:
        def energy(rr):
            s = two_particles(rr)
            if style is not None:
                s.add_bond(0, 1, style)
            return orc.forces(s, md)[1]
        s = two_particles(r)
        if style is not None:
            s.add_bond(0, 1, style)
        f, _ = orc.forces(s, md)
        fd = -(energy(r + h) - energy(r - h)) / (2 * h)
        assert f[1, 0] == pytest.approx(fd, rel=1e-6, abs=1e-6)


def test_fene_overstretch_is_an_error():
    s = two_particles(1.5)
    s.add_bond(0, 1)
    with pytest.raises(orc.OracleError) as e:
        orc.forces(s, orc.MDParams(L=(10.0,) * 3))
    assert e.value.code == orc.EOVERSTRETCH


def test_minimum_image_across_the_boundary():
    L = 5.0
    x = np.array([[0.1, 2.0, 2.0], [L - 0.9, 2.0, 2.0]])  # 1.0 apart through the face
    s = orc.System(x, np.zeros((2, 3)), np.zeros(2, np.uint8), np.zeros(2, np.int8))
    f, e = orc.forces(s, orc.MDParams(L=(L,) * 3))
    assert e == pytest.approx(1.0, rel=1e-12)
    assert f[0, 0] == pytest.approx(24.0, rel=1e-12)  # pushed to +x, away from its image


def test_force_cap():
    s = two_particles(0.7)
    md = orc.MDParams(L=(10.0,) * 3, force_cap=50.0)
    f, _ = orc.forces(s, md)
    assert f[1, 0] == pytest.approx(50.0, rel=1e-14)


def test_newton_third_law_and_cells_match_all_pairs():
    inp = synth.step_growth(700, 100, 4, seed=5, jitter=0.4)
    s = orc.System(inp.x, inp.v, inp.type, inp.state, cap=4)
    rng = np.random.default_rng(1)
    # some FENE bonds between close pairs
    f0, _ = orc.forces(s, orc.MDParams(L=(inp.L,) * 3))
    pairs = 0
    for i in rng.permutation(inp.n)[:200]:
        d = inp.x - inp.x[i]
        d -= inp.L * np.round(d / inp.L)
        r = np.sqrt((d ** 2).sum(1))
        r[i] = 9
        j = int(np.argmin(r))
        if r[j] < 1.3 and s.nadj[i] < 4 and s.nadj[j] < 4 and j not in s.adj[i, :s.nadj[i]]:
            s.add_bond(int(i), j)
            pairs += 1
    assert pairs > 50
    md = orc.MDParams(L=(inp.L,) * 3)
    fb, eb = orc.forces(s, md, use_cells=False)
    fc, ec = orc.forces(s, md, use_cells=True)
    scale = np.sqrt((fb ** 2).sum(1).mean())
    assert np.abs(fb - fc).max() < 1e-12 * scale
    assert ec == pytest.approx(eb, rel=1e-12)
    assert np.abs(fb.sum(0)).max() < 1e-10 * scale * math.sqrt(inp.n)


# --------------------------------------------------------------------------
# Integrator
# --------------------------------------------------------------------------
def test_nve_conserves_momentum_and_energy():
    inp = synth.step_growth(400, 100, 4, seed=3)
    s = orc.System(inp.x, inp.v, inp.type, inp.state, cap=4)
    md = orc.MDParams(L=(inp.L,) * 3, gamma=0.0, dt=0.005)
    p0 = s.v.sum(0)
    energies = []
    for it in range(1500):
        # the full-step velocity (v + v')/2 of a step belongs to the positions
        # the step starts from, so pair it with the potential there
        _, pe = orc.forces(s, md) if it >= 500 else (None, 0.0)
        ke = orc.step(s, md)
        if it >= 500:  # after the lattice has melted
            energies.append(ke + pe)
    assert np.abs(s.v.sum(0) - p0).max() < 1e-10
    e = np.array(energies) / inp.n
    slope = np.polyfit(np.arange(len(e)), e, 1)[0] * len(e)
    assert abs(slope) < 1e-3
    assert e.std() < 1e-3


def test_langevin_free_particle_discrete_stationary_law():
    """Without conservative forces the kick-drift Langevin step is the AR(1)
    process v' = (1 - g dt) v + (dt/m) R with Var R = 2 g kT m / dt, whose
    stationary variance is (kT/m) 2/(2 - g dt); the full-step velocity
    (v + v')/2 has variance exactly kT/m; the lag-k autocorrelation of the
    stored velocity is (1 - g dt)^k."""
    n = 3000
    gamma, dt = 10.0, 0.005
    rng = np.random.default_rng(9)
    x = rng.random((n, 3)) * 20.0
    s = orc.System(x, np.zeros((n, 3)), np.zeros(n, np.uint8), np.zeros(n, np.int8), cap=1)
    md = orc.MDParams(L=(20.0,) * 3, gamma=gamma, dt=dt, eps=0.0, seed=77)
    for _ in range(200):
        orc.step(s, md)
    v2h, kef, lag = [], [], []
    for it in range(1200):
        prev = s.v.copy()
        ke = orc.step(s, md)
        v2h.append((s.v ** 2).mean())
        kef.append(2 * ke / (3 * n))
        lag.append((prev * s.v).mean())
    a = 1 - gamma * dt
    var_h = 2.0 / (2.0 - gamma * dt)
    assert np.mean(v2h) == pytest.approx(var_h, rel=4e-3)
    assert np.mean(kef) == pytest.approx(1.0, rel=4e-3)
    assert np.mean(lag) / np.mean(v2h) == pytest.approx(a, abs=3e-3)


# --------------------------------------------------------------------------
# Reaction rule (Table I)
# --------------------------------------------------------------------------
def rx_of(d):
    return orc.Reaction(**d)


def make(x, types, states, L=10.0, cap=8):
    x = np.asarray(x, np.float64)
    n = len(x)
    return orc.System(x, np.zeros((n, 3)), np.asarray(types, np.uint8),
                      np.asarray(states, np.int8), cap=cap)


def md_for(L, **kw):
    return orc.MDParams(L=(L,) * 3, **kw)


def test_single_pair_certain_acceptance():
    # k dt Theta = 200 * 0.005 * 1 = 1 -> every candidate is retained
    rx = rx_of(synth.step_growth_scheme(f=4, k=200.0, theta=1))
    s = make([[1, 1, 1], [2.05, 1, 1]], [synth.TYPE_A, synth.TYPE_B], [4, 0])
    tr = orc.react(s, md_for(10.0), rx, step=1)
    assert tr == dict(candidates=1, retained=1, a_winners=1, formed=1)
    assert s.state.tolist() == [3, 1]
    assert s.bonds().tolist() == [[1, 0, 1, 0]]
    assert s.adj[0, 0] == 1 and s.adj[1, 0] == 0


@pytest.mark.parametrize("use_cells", [False, True])
def test_cutoff_is_strict(use_cells):
    rx = rx_of(synth.step_growth_scheme(f=4, k=200.0, theta=1))
    r = 1.1
    inside = make([[1, 1, 1], [1 + np.nextafter(r, 0), 1, 1]], [1, 0], [4, 0])
    at = make([[1, 1, 1], [1 + r, 1, 1]], [1, 0], [4, 0])
    # 1 + r rounds: check the exact distance that the oracle sees
    d_at = (1 + r) - 1
    orc.react(inside, md_for(10.0), rx, 1, use_cells)
    orc.react(at, md_for(10.0), rx, 1, use_cells)
    assert inside.nb == 1
    assert at.nb == (1 if d_at * d_at < r * r else 0)


def test_no_rebond_of_bonded_pair_and_windows():
    rx = rx_of(synth.step_growth_scheme(f=4, k=200.0, theta=1))
    s = make([[1, 1, 1], [2, 1, 1]], [1, 0], [4, 0])
    for st in range(1, 4):
        orc.react(s, md_for(10.0), rx, st)
    assert s.nb == 1  # the pair is bonded once, never again
    # B at state 2 (two bonds) is no longer a target
    s2 = make([[1, 1, 1], [2, 1, 1]], [1, 0], [4, 2])
    orc.react(s2, md_for(10.0), rx, 1)
    assert s2.nb == 0
    # A at state 0 is exhausted
    s3 = make([[1, 1, 1], [2, 1, 1]], [1, 0], [0, 0])
    orc.react(s3, md_for(10.0), rx, 1)
    assert s3.nb == 0


def test_overlapping_windows_rejected():
    d = synth.chain_growth_scheme(k=0.1)
    assert orc.check_reaction(rx_of(d)) == orc.OK
    d2 = dict(d, t_hi=2)  # type B would be eligible as A and T at state 2
    assert orc.check_reaction(rx_of(d2)) == orc.EINVAL


def ring(n_around, center_type, around_type, center_state, around_state, radius=1.0):
    pts = [[5.0, 5.0, 5.0]]
    for q in range(n_around):
        a = 2 * math.pi * q / n_around
        pts.append([5.0 + radius * math.cos(a), 5.0 + radius * math.sin(a), 5.0])
    return make(pts, [center_type] + [around_type] * n_around,
                [center_state] + [around_state] * n_around)


def test_one_target_many_actives_uniform_choice():
    """Step 7: a T named by n A's reacts with exactly one, each with 1/n."""
    n = 5
    rx = rx_of(synth.step_growth_scheme(f=4, k=200.0, theta=1))
    wins = np.zeros(n, int)
    trials = 2000
    for seed in range(trials):
        s = ring(n, synth.TYPE_B, synth.TYPE_A, 0, 4, radius=0.9)
        tr = orc.react(s, md_for(10.0, seed=seed), rx, step=1)
        assert tr["formed"] == 1 and tr["a_winners"] == n
        assert s.state[0] == 1
        wins[int(s.bonds()[0, 1]) - 1] += 1
    chi2 = ((wins - trials / n) ** 2 / (trials / n)).sum()
    assert chi2 < 18.5  # 4 dof, p ~ 1e-3


def test_one_active_many_targets_uniform_choice():
    """Step 5: an A with n retained targets keeps exactly one, each with 1/n."""
    n = 6
    rx = rx_of(synth.step_growth_scheme(f=4, k=200.0, theta=1))
    wins = np.zeros(n, int)
    trials = 2400
    for seed in range(trials):
        s = ring(n, synth.TYPE_A, synth.TYPE_B, 4, 0, radius=0.9)
        tr = orc.react(s, md_for(10.0, seed=seed), rx, step=1)
        assert tr["formed"] == 1 and tr["retained"] == n
        wins[int(s.bonds()[0, 2]) - 1] += 1
    chi2 = ((wins - trials / n) ** 2 / (trials / n)).sum()
    assert chi2 < 20.5  # 5 dof, p ~ 1e-3


def test_isolated_pair_acceptance_rate():
    """Eq. 4: a lone candidate pair bonds with probability k dt Theta per
    reaction step, so after m steps P(bonded) = 1 - (1 - p)^m."""
    k, theta = 6.0, 10
    p = k * 0.005 * theta  # 0.3
    rx = rx_of(synth.step_growth_scheme(f=4, k=k, theta=theta))
    trials, m = 3000, 3
    bonded = 0
    for seed in range(trials):
        s = make([[1, 1, 1], [2, 1, 1]], [1, 0], [4, 0])
        for st in range(1, m + 1):
            orc.react(s, md_for(10.0, seed=seed + 10_000), rx, step=theta * st)
        bonded += s.nb
    expect = 1 - (1 - p) ** m
    sd = math.sqrt(trials * expect * (1 - expect))
    assert abs(bonded - trials * expect) < 4 * sd


def test_brute_force_enumeration_tiny():
    """Independent enumeration of Table I on a tiny frozen configuration with
    every candidate retained: the outcome must be a maximal set of disjoint
    candidate pairs in which every A that has a candidate either bonded or
    lost its chosen T to another A."""
    rng = np.random.default_rng(4)
    rx = rx_of(synth.step_growth_scheme(f=4, k=200.0, theta=1))
    for trial in range(200):
        n = 14
        L = 3.2
        x = rng.random((n, 3)) * L
        types = rng.integers(0, 2, n)
        states = np.where(types == synth.TYPE_A, rng.integers(0, 5, n), rng.integers(0, 3, n))
        s = make(x, types, states, L=L)
        md = md_for(L, seed=trial)
        before = s.state.copy()
        orc.react(s, md, rx, step=1)
        # independent enumeration of the candidate set
        cand = set()
        for i in range(n):
            if types[i] == 1 and 1 <= before[i] <= 4:
                for j in range(n):
                    if types[j] == 0 and 0 <= before[j] <= 1:
                        d = x[j] - x[i]
                        d = np.where(d > L / 2, d - L, np.where(d < -L / 2, d + L, d))
                        if d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < 1.21 - 1e-12:
                            cand.add((i, j))
        b = s.bonds()
        formed = {(int(r[1]), int(r[2])) for r in b}
        assert formed <= cand
        a_used = [p[0] for p in formed]
        t_used = [p[1] for p in formed]
        assert len(set(a_used)) == len(a_used) and len(set(t_used)) == len(t_used)
        # every A with a candidate whose candidates' Ts are all free would have bonded
        for i in {p[0] for p in cand}:
            if i not in a_used:
                assert any(p[1] in t_used for p in cand if p[0] == i)
        # states moved by exactly delta_A, delta_T
        for a, t in formed:
            assert s.state[a] == before[a] - 1 and s.state[t] == before[t] + 1


# ---- the LAMMPS nearest-partner rule (Sec. IV.A) -----------------------------
def nearest_rx(k=200.0, theta=1, f=4):
    return rx_of(synth.step_growth_scheme(f=f, k=k, theta=theta, selection=orc.SELECT_NEAREST))


def test_nearest_rule_hand_built():
    """A0 - T1 at 0.9 and A3 - T2 at 0.8 are mutual nearest pairs; A0 - T2 at
    1.0 is in range but neither picks the other: two bonds, always (p = 1),
    where the random rule would sometimes pair A0 with T2."""
    A, B = synth.TYPE_A, synth.TYPE_B
    x = [[1, 1, 1], [1.9, 1, 1], [1, 2.0, 1], [1, 2.8, 1]]
    s = make(x, [A, B, B, A], [4, 0, 0, 4])
    tr = orc.react(s, md_for(10.0), nearest_rx(), step=7)
    assert tr == dict(candidates=3, retained=2, a_winners=2, formed=2)
    assert sorted(map(tuple, s.bonds()[:, 1:3].tolist())) == [(0, 1), (3, 2)]
    # without T1, A0's nearest is T2, whose nearest is A3: A0 stays unbonded
    s = make([x[0], [5.0, 5.0, 5.0], x[2], x[3]], [A, B, B, A], [4, 0, 0, 4])
    tr = orc.react(s, md_for(10.0), nearest_rx(), step=7)
    assert tr["retained"] == 1 and s.bonds()[:, 1:3].tolist() == [[3, 2]]


def test_nearest_rule_brute_force():
    """Independent enumeration on random dense configurations: with p = 1 the
    bonds are exactly the mutual nearest (A, T) pairs; with p < 1 a subset, of
    which each pair's draw, keyed by (step, smaller id, larger id, tag 5),
    is below p."""
    rng = np.random.default_rng(11)
    for trial in range(120):
        n, L = 30, 4.0
        x = rng.random((n, 3)) * L
        types = rng.integers(0, 2, n)
        states = np.where(types == synth.TYPE_A, rng.integers(0, 5, n), rng.integers(0, 3, n))
        isA = (types == synth.TYPE_A) & (states >= 1) & (states <= 4)
        isT = (types == synth.TYPE_B) & (states <= 1)
        d2 = np.full((n, n), np.inf)
        for i in range(n):
            for j in range(n):
                if (isA[i] and isT[j]) or (isT[i] and isA[j]):
                    d = x[j] - x[i]
                    d = np.where(d > L / 2, d - L, np.where(d < -L / 2, d + L, d))
                    r2 = float(d @ d)
                    if r2 < 1.21:
                        d2[i, j] = r2
        near = [int(np.argmin(d2[i])) if np.isfinite(d2[i]).any() else -1 for i in range(n)]
        mutual = {(a, near[a]) for a in range(n) if isA[a] and near[a] >= 0 and near[near[a]] == a}
        k = 200.0 if trial % 2 == 0 else 60.0  # p = 1 or 0.3
        s = make(x, types, states, L=L)
        md = md_for(L, seed=1000 + trial)
        tr = orc.react(s, md, nearest_rx(k=k), step=3)
        formed = {(int(r[1]), int(r[2])) for r in s.bonds()}
        assert tr["retained"] == len(mutual)
        if k == 200.0:
            assert formed == mutual
        else:
            assert formed <= mutual
            p = k * 0.005
            for a, t in mutual:
                lo, hi = min(a, t), max(a, t)
                w = orc.philox4x32_10([3, lo, hi, 5], [1000 + trial, 0])
                assert ((a, t) in formed) == (orc.u53(w[0], w[1]) < p)


def check_invariants(s, scheme, f, new_steps):
    n = s.n
    b = s.bonds()
    assert len({(int(r[1]), int(r[2])) for r in b}) == len(b)
    assert all(r[1] != r[2] for r in b)
    deg = np.zeros(n, int)
    for r in b:
        deg[r[1]] += 1
        deg[r[2]] += 1
    assert (deg == s.nadj).all()
    for st in new_steps:
        rows = b[b[:, 0] == st]
        ends = np.concatenate([rows[:, 1], rows[:, 2]])
        assert len(ends) == len(set(ends.tolist()))  # at most one new bond per particle
    if scheme == "step":
        A = s.type == synth.TYPE_A
        assert (deg[A] == f - s.state[A]).all()      # bonds formed per A = f - state
        assert (deg[~A] == s.state[~A]).all()
        assert deg[A].max(initial=0) <= f and deg[~A].max(initial=0) <= 2
        assert (s.state >= 0).all()
    else:
        assert deg.max(initial=0) <= 2
        assert set(np.unique(s.state).tolist()) <= {0, 1, 2}


def test_step_growth_invariants_during_a_run():
    inp = synth.step_growth(450, 50, 4, seed=11)
    s = orc.System(inp.x, inp.v, inp.type, inp.state, cap=4)
    md = md_for(inp.L)
    rx = rx_of(synth.step_growth_scheme(f=4, k=1.0))
    for chunk in range(60):
        orc.run(s, md, rx, 10)
        check_invariants(s, "step", 4, [s.step])
    assert s.nb > 20


def chains_are_paths(s):
    """Chain growth: every connected component is a simple path whose single
    P* (state 2) is an end, and whose other end is the initiator (Sec. II.A)."""
    n = s.n
    adj = [list(s.adj[i, :s.nadj[i]]) for i in range(n)]
    seen = np.zeros(n, bool)
    for i in range(n):
        if seen[i] or s.nadj[i] == 0:
            continue
        comp, stack = [], [i]
        seen[i] = True
        while stack:
            u = stack.pop()
            comp.append(u)
            for w in adj[u]:
                if not seen[w]:
                    seen[w] = True
                    stack.append(w)
        edges = sum(len(adj[u]) for u in comp) // 2
        assert edges == len(comp) - 1  # a tree ...
        assert max(len(adj[u]) for u in comp) <= 2  # ... of degree <= 2: a path
        ends = [u for u in comp if len(adj[u]) == 1]
        actives = [u for u in comp if s.state[u] == 2]
        inits = [u for u in comp if s.type[u] == synth.TYPE_A]
        assert len(actives) == 1 and actives[0] in ends
        assert len(inits) == 1 and inits[0] in ends


def test_chain_growth_produces_linear_chains():
    inp = synth.chain_growth(480, 20, seed=2)
    s = orc.System(inp.x, inp.v, inp.type, inp.state, cap=2)
    md = md_for(inp.L)
    rx = rx_of(synth.chain_growth_scheme(k=2.0))
    for chunk in range(60):
        orc.run(s, md, rx, 10)
        check_invariants(s, "chain", 1, [s.step])
    chains_are_paths(s)
    assert s.nb > 40
    # every initiator has either stayed P* or handed the activity on
    init = s.type == synth.TYPE_A
    assert ((s.state[init] == 2) | (s.state[init] == 1)).all()


def test_reaction_cells_match_all_pairs():
    for seed in range(3):
        inp = synth.step_growth(900, 100, 4, seed=seed, jitter=0.5)
        md = md_for(inp.L, seed=seed)
        rx = rx_of(synth.step_growth_scheme(f=4, k=20.0))
        a = orc.System(inp.x, inp.v, inp.type, inp.state, cap=4)
        b = orc.System(inp.x, inp.v, inp.type, inp.state, cap=4)
        ta = orc.react(a, md, rx, 10, use_cells=False)
        tb = orc.react(b, md, rx, 10, use_cells=True)
        assert ta == tb and ta["formed"] > 10
        assert (a.bonds() == b.bonds()).all()
        assert (a.state == b.state).all()


# --------------------------------------------------------------------------
# Rate equations (Secs. II.A, II.B)
# --------------------------------------------------------------------------
from oracle import rate_equations as req  # noqa: E402


def test_step_kinetics_closed_forms():
    t = np.linspace(0, 8, 17)
    # f = 1: x0 = exp(-k0 t)
    x = req.step_kinetics(t, [0.7], 1)
    assert np.allclose(x[:, 0], np.exp(-0.7 * t), atol=1e-9)
    assert np.allclose(x[:, 1], 1 - np.exp(-0.7 * t), atol=1e-9)
    # equal rates: a chain of first-order steps gives Poisson populations for s < f
    k, f = 0.45, 4
    x = req.step_kinetics(t, [k] * f, f)
    for s in range(f):
        assert np.allclose(x[:, s], (k * t) ** s * np.exp(-k * t) / math.factorial(s), atol=1e-9)
    assert np.allclose(x.sum(1), 1.0, atol=1e-12)
    # distinct rates, f = 2 (Bateman): x1 = k0/(k1-k0) (e^{-k0 t} - e^{-k1 t})
    k0, k1 = 0.9, 0.3
    x = req.step_kinetics(t, [k0, k1], 2)
    assert np.allclose(x[:, 1], k0 / (k1 - k0) * (np.exp(-k0 * t) - np.exp(-k1 * t)), atol=1e-9)


def test_chain_fraction_limits():
    assert req.chain_fraction(0.0, 0.1, 3.25, 0.01) == pytest.approx(0.01)
    assert req.chain_fraction(1e6, 0.1, 3.25, 0.01) == pytest.approx(1.0)
    assert req.chain_fraction(0.0, 0.1, 3.25, 0.01, approximate=True) == 0.0


# ---- pair-distance histogram (g(r) -> <N>, Secs. V-VI) ----------------------
def test_pair_histogram_lattice_shells():
    """Simple cubic lattice: 6, 12 and 8 neighbours at a, a sqrt2, a sqrt3."""
    m, a = 6, 1.0
    g = np.stack(np.meshgrid(*[np.arange(m)] * 3, indexing="ij"), -1).reshape(-1, 3) * a + 0.5
    s = orc.System(g, np.zeros_like(g), np.zeros(len(g), np.uint8), np.zeros(len(g), np.int8),
                   cap=1)
    c, na, nb = orc.pair_histogram(s, md_for(m * a), (1, 0, 0), (1, 0, 0), 2.0, 20)
    assert na == nb == m ** 3
    expect = np.zeros(20, np.int64)
    expect[10], expect[14], expect[17] = 6 * na, 12 * na, 8 * na  # bins of 0.1
    assert np.array_equal(c, expect)


def test_pair_histogram_ideal_gas_and_symmetry():
    """Uniform random points: counts per shell = N_a rho_b V_shell within 5
    sigma; counting (a, b) and (b, a) gives the same histogram."""
    rng = np.random.default_rng(5)
    n, L = 3000, 12.0
    x = rng.random((n, 3)) * L
    t = rng.integers(0, 2, n).astype(np.uint8)
    s = orc.System(x, np.zeros_like(x), t, np.zeros(n, np.int8), cap=1)
    ca, na, nb = orc.pair_histogram(s, md_for(L), (1, 0, 0), (2, 0, 0), 1.5, 15)
    cb, nb2, na2 = orc.pair_histogram(s, md_for(L), (2, 0, 0), (1, 0, 0), 1.5, 15)
    assert np.array_equal(ca, cb) and na == na2 and nb == nb2
    edges = np.linspace(0, 1.5, 16)
    expect = na * nb / L ** 3 * 4.0 / 3.0 * np.pi * np.diff(edges ** 3)
    assert np.all(np.abs(ca - expect) < 5 * np.sqrt(expect) + 1)


# ---- thermoneutral bonding (mirror LJ, Eq. 17 and Sec. II) ------------------
@pytest.mark.parametrize("style", [orc.BOND_FENE, orc.BOND_MIRROR_LJ])
def test_bond_creation_energy_jump(style):
    """A reaction step changes no position or velocity, so the energy changes
    by the new bonds' potential alone: zero for mirror-LJ bonds formed at
    r <= r_react <= sigma_c (thermoneutral), and the sum of the FENE energies
    -k R0^2 / 2 ln(1 - (r/R0)^2) of the new bonds otherwise."""
    inp = synth.step_growth(1600, 400, 4, 9, jitter=0.5)
    s = orc.System(inp.x, inp.v, inp.type, inp.state, cap=4)
    md = md_for(inp.L, seed=9)
    _, e0 = orc.forces(s, md, use_cells=True)
    rx = rx_of(synth.step_growth_scheme(4, k=200.0, theta=1, bond_style=style))
    orc.react(s, md, rx, step=1)
    _, e1 = orc.forces(s, md, use_cells=True)
    b = s.bonds()
    assert len(b) > 50
    if style == orc.BOND_MIRROR_LJ:
        assert e1 == e0
    else:
        d = s.x[b[:, 2]] - s.x[b[:, 1]]
        d -= inp.L * np.round(d / inp.L)
        r2 = (d ** 2).sum(1)
        jump = (-0.5 * 30.0 * 1.5 ** 2 * np.log(1.0 - r2 / 1.5 ** 2)).sum()
        assert abs((e1 - e0) - jump) < 1e-9 * jump and jump > 10.0 * len(b)


# ---- step growth against the rate equation (Sec. II.B, Eq. step-kin) --------
def test_low_functionality_step_growth_follows_the_rate_equation():
    """f = 1 crosslinkers among difunctional targets in the short-time regime
    (k <N> t <= 1, t <= 3): the fraction of crosslinkers that have not
    reacted decays as exp(-k <N_XE> t), <N_XE> the mean number of available
    targets within r_react per unreacted crosslinker, measured on the same
    runs (Table I candidates).  Four seeds; within 3 standard errors (or
    0.02)."""
    k, theta, nsteps = 0.1, 10, 600
    rx = rx_of(synth.step_growth_scheme(f=1, k=k, theta=theta))
    fr, cand, elig = [], 0, 0
    for seed in range(4):
        inp = synth.step_growth(1000, 250, 1, 300 + seed)
        s = orc.System(inp.x, inp.v, inp.type, inp.state, cap=2)
        md = md_for(inp.L, seed=300 + seed)
        curve = []
        for q in range(nsteps // theta):
            for _ in range(theta):
                orc.step(s, md)
            n_el = int(((s.type == synth.TYPE_A) & (s.state == 1)).sum())
            tr = orc.react(s, md, rx, step=s.step, use_cells=True)
            cand += tr["candidates"]
            elig += n_el
            curve.append(((s.type == synth.TYPE_A) & (s.state == 1)).sum() / 250.0)
        fr.append(curve)
    fr = np.array(fr)
    n_mean = cand / elig
    t = 0.005 * theta * np.arange(1, nsteps // theta + 1)
    theory = np.exp(-k * n_mean * t)
    assert k * n_mean * t[-1] <= 1.1
    for q in (19, 39, 59):  # t = 1, 2, 3
        se = fr[:, q].std(ddof=1) / 2.0
        assert abs(fr[:, q].mean() - theory[q]) < max(3 * se, 0.02), (q, fr[:, q].mean(), theory[q])
    assert 1.0 < n_mean < 8.0 and fr[:, -1].mean() < 0.5
