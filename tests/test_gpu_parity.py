"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Both sides start from the same seeded synthetic inputs (synth); the oracle
never receives anything the GPU produced.  Bars:
  * reaction step: bit-exact bonds, states and Table I counts;
  * forces, FP64 mode: relative 1e-12; FP32 mode: max_i |df_i| / RMS |f| and
    RMS |df| / RMS |f| both <= 1e-5 (the stated force tolerance);
  * FP64-mode trajectories: positions within 1e-9 after hundreds of steps and
    bit-identical bond lists (same random draws, same decisions).
"""
import math

import numpy as np
import pytest

import oracle as orc
import synth
from helpers import (bonds_of_oracle, canonical, force_errors, gpu, gpu_reaction, gpu_system,
                     md_params, oracle_system, orc_reaction)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return gpu()


def seeded_state(kind, n, seed, jitter=0.5, pre_reactions=0, k_pre=2.0):
    """Synthetic system, optionally given some bonds by oracle reaction steps
    (the oracle's output only ever flows into the GPU, never back)."""
    if kind == "step4":
        inp = synth.step_growth_sites(n, 4, seed, jitter=jitter)
        scheme = synth.step_growth_scheme(4, k=0.1)
    elif kind == "step6":
        inp = synth.step_growth_sites(n, 6, seed, jitter=jitter)
        scheme = synth.step_growth_scheme(6, k=0.1)
    elif kind == "step_cfg1":
        inp = synth.step_growth(int(n * 0.8), n - int(n * 0.8), 4, seed, jitter=jitter)
        scheme = synth.step_growth_scheme(4, k=0.1)
    else:
        inp = synth.chain_growth(n - max(1, n // 100), max(1, n // 100), seed, jitter=jitter)
        scheme = synth.chain_growth_scheme(k=0.1)
    cap = max(scheme["max_valence"])
    o = oracle_system(inp.x, inp.v, inp.type, inp.state, cap)
    md = md_params(inp.L, seed)
    pre = dict(scheme, k=k_pre)
    for q in range(pre_reactions):
        orc.react(o, md, orc_reaction(pre), step=1000 + 10 * q, use_cells=True)
    return inp, scheme, cap, o, md


def gpu_from_oracle_state(P, inp, o, cap, seed, fp64=False, **kw):
    return gpu_system(P, inp.L, o.x, o.v, o.type, o.state, cap=cap, fp64=fp64, seed=seed,
                      bonds=bonds_of_oracle(o), **kw)


# ---------------------------------------------------------------------------
# Reaction step: bit-exact
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind,n,k,pre,sel", [
    ("step_cfg1", 1250, 0.1, 0, 0),
    ("step_cfg1", 1250, 20.0, 3, 0),
    ("step4", 1257, 200.0, 2, 0),       # p = 1: every candidate retained
    ("step6", 4099, 5.0, 2, 0),
    ("chain", 3001, 1.0, 4, 0),
    ("chain", 33096, 0.1, 2, 0),
    ("step4", 33096, 2.0, 3, 0),
    # the LAMMPS nearest-partner rule (Sec. IV.A)
    ("step_cfg1", 1250, 20.0, 3, 1),
    ("step4", 1257, 200.0, 2, 1),
    ("chain", 3001, 1.0, 4, 1),
    ("step4", 33096, 2.0, 3, 1),
])
def test_react_once_bit_exact(P, kind, n, k, pre, sel):
    seed = 7 + n
    inp, scheme, cap, o, md = seeded_state(kind, n, seed, pre_reactions=pre)
    sch = dict(scheme, k=k, selection=sel)
    g = gpu_from_oracle_state(P, inp, o, cap, seed)
    g.set_reaction(gpu_reaction(P, sch))
    for step in (10, 20, 30):
        tr_o = orc.react(o, md, orc_reaction(sch), step=step, use_cells=True)
        tr_g = g.react_once(step)
        assert tr_g == tr_o, (step, tr_g, tr_o)
        assert (g.states() == o.state).all()
        assert np.array_equal(canonical(g.bonds()), canonical(bonds_of_oracle(o)))
    assert o.nb > 0
    g.close()


@pytest.mark.parametrize("sel", [0, 1])
def test_react_once_bit_exact_wide_cutoff(P, sel):
    """A reaction cutoff beyond the WCA cutoff (r_react = 1.6): the Verlet
    lists grow to ~35 entries, so each lane of the four-lane search walks
    several groups of four entries."""
    n, seed = 4099, 77
    inp, scheme, cap, o, md = seeded_state("step4", n, seed, pre_reactions=0)
    sch = dict(scheme, k=0.5, selection=sel, r_react=1.6)
    g = gpu_from_oracle_state(P, inp, o, cap, seed)
    g.set_reaction(gpu_reaction(P, sch))
    for step in (10, 20, 30):
        tr_o = orc.react(o, md, orc_reaction(sch), step=step, use_cells=True)
        tr_g = g.react_once(step)
        assert tr_g == tr_o, (step, tr_g, tr_o)
        assert (g.states() == o.state).all()
        assert np.array_equal(canonical(g.bonds()), canonical(bonds_of_oracle(o)))
    assert o.nb > 0
    g.close()


def test_react_once_edge_cases(P):
    # empty system
    d = P.make_desc(0, 10.0)
    with P.System(d, np.zeros((0, 3)), None, np.zeros(0, np.uint8), np.zeros(0, np.int8)) as g:
        g.set_reaction(gpu_reaction(P, synth.step_growth_scheme(4, 0.1)))
        assert g.react_once(10) == dict(candidates=0, retained=0, a_winners=0, formed=0)
        g.run(25)
        assert g.bonds().shape == (0,)
    # a lone pair exactly at, just inside and just outside the cutoff
    sch = synth.step_growth_scheme(4, k=200.0, theta=1)
    for r, expect in ((1.0999999, 1), (np.nextafter(1.1, 2.0), 0)):
        x = np.array([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]])
        o = oracle_system(x, np.zeros((2, 3)), np.array([1, 0]), np.array([4, 0]), 4)
        orc.react(o, md_params(10.0, 3), orc_reaction(sch), step=1)
        with gpu_system(P, 10.0, x, None, np.array([1, 0], np.uint8), np.array([4, 0], np.int8),
                        seed=3) as g:
            g.set_reaction(gpu_reaction(P, sch))
            tr = g.react_once(1)
            assert tr["formed"] == o.nb
            assert (g.states() == o.state).all()
    # overlapping windows are rejected
    with gpu_system(P, 10.0, np.array([[1.0, 1, 1]]), None, np.array([0], np.uint8),
                    np.array([0], np.int8)) as g:
        bad = dict(synth.chain_growth_scheme(0.1), t_hi=2)
        with pytest.raises(P.PolyrxError) as e:
            g.set_reaction(gpu_reaction(P, bad))
        assert e.value.code == P.PRX_EINVAL


def test_valence_overflow_is_reported(P):
    # max valence 1 for B while the scheme lets a B react twice
    sch = dict(synth.step_growth_scheme(4, k=200.0, theta=1))
    mv = list(sch["max_valence"])
    mv[synth.TYPE_B] = 1
    sch["max_valence"] = tuple(mv)
    x = np.array([[1.0, 1.0, 1.0], [2.0, 1.0, 1.0], [3.0, 1.0, 1.0]])
    with gpu_system(P, 10.0, x, None, np.array([1, 0, 1], np.uint8), np.array([4, 0, 4], np.int8),
                    cap=4) as g:
        g.set_reaction(gpu_reaction(P, sch))
        g.react_once(1)
        with pytest.raises(P.PolyrxError) as e:
            g.react_once(2)
        assert e.value.code == P.PRX_ECAPACITY


# ---------------------------------------------------------------------------
# Forces
# ---------------------------------------------------------------------------
def melted(kind, n, seed, steps=200, pre=3):
    inp, scheme, cap, o, md = seeded_state(kind, n, seed, jitter=0.05, pre_reactions=pre)
    orc.run(o, md, None, steps)  # oracle melts the lattice
    return inp, scheme, cap, o, md


@pytest.mark.parametrize("fp64", [True, False])
@pytest.mark.parametrize("kind,n", [("step_cfg1", 1250), ("chain", 8191)])
def test_forces_match_oracle(P, fp64, kind, n):
    inp, scheme, cap, o, md = melted(kind, n, 11)
    f_ref, e_ref = orc.forces(o, md, use_cells=True)
    with gpu_from_oracle_state(P, inp, o, cap, 11, fp64=fp64) as g:
        f, e = g.forces()
    err = force_errors(f, f_ref)
    if fp64:
        assert err["max_over_rms"] < 1e-12
        assert e == pytest.approx(e_ref, rel=1e-12)
    else:
        assert err["max_over_rms"] < 1e-5, err
        assert err["rms_rel"] < 1e-5, err
        assert e == pytest.approx(e_ref, rel=1e-5)


def test_force_cap_and_mirror_lj(P):
    # uniform placement overlaps particles: the capped warm-up force applies
    rng = np.random.default_rng(5)
    n, L = 2000, synth.box_edge(2000)
    x = synth.uniform_positions(n, L, rng)
    # a hundred mirror-LJ bonds between consecutive ids, at lengths a created bond
    # reaches in a run (the force diverges as r -> 2 sigma_c)
    for i in range(0, 200, 2):
        r = 1.13 + 0.17 * rng.random()
        u = rng.standard_normal(3)
        x[i + 1] = (x[i] + r * u / np.sqrt((u ** 2).sum())) % L
    o = oracle_system(x, np.zeros((n, 3)), np.zeros(n, np.uint8), np.zeros(n, np.int8), 2)
    for i in range(0, 200, 2):
        o.add_bond(i, i + 1, orc.BOND_MIRROR_LJ)
    md = md_params(L, 1, force_cap=50.0)
    f_ref, _ = orc.forces(o, md, use_cells=True)
    for fp64 in (True, False):
        with gpu_system(P, L, x, None, o.type, o.state, cap=2, fp64=fp64, force_cap=50.0,
                        bonds=bonds_of_oracle(o)) as g:
            f, _ = g.forces()
        err = force_errors(f, f_ref)
        assert err["max_over_rms"] < (1e-12 if fp64 else 1e-5), (fp64, err)


@pytest.mark.parametrize("cap", [1, 3, 6])
def test_bond_forces_at_every_bond_count(P, cap):
    """FENE bonds on a jittered lattice, each bead bonded to up to `cap` of
    its lattice neighbours, so that every bond count from 0 to cap occurs
    (odd counts, a single bond with an adjacency row of one entry, rows
    longer than four): FP32 forces of the step kernel's code and the one
    MD step after it against the oracle."""
    rng = np.random.default_rng(100 + cap)
    m = 12
    n = m ** 3
    L = synth.box_edge(n)
    a = L / m
    g3 = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"), -1)
    g3 = g3.reshape(-1, 3)
    x = (g3 + 0.5) * a + rng.uniform(-0.03, 0.03, (n, 3))
    o = oracle_system(x, np.zeros((n, 3)), np.zeros(n, np.uint8), np.zeros(n, np.int8), cap)
    deg = np.zeros(n, int)
    want = rng.integers(0, cap + 1, n)  # each bead's target bond count
    idx = lambda c: int(((c[0] % m) * m + (c[1] % m)) * m + (c[2] % m))
    for i in range(n):
        for d in ((1, 0, 0), (0, 1, 0), (0, 0, 1), (-1, 0, 0), (0, -1, 0), (0, 0, -1)):
            j = idx(g3[i] + np.array(d))
            if i < j and deg[i] < want[i] and deg[j] < cap:
                o.add_bond(i, j, orc.BOND_FENE)
                deg[i] += 1
                deg[j] += 1
    assert set(range(cap + 1)) <= set(deg.tolist()), np.bincount(deg)
    md = md_params(L, 7)
    f_ref, _ = orc.forces(o, md, use_cells=True)
    with gpu_system(P, L, x, None, o.type, o.state, cap=cap, seed=7,
                    bonds=bonds_of_oracle(o)) as g:
        f, _ = g.forces()
        err = force_errors(f, f_ref)
        assert err["max_over_rms"] < 1e-5, err
        g.run(1)
        xg = g.positions()
    orc.step(o, md)
    # FP32 force error (1e-5 of ~50) times dt^2, plus the kick's FP32 rounding:
    # ~1e-8; a missing or doubled bond term would move a bead by ~1e-3
    assert min_image_diff(xg, o.x, L) < 1e-7


# ---------------------------------------------------------------------------
# Trajectories (FP64 mode follows the oracle's arithmetic step for step)
# ---------------------------------------------------------------------------
def min_image_diff(a, b, L):
    d = a - b
    return np.abs(d - L * np.round(d / L)).max()


def test_fp64_trajectory_with_reactions_matches_oracle(P):
    seed = 14097498
    inp = synth.step_growth(1000, 250, 4, seed)
    sch = synth.step_growth_scheme(4, k=1.0)  # p = 0.05: many reactions early
    o = oracle_system(inp.x, inp.v, inp.type, inp.state, 4)
    md = md_params(inp.L, seed)
    with gpu_system(P, inp.L, inp.x, inp.v, inp.type, inp.state, cap=4, fp64=True, seed=seed) as g:
        g.set_reaction(gpu_reaction(P, sch))
        for chunk in range(3):
            obs = orc.run(o, md, orc_reaction(sch), 100)
            g.run(100)
            assert g.step() == o.step
            assert min_image_diff(g.positions(), o.x, inp.L) < 1e-9
            assert np.abs(g.velocities() - o.v).max() < 1e-8
            assert np.array_equal(canonical(g.bonds()), canonical(bonds_of_oracle(o)))
            assert (g.states() == o.state).all()
        hist = g.history()
        assert len(hist) == 30
        assert hist[-1]["bonds"] == o.nb
        assert (hist[-1]["counts"][:8, :16] == obs[-1]["counts"]).all()
        assert o.nb > 50


def test_fp32_trajectory_stays_close(P):
    seed = 99
    inp = synth.chain_growth(3900, 100, seed)
    o = oracle_system(inp.x, inp.v, inp.type, inp.state, 2)
    md = md_params(inp.L, seed)
    with gpu_system(P, inp.L, inp.x, inp.v, inp.type, inp.state, cap=2, seed=seed) as g:
        orc.run(o, md, None, 40)
        g.run(40)
        assert min_image_diff(g.positions(), o.x, inp.L) < 1e-4


def test_langevin_discrete_stationary_law_on_gpu(P):
    """Free particles (eps = 0): stored velocities follow the AR(1) law with
    variance (kT/m) 2/(2 - gamma dt) and lag-1 autocorrelation 1 - gamma dt."""
    n, gamma, dt = 20000, 10.0, 0.005
    rng = np.random.default_rng(3)
    L = 40.0
    x = rng.random((n, 3)) * L
    with gpu_system(P, L, x, None, np.zeros(n, np.uint8), np.zeros(n, np.int8), cap=1, eps=0.0,
                    gamma=gamma, seed=5) as g:
        g.run(300)
        v2, lag = [], []
        prev = g.velocities()
        for _ in range(60):
            g.run(5)
            v = g.velocities()
            v2.append((v ** 2).mean())
            prev = v
        g.run(1)
        a = g.velocities()
        g.run(1)
        b = g.velocities()
    assert np.mean(v2) == pytest.approx(2.0 / (2.0 - gamma * dt), rel=5e-3)
    assert (a * b).mean() / (a * a).mean() == pytest.approx(1 - gamma * dt, abs=1e-2)


# ---------------------------------------------------------------------------
# Whole runs: invariants, determinism, checkpoint, history
# ---------------------------------------------------------------------------
def test_chain_growth_run_invariants_and_determinism(P):
    seed = 5
    inp = synth.chain_growth(32768, 328, seed)
    sch = synth.chain_growth_scheme(k=1.0)
    runs = []
    for rep in range(2):
        with gpu_system(P, inp.L, inp.x, inp.v, inp.type, inp.state, cap=2, seed=seed) as g:
            g.set_reaction(gpu_reaction(P, sch))
            g.run(2000)
            runs.append((g.positions(), canonical(g.bonds()), g.states(), g.stats()))
    (x0, b0, s0, st0), (x1, b1, s1, st1) = runs
    assert np.array_equal(x0, x1) and np.array_equal(b0, b1) and np.array_equal(s0, s1)
    assert st0["rebins"] > 10 and st0["reactions"] == 200
    assert len(b0) > 1000
    # Sec. II.A: linear chains, one active end each, no termination
    n = inp.n
    assert len({(r[1], r[2]) for r in b0.tolist()}) == len(b0) and (b0[:, 1] != b0[:, 2]).all()
    for st in np.unique(b0[:, 0]):  # at most one new bond per particle per reaction step
        ends = b0[b0[:, 0] == st][:, 1:3].ravel()
        assert len(ends) == len(np.unique(ends))
    adj = [[] for _ in range(n)]
    for _, a, t, _ in b0.tolist():
        adj[a].append(t)
        adj[t].append(a)
    assert max(len(r) for r in adj) <= 2
    seen = np.zeros(n, bool)
    for i in range(n):
        if seen[i] or not adj[i]:
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
        assert sum(len(adj[u]) for u in comp) // 2 == len(comp) - 1  # a path
        actives = [u for u in comp if s0[u] == 2]
        inits = [u for u in comp if inp.type[u] == synth.TYPE_A]
        assert len(actives) == 1 and len(adj[actives[0]]) == 1
        assert len(inits) == 1 and len(adj[inits[0]]) == 1
    assert (s0 == 2).sum() == 328  # one P* per chain


def test_checkpoint_continues_bit_for_bit(P, tmp_path):
    seed = 17
    inp = synth.step_growth_sites(20000, 4, seed)
    sch = synth.step_growth_scheme(4, k=0.5)
    path = str(tmp_path / "ck.bin")
    with gpu_system(P, inp.L, inp.x, inp.v, inp.type, inp.state, cap=4, seed=seed) as g:
        g.set_reaction(gpu_reaction(P, sch))
        g.run(137)
        g.save(path)
        g.run(213)
        ref = (g.positions(), g.velocities(), canonical(g.bonds()), g.states())
    g2 = P.System.load(path)
    try:
        assert g2.step() == 137
        g2.run(213)
        got = (g2.positions(), g2.velocities(), canonical(g2.bonds()), g2.states())
    finally:
        g2.close()
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


def test_overstretch_and_bad_input_are_errors(P):
    x = np.array([[1.0, 1.0, 1.0], [2.6, 1.0, 1.0]])  # bond longer than R0 = 1.5
    b = np.zeros(1, P.BOND_DTYPE)
    b["a"], b["t"] = 0, 1
    with gpu_system(P, 10.0, x, None, np.zeros(2, np.uint8), np.zeros(2, np.int8), bonds=b) as g:
        g.run(1)
        with pytest.raises(P.PolyrxError) as e:
            g.sync()
        assert e.value.code == P.PRX_EOVERSTRETCH
    with pytest.raises(P.PolyrxError) as e:  # box below three cutoffs
        gpu_system(P, 3.0, np.array([[1.0, 1, 1]]), None, np.zeros(1, np.uint8), np.zeros(1, np.int8))
    assert e.value.code == P.PRX_EINVAL


def test_observables_and_history_consistent(P):
    seed = 23
    inp = synth.step_growth_sites(10007, 4, seed)
    sch = synth.step_growth_scheme(4, k=0.3)
    with gpu_system(P, inp.L, inp.x, inp.v, inp.type, inp.state, cap=4, seed=seed) as g:
        g.set_reaction(gpu_reaction(P, sch))
        g.run(305)
        ob = g.observables()
        st = g.states()
        ty = g.types()
        h = g.history()
        v = g.velocities()
    assert len(h) == 30 and h[-1]["step"] == 300
    counts = np.zeros((8, 16), np.int64)
    np.add.at(counts, (ty, st), 1)
    assert (ob["counts"] == counts).all()
    assert ob["bonds"] == h[-1]["bonds"]
    assert ob["ke_half"] == pytest.approx(0.5 * (v ** 2).sum(), rel=1e-12)
    assert np.allclose(ob["momentum"], v.sum(0), atol=1e-9)
    # bonds formed per A = f - state (step-growth bookkeeping)
    A = ty == synth.TYPE_A
    assert ob["bonds"] == (4 - st[A]).sum()


def test_pipelined_observables_match_the_synchronous_read(P):
    """prx_observables_begin/end return, for each slot, exactly what the
    synchronous read returns at the same step, while later runs proceed."""
    seed = 29
    inp = synth.step_growth_sites(5003, 4, seed)
    sch = synth.step_growth_scheme(4, k=0.3)

    def make():
        g = gpu_system(P, inp.L, inp.x, inp.v, inp.type, inp.state, cap=4, seed=seed)
        g.set_reaction(gpu_reaction(P, sch))
        return g

    with make() as g:
        g.run(100)
        ref0 = g.observables()
        g.run(100)
        ref1 = g.observables()
    with make() as g:
        g.run(100)
        g.observables_begin(0)
        g.run(100)
        g.observables_begin(1)
        with pytest.raises(P.PolyrxError) as e:
            g.observables_begin(1)  # still pending
        assert e.value.code == P.PRX_EINVAL
        got0 = g.observables_end(0)
        got1 = g.observables_end(1)
        for bad in (lambda: g.observables_end(0), lambda: g.observables_begin(P.PRX_OBS_SLOTS),
                    lambda: g.observables_begin(-1)):
            with pytest.raises(P.PolyrxError) as e:
                bad()
            assert e.value.code == P.PRX_EINVAL
    for got, ref in ((got0, ref0), (got1, ref1)):
        assert got["step"] == ref["step"] and got["bonds"] == ref["bonds"]
        assert (got["counts"] == ref["counts"]).all()
        assert got["ke_half"] == ref["ke_half"]
        assert (got["momentum"] == ref["momentum"]).all()
    assert got0["step"] == 100 and got1["step"] == 200 and got1["bonds"] > got0["bonds"]


def test_ragged_sizes_profile_and_launch_counts(P):
    for n in (1, 2, 127, 128, 129, 4097):
        L = max(4.4, synth.box_edge(n))
        inp = synth.step_growth(n - max(1, n // 9), max(1, n // 9), 4, n, rho=n / L ** 3)
        with gpu_system(P, L, inp.x, inp.v, inp.type, inp.state, cap=4, seed=n) as g:
            g.set_reaction(gpu_reaction(P, synth.step_growth_scheme(4, 1.0)))
            g.run(23)
            P.prx_profile_begin(g.h)
            g.run(10)
            prof = {r["name"]: r for r in P.prx_profile_end(g.h)}
            st = g.stats()
        assert prof["step"]["launches"] == 10 and prof["rx_find"]["launches"] == 1
        assert st["steps"] == 33 and st["kernel_launches"] >= 33


def test_pipelined_newest_reaction_record(P):
    """prx_history_begin / end return the newest reaction record (the same as
    the last entry of prx_get_history), all zero before the first reaction
    step, and the populations equal the states read back."""
    seed = 8
    inp = synth.step_growth(3000, 600, 4, seed)
    with gpu_system(P, inp.L, inp.x, inp.v, inp.type, inp.state, cap=4, seed=seed) as g:
        g.history_begin(0)
        z = g.history_end(0)
        assert z["step"] == 0 and z["bonds"] == 0 and (z["counts"] == 0).all()
        g.set_reaction(gpu_reaction(P, synth.step_growth_scheme(4, k=2.0)))
        for q in range(5):
            g.run(30)
            g.history_begin(q % 2)
            if q:
                prev = g.history_end((q - 1) % 2)
                assert prev["step"] == 30 * q
        last = g.history_end(4 % 2)
        h = g.history()
        assert last["step"] == 150 == h[-1]["step"] and last["bonds"] == h[-1]["bonds"] > 0
        assert np.array_equal(last["counts"], h[-1]["counts"])
        st, ty = g.states(), g.types()
        for t in (synth.TYPE_A, synth.TYPE_B):
            assert np.array_equal(np.bincount(st[ty == t], minlength=16)[:16], last["counts"][t])
