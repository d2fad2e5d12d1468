"""Batched ensemble through the C ABI: many uneven replicas advanced by one
launch per kernel must compute, member by member, exactly what each computes
alone (prx_run): positions and velocities bit for bit, the same bonds,
states, reaction history and rebuild count.  The kernels are the same code
on the same data, so the tolerance is zero.
"""
import numpy as np
import pytest

import synth
from helpers import canonical, gpu, gpu_reaction, gpu_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return gpu()


# kind, beads, rate k, seed: sizes span one block to many, both schemes,
# rates from slow to every-candidate, and one replica with no reaction.
SPECS = [
    dict(kind="step", n=1100, k=1.0, seed=31),
    dict(kind="chain", n=5003, k=1.0, seed=32),
    dict(kind="step", n=20000, k=0.1, seed=33),
    dict(kind="chain", n=9000, k=0.05, seed=34),
    dict(kind="none", n=3001, k=0.0, seed=35),
    dict(kind="step", n=2600, k=0.3, seed=36),
]


def make(P, spec):
    if spec["kind"] == "none":
        inp, _, cap = synth.replica(dict(spec, kind="step", k=0.1))
        g = gpu_system(P, inp.L, inp.x, inp.v, inp.type, inp.state, cap=cap, seed=spec["seed"])
        return g
    inp, sch, cap = synth.replica(spec)
    g = gpu_system(P, inp.L, inp.x, inp.v, inp.type, inp.state, cap=cap, seed=spec["seed"])
    g.set_reaction(gpu_reaction(P, sch))
    return g


def result(g):
    st = g.stats()
    return dict(x=g.positions(), v=g.velocities(), bonds=canonical(g.bonds()), states=g.states(),
                hist=g.history(), step=g.step(), reactions=st["reactions"], rebins=st["rebins"])


def assert_same(a, b):
    for key in ("x", "v", "bonds", "states", "hist"):
        assert np.array_equal(a[key], b[key]), key
    for key in ("step", "reactions", "rebins"):
        assert a[key] == b[key], key


def run_alone(P, spec, chunks):
    g = make(P, spec)
    try:
        for c in chunks:
            g.run(c)
        return result(g)
    finally:
        g.close()


def test_batch_members_match_alone_bit_for_bit(P):
    chunks = (137, 163)  # a partial reaction interval, then the rest
    ref = [run_alone(P, s, chunks) for s in SPECS]
    members = [make(P, s) for s in SPECS]
    with P.Batch() as b:
        for g in members:
            b.add(g)
        for c in chunks:
            b.run(c)
        b.sync()
        st = b.stats()
        got = [result(g) for g in members]
    for g in members:
        g.close()
    for s, r, q in zip(SPECS, ref, got):
        assert_same(r, q)
    assert ref[1]["bonds"].shape[0] > 50 and ref[2]["bonds"].shape[0] > 100
    assert max(r["rebins"] for r in ref) > 3
    assert st["members"] == len(SPECS) and st["active"] == len(SPECS)
    assert st["particles"] == sum(s["n"] for s in SPECS)
    assert st["steps"] == sum(chunks) and st["reactions"] == sum(chunks) // 10
    # one step kernel per step, ten per rebuild (a plan and nine), five per
    # reaction step; device-driven runs add the one-block kernel after each
    # step and one arming kernel per run
    base = st["steps"] + 10 * st["rebuilds"] + 5 * st["reactions"]
    assert st["kernel_launches"] - base in (0, st["steps"] + len(chunks)), (st, base)
    # a rebuild of the batch happens at the union of the members' rebuild steps
    assert max(r["rebins"] for r in ref) - 1 <= st["rebuilds"] <= sum(r["rebins"] - 1 for r in ref)


def test_members_join_and_leave_between_runs(P):
    a, bb, c = SPECS[0], SPECS[2], SPECS[3]
    ref_a = run_alone(P, a, (100, 200))
    ref_b = run_alone(P, bb, (300,))
    ref_c = run_alone(P, c, (200,))
    ga, gb, gc = make(P, a), make(P, bb), make(P, c)
    try:
        with P.Batch() as b:
            b.add(ga)
            b.add(gb)
            b.run(100)
            b.remove(ga)
            ga.run(200)  # continues alone
            b.add(gc)  # joins at step 0, the batch at step 100: same point of the cycle
            b.run(200)
            b.sync()
            got_b, got_c = result(gb), result(gc)
        got_a = result(ga)
    finally:
        for g in (ga, gb, gc):
            g.close()
    assert_same(ref_a, got_a)
    assert_same(ref_b, got_b)
    assert_same(ref_c, got_c)


def test_batch_membership_rules(P):
    g1 = make(P, SPECS[0])
    g2 = make(P, SPECS[5])
    try:
        with P.Batch() as b:
            b.add(g1)
            with pytest.raises(P.PolyrxError) as e:
                g1.run(1)  # members are driven by their batch only
            assert e.value.code == P.PRX_EINVAL
            with pytest.raises(P.PolyrxError) as e:
                b.add(g1)
            assert e.value.code == P.PRX_EINVAL
            g2.run(5)  # half-way through its reaction interval
            with pytest.raises(P.PolyrxError) as e:
                b.add(g2)
            assert e.value.code == P.PRX_EINVAL
            g2.run(5)
            b.add(g2)  # back in phase
            b.run(20)
            b.sync()
            assert g1.step() == 20 and g2.step() == 30
        # the batch is gone: both systems run on their own again
        g1.run(10)
        assert g1.step() == 30
    finally:
        g1.close()
        g2.close()
    inp, sch, cap = synth.replica(SPECS[0])
    with gpu_system(P, inp.L, inp.x, inp.v, inp.type, inp.state, cap=cap, fp64=True) as g64:
        with P.Batch() as b:
            with pytest.raises(P.PolyrxError) as e:
                b.add(g64)
            assert e.value.code == P.PRX_EINVAL
    with make(P, SPECS[0]) as g, make(P, SPECS[5]) as h:
        rx = dict(synth.step_growth_scheme(4, 0.1, theta=7))
        h.set_reaction(gpu_reaction(P, rx))
        with P.Batch() as b:
            b.add(g)
            with pytest.raises(P.PolyrxError) as e:
                b.add(h)  # another reaction interval
            assert e.value.code == P.PRX_EINVAL


def test_batch_reports_the_failing_member(P):
    good = make(P, SPECS[0])
    x = np.array([[1.0, 1.0, 1.0], [2.6, 1.0, 1.0]])  # a bond longer than R0 = 1.5
    bond = np.zeros(1, P.BOND_DTYPE)
    bond["a"], bond["t"] = 0, 1
    bad = gpu_system(P, 10.0, x, None, np.zeros(2, np.uint8), np.zeros(2, np.int8), bonds=bond)
    empty = gpu_system(P, 10.0, np.zeros((0, 3)), None, np.zeros(0, np.uint8), np.zeros(0, np.int8))
    try:
        with P.Batch() as b:
            b.add(good)
            b.add(empty)
            b.add(bad)
            b.run(10)
            with pytest.raises(P.PolyrxError) as e:
                b.sync()
            assert e.value.code == P.PRX_EOVERSTRETCH and e.value.member == 2
        assert good.step() == 10 and empty.step() == 10
    finally:
        for g in (good, bad, empty):
            g.close()


def test_systems_of_different_sizes_coexist(P):
    """A larger system created before a smaller one still runs alone: the
    list-build kernel's shared-memory limit is shared by every system."""
    big = make(P, dict(kind="step", n=60000, k=0.1, seed=41))
    small = make(P, dict(kind="step", n=1100, k=0.1, seed=42))
    try:
        big.run(30)
        small.run(30)
        big.sync()
        small.sync()
        assert big.step() == 30 and small.step() == 30
        assert big.stats()["rebins"] > 1
    finally:
        big.close()
        small.close()
