"""The oracle's OpenMP timing driver (used only to time the oracle on every
host core) runs the same trajectory as the single-threaded orc_run, bit for
bit: positions, velocities, states and bonds after MD steps with reactions
(Table I every Theta steps) on several thread counts."""
import numpy as np
import pytest

import oracle as orc
import synth


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_run_omp_is_bit_identical_to_run(threads):
    if orc.omp_lib() is None:
        pytest.skip("no OpenMP compiler on this host")
    inp = synth.step_growth(1000, 250, 4, 11, jitter=0.05)
    sch = synth.step_growth_scheme(4, k=2.0)
    md = orc.MDParams(L=(inp.L,) * 3, seed=11)
    a = orc.System(inp.x, inp.v, inp.type, inp.state, cap=4)
    b = orc.System(inp.x, inp.v, inp.type, inp.state, cap=4)
    orc.run(a, md, orc.Reaction(**sch), 60)
    used = orc.run_omp(b, md, orc.Reaction(**sch), 60, threads)
    assert used == threads
    assert a.nb > 50
    assert np.array_equal(a.x, b.x) and np.array_equal(a.v, b.v)
    assert np.array_equal(a.state, b.state)
    assert np.array_equal(a.bonds(), b.bonds())
