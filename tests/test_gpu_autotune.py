"""Skin autotuner through the C ABI: it times every candidate, marks a
candidate that cannot run (list radius too large for the box) with -1, and
returns the fastest of the others."""
import pytest

import synth
from helpers import gpu, gpu_reaction

pytestmark = pytest.mark.gpu


def test_autotune_returns_the_fastest_runnable_skin():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P = gpu()
    inp = synth.step_growth_sites(20000, 4, 3)
    desc = P.make_desc(inp.n, inp.L, adj_cap=4, seed=3)
    rx = gpu_reaction(P, synth.step_growth_scheme(4, k=0.1))
    skins = (0.2, 0.3, 0.4, 50.0)  # the last one cannot fit three list radii in the box
    best, times = P.prx_autotune_skin(desc, inp.x, inp.v, inp.type, inp.state, rx, steps=40,
                                      skins=skins)
    assert times[50.0] == -1.0
    ran = {s: t for s, t in times.items() if t > 0}
    assert set(ran) == {0.2, 0.3, 0.4}
    assert best == min(ran, key=ran.get)
    with pytest.raises(P.PolyrxError):
        P.prx_autotune_skin(desc, inp.x, inp.v, inp.type, inp.state, rx, steps=10, skins=(50.0,))
