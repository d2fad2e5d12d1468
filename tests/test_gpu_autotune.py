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


def test_launch_configurations_give_identical_results():
    """Block shape, blocks per SM and reaction intervals per graph replay
    change only the speed: the same run under each is identical bit for bit."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import numpy as np
    P = gpu()
    inp = synth.step_growth_sites(30000, 4, 5)
    rx = gpu_reaction(P, synth.step_growth_scheme(4, k=1.0))
    out = []
    for cfg in [(0, 0, 0), (128, 0, 4), (512, 2, 3), (256, 1, 1)]:
        desc = P.make_desc(inp.n, inp.L, adj_cap=4, seed=5)
        with P.System(desc, inp.x, inp.v, inp.type, inp.state) as g:
            g.set_reaction(rx)
            g.set_launch_config(*cfg)
            lc = g.launch_config()
            assert lc["step_threads"] == (cfg[0] or 256)
            g.run(247)  # not a multiple of the chunk: the run ends interval by interval
            out.append((g.positions(), g.states(), np.sort(g.bonds(), order=["step", "a", "t"])))
    for pos, st, b in out[1:]:
        assert np.array_equal(pos, out[0][0]) and np.array_equal(st, out[0][1])
        assert np.array_equal(b, out[0][2])
    assert len(out[0][2]) > 100
    desc = P.make_desc(inp.n, inp.L, adj_cap=4, seed=5)
    with P.System(desc, inp.x, inp.v, inp.type, inp.state) as g:
        for bad in [(64, 0, 0), (256, 0, 65), (256, 33, 1)]:
            with pytest.raises(P.PolyrxError):
                g.set_launch_config(*bad)


def test_autotune_picks_the_fastest_of_each_stage_and_caches(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P = gpu()
    inp = synth.step_growth_sites(60000, 4, 9)
    desc = P.make_desc(inp.n, inp.L, adj_cap=4, seed=9)
    rx = gpu_reaction(P, synth.step_growth_scheme(4, k=0.1))
    cache = str(tmp_path / "tune.txt")
    kw = dict(steps=60, skins=(0.3, 0.45), shapes=((128, 0), (256, 0), (512, 0), (256, 4)),
              chunks=(1, 2, 4), cache_path=cache)
    best, tried = P.prx_autotune(desc, inp.x, inp.v, inp.type, inp.state, rx, **kw)
    assert [t["stage"] for t in tried] == [0, 0, 1, 1, 1, 1, 2, 2, 2]
    assert all(t["ms_per_step"] > 0 for t in tried)
    # each stage starts from the previous stage's fastest candidate
    s0 = min((t for t in tried if t["stage"] == 0), key=lambda t: t["ms_per_step"])
    s1 = min((t for t in tried if t["stage"] == 1), key=lambda t: t["ms_per_step"])
    s2 = min((t for t in tried if t["stage"] == 2), key=lambda t: t["ms_per_step"])
    assert all(t["skin"] == s0["skin"] for t in tried if t["stage"] > 0)
    assert all((t["step_threads"], t["step_blocks_per_sm"]) ==
               (s1["step_threads"], s1["step_blocks_per_sm"]) for t in tried if t["stage"] == 2)
    assert best == dict(s2, cached=False)
    # the second call comes from the cache (no candidate timed), as does a
    # fresh process reading the file
    again, tried2 = P.prx_autotune(desc, inp.x, inp.v, inp.type, inp.state, rx, **kw)
    assert again["cached"] and not tried2
    assert (again["skin"], again["step_threads"], again["chunk_intervals"]) == \
        (best["skin"], best["step_threads"], best["chunk_intervals"])
    lines = open(cache).read().strip().splitlines()
    assert len(lines) == 1 and "\t" in lines[0]


def test_four_lanes_per_particle_forces_and_run():
    """The four-lane step kernel: forces within the FP32 tolerance of the
    oracle (prx_compute_forces takes the configured lanes), a short run that
    stays close to the one-lane kernel's, and batches refuse such systems."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import numpy as np
    import oracle as orc
    from helpers import force_errors, md_params, oracle_system
    P = gpu()
    inp = synth.step_growth_sites(20000, 4, 13)
    o = oracle_system(inp.x, inp.v, inp.type, inp.state, 4)
    f_ref, e_ref = orc.forces(o, md_params(inp.L, 13), use_cells=True)
    runs = []
    for lanes in (1, 4):
        desc = P.make_desc(inp.n, inp.L, adj_cap=4, seed=13)
        with P.System(desc, inp.x, inp.v, inp.type, inp.state) as g:
            g.set_launch_config(step_lanes=lanes)
            assert g.launch_config()["step_lanes"] == lanes
            f, e = g.forces()
            err = force_errors(f, f_ref)
            assert err["max_over_rms"] < 1e-5 and err["rms_rel"] < 1e-5, (lanes, err)
            assert abs(e - e_ref) / abs(e_ref) < 1e-5
            g.set_reaction(gpu_reaction(P, synth.step_growth_scheme(4, k=1.0)))
            g.run(40)
            runs.append(g.positions())
            if lanes == 4:
                with P.Batch() as b, pytest.raises(P.PolyrxError):
                    b.add(g)
    d = runs[0] - runs[1]
    d -= inp.L * np.round(d / inp.L)
    assert np.abs(d).max() < 1e-3  # FP32 sums in another order, 40 steps apart
