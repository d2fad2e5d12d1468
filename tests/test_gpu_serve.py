"""Serving loop on the GPU: jobs that arrive while others run are admitted by
device memory, share the GPU through one batch, and each job's result (bonds,
states and positions) is the same as when the job runs alone, bit for bit.
"""
import numpy as np
import pytest

import synth
from helpers import canonical, gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return gpu()


def job_system(P, spec):
    inp, sch, cap = synth.replica(spec)
    return dict(desc=P.make_desc(inp.n, inp.L, adj_cap=cap, seed=spec["seed"]), pos=inp.x,
                vel=inp.v, type=inp.type, state=inp.state, reaction=P.make_reaction(**sch))


def test_each_served_job_matches_its_run_alone(P):
    from paper_1409_7498_gb300.serve import Job, PolyrxBackend, Server, serve_trace
    specs = synth.serving_trace(12, rate=400.0, n_lo=1024, n_hi=12000, steps_lo=8, steps_hi=400,
                                k_lo=0.1, k_hi=1.0, seed=77)
    jobs = [Job(job_id=i, nsteps=sp["nsteps"], arrival=sp["arrival"], system=job_system(P, sp),
                n=sp["n"]) for i, sp in enumerate(specs)]
    be = PolyrxBackend(P, positions=True)
    est = sorted(P.prx_estimate_bytes(j.system["desc"]) for j in jobs)
    budget = sum(est[-3:])  # at most about three jobs resident: admission must queue
    srv = Server(be, budget, round_steps=50, theta=10)
    res = serve_trace(srv, jobs)
    be.shutdown()
    assert res["jobs"] == len(jobs)
    assert srv.peak_in_use <= budget
    assert srv.max_members >= 2  # jobs overlapped on the GPU
    assert any(j.admitted - j.arrival > 1e-3 for j in srv.done)  # and some waited for memory
    assert any(j.nsteps % 10 for j in jobs) and min(j.nsteps for j in jobs) < 50
    for j in srv.done:
        s = j.system
        with P.System(s["desc"], s["pos"], s["vel"], s["type"], s["state"]) as g:
            g.set_reaction(s["reaction"])
            g.run(j.nsteps)
            assert g.step() == j.nsteps == j.result["step"]
            assert np.array_equal(canonical(g.bonds()), canonical(j.result["bonds"]))
            assert np.array_equal(g.states(), j.result["states"])
            assert np.array_equal(g.positions(), j.result["positions"])


def test_memory_estimate_covers_the_allocation(P):
    import torch
    spec = dict(kind="step", n=200_000, k=0.1, seed=5)
    s = job_system(P, spec)
    est = P.prx_estimate_bytes(s["desc"])
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    g = P.System(s["desc"], s["pos"], s["vel"], s["type"], s["state"])
    g.set_reaction(s["reaction"])
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    used = free0 - free1
    g.close()
    assert 0.8 * used <= est <= 1.6 * used, (est, used)
