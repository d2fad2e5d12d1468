"""Serving loop on the GPU: jobs that arrive while others run are admitted by
device memory, share the GPU through one batch, and each job's result (bonds,
states and positions) is the same as when the job runs alone, bit for bit.
"""
import time

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
    est = sorted(P.prx_estimate_bytes(j.system["desc"], j.system["reaction"]) for j in jobs)
    budget = sum(est[-3:])  # at most about three jobs resident: admission must queue
    be = PolyrxBackend(P, positions=True, mem_budget=budget)
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
    est = P.prx_estimate_bytes(s["desc"], s["reaction"])
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    g = P.System(s["desc"], s["pos"], s["vel"], s["type"], s["state"])
    g.set_reaction(s["reaction"])
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    used = free0 - free1
    g.close()
    assert 0.8 * used <= est <= 1.6 * used, (est, used)


def test_admission_by_slots_and_memory_epochs_and_poll(P):
    """prx_batch_admit refuses (PRX_ENOMEM) beyond the slots or the memory
    budget; prx_batch_step_epoch never runs a member past its step count
    (a member with less than an interval left finishes alone);
    prx_batch_poll reports each member once its steps are done, frees its
    slot and budget, and the member's result equals its run alone."""
    specs = [dict(kind="step", n=3000, k=1.0, seed=11), dict(kind="chain", n=2500, k=1.0, seed=12),
             dict(kind="step", n=4000, k=0.5, seed=13)]
    systems = [job_system(P, sp) for sp in specs]
    steps = [25, 60, 40]
    est = [P.prx_estimate_bytes(s["desc"], s["reaction"]) for s in systems]

    def make(s):
        g = P.System(s["desc"], s["pos"], s["vel"], s["type"], s["state"])
        g.set_reaction(s["reaction"])
        return g

    # two slots: the third admission is refused, and admitted again once a slot is free
    with P.Batch(max_slots=2) as b:
        gs = [make(s) for s in systems]
        assert b.admit(gs[0], steps[0]) == 0 and b.admit(gs[1], steps[1]) == 1
        assert b.admit(gs[2], steps[2]) is None
        st = b.stats()
        assert st["slots_used"] == 2 and st["bytes_admitted"] == est[0] + est[1]
        owner = {0: gs[0], 1: gs[1]}
        finished, ran = [], []
        t_end = time.time() + 120
        while len(finished) < 3 and time.time() < t_end:
            ran.append(b.step_epoch(100))
            for q in b.poll():
                finished.append(owner.pop(q))
            if gs[2] not in finished and gs[2] not in owner.values():
                q = b.admit(gs[2], steps[2])
                if q is not None:
                    owner[q] = gs[2]
        assert len(finished) == 3
        # epochs were whole reaction intervals that never passed a step count
        assert all(e % 10 == 0 for e in ran) and ran[0] == 20
        for g, s, k in zip(gs, systems, steps):
            assert g.step() == k
            with make(s) as a:
                a.run(k)
                assert np.array_equal(canonical(a.bonds()), canonical(g.bonds()))
                assert np.array_equal(a.states(), g.states())
                assert np.array_equal(a.positions(), g.positions())
        st = b.stats()
        assert st["slots_used"] == 0 and st["bytes_admitted"] == 0 and st["epochs"] >= 3
        for g in gs:
            g.close()
    # memory: a budget for the first system alone refuses the second
    with P.Batch(mem_budget=est[0] + 1) as b:
        g0, g1 = make(systems[0]), make(systems[1])
        assert b.admit(g0, 10) is not None
        assert b.admit(g1, 10) is None
        assert b.step_epoch(100) == 10
        t_end = time.time() + 60
        while not b.poll() and time.time() < t_end:
            pass
        assert b.admit(g1, 10) is not None  # the budget is free again
        assert b.step_epoch(100) == 10
        g0.close()
        g1.close()
