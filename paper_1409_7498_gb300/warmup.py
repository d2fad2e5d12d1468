"""The workloads' start: a seeded uniform placement relaxed on the GPU.

Random placement overlaps particles, so the paper's protocol (App. A) first
runs with a capped pair force and only then with the full potential.  Here:
CAP_STEPS Langevin steps with the WCA pair force capped at F_CAP
(prx_system_desc.force_cap), then FREE_STEPS uncapped steps, no reactions.
Both phases run in the library's kernels; this module only sequences them
through the C ABI binding.
"""
from __future__ import annotations

F_CAP, CAP_STEPS, FREE_STEPS = 100.0, 2000, 1000
SEED_OFFSET = 1_000_003  # the warm-up's thermostat draws differ from a run's


def warmed_liquid(P, inp, adj_cap: int, seed: int, fp64: bool = False, stream=None,
                  cap_steps: int = CAP_STEPS, free_steps: int = FREE_STEPS):
    """Host positions and half-step velocities (by particle id) of `inp`
    (a uniform placement: L, x, v, type, state, n) after the capped and the
    uncapped warm-up phases.  The second phase runs in the force precision
    of the run that follows (fp64)."""
    ws = seed + SEED_OFFSET
    d1 = P.make_desc(inp.n, inp.L, adj_cap=adj_cap, seed=ws, force_cap=F_CAP)
    with P.System(d1, inp.x, inp.v, inp.type, inp.state, stream=stream) as g:
        g.run(cap_steps)
        x, v = g.positions(), g.velocities()
    d2 = P.make_desc(inp.n, inp.L, adj_cap=adj_cap, seed=ws + 1, fp64=fp64)
    with P.System(d2, x, v, inp.type, inp.state, stream=stream) as g:
        g.run(free_steps)
        return g.positions(), g.velocities()
