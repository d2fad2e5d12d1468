"""Benchmark: particle-steps/s of the reactive MD hot path on GB300.

Headline workload: 1,048,576-bead step growth (difunctional B monomers and A
crosslinkers of functionality 4 at a 4:1 B:A site ratio, density 0.85, WCA +
FENE + Langevin, dt = 0.005, reaction every Theta = 10 steps with
r_react = 1.1 and k = 0.1), FP32 forces with FP64 integration.  The start is
the workload's recipe: seeded uniform placement, a capped-force WCA warm-up
(2,000 steps with the pair force capped at 100, then 1,000 uncapped steps, no
reactions, untimed).  The timed region is the whole reaction run: K bench
steps of one reaction interval each (K = 2,000 by default: the 20,000 MD
steps of the workload), every step of the hot path included.

One bench step = one reaction interval: Theta MD steps (fused force +
integrate kernel, conditional neighbour-list rebuilds) followed by the
reaction step and its populations record.  The metric counts particles x MD
steps.  The K steps are one timed region (CUDA events on the launching
stream) replayed in the autotuned graph chunks; the L2 is flushed once
before it, and every step streams the whole system state (~270 MB, more
than the 129 MB L2).

The same JSON line carries the other workloads: the 1,250-bead FP64 step
growth and the 33,096-bead chain growth at k = 0.01, 0.1 and 1 (each a full
run, with its roofline and the oracle timed beside it), the batched ensemble
(256 replicas) against one job at a time, and the serving stream (Poisson
arrivals at 20 jobs/s, unscaled step counts) against serving the same trace
one job at a time.

Multi-GPU (torchrun): every rank advances its own independent replica of the
headline workload (own seed) and its share of the ensemble's replicas; there
is no data-path collective ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from paper_1409_7498_gb300.warmup import CAP_STEPS, F_CAP, FREE_STEPS, warmed_liquid  # noqa: E402

WORKLOAD = "step_growth_1m"
N_BEADS = 1_048_576
FUNC = 4
K_RATE = 0.1
THETA = 10
MD_STEPS = 20_000
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
SKINS = (0.3, 0.35, 0.4, 0.45, 0.5)  # autotuner candidates: Verlet skin,
SHAPES = ((128, 0, 1), (256, 0, 1), (512, 0, 1), (256, 5, 1), (256, 0, 4), (512, 0, 4))
# (step-kernel threads per block, blocks per SM, lanes per particle),
CHUNKS = (1, 2, 5, 10)  # reaction intervals per graph replay


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=MD_STEPS // THETA,
                    help="timed bench steps (reaction intervals of Theta MD steps)")
    ap.add_argument("--warmup", type=int, default=10,
                    help="untimed bench steps of MD on the warmed liquid before the timed run")
    ap.add_argument("--impl", default="polyrx", choices=["polyrx", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=8.0,
                    help="seconds of oracle work per CPU timing")
    ap.add_argument("--direct", action="store_true",
                    help="launch kernels one by one instead of CUDA graphs (for ncu launch lists)")
    ap.add_argument("--profile-roofline", action="store_true",
                    help="bracket the headline's roofline leg with cudaProfilerStart / Stop "
                         "(for ncu --profile-from-start off)")
    ap.add_argument("--no-ensemble", action="store_true",
                    help="skip the batched-ensemble measurement")
    ap.add_argument("--ensemble-steps", type=int, default=20,
                    help="timed reaction intervals of the ensemble measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 1,250-bead and 33,096-bead workload lines")
    ap.add_argument("--skin", type=float, default=0.0,
                    help="Verlet skin to use (default: the library's autotuner picks it)")
    ap.add_argument("--serving-arrivals", type=int, default=64)
    ap.add_argument("--serving-step-scale", type=float, default=1.0)
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def inputs(rank: int, placement: str = "uniform"):
    return synth.step_growth_sites(N_BEADS, FUNC, synth.BASE_SEED + rank, placement=placement)


def scheme():
    return synth.step_growth_scheme(FUNC, k=K_RATE, theta=THETA)


class Clocks:
    """nvidia-smi sampling while the timed region runs."""

    def __init__(self, gpu_index: int):
        self.p = None
        self.path = os.path.join(tempfile.gettempdir(), f"clocks_bench_{os.getpid()}.csv")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_index}",
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [q.strip() for q in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate_throughput(ms_local: float, units_per_rank: int, world: int, dist=None,
                         device="cpu"):
    """Whole-job throughput of independent replicas (weak scaling): the
    slowest rank's time (max over ranks) and all ranks' units over it."""
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if dist is not None and world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, world * units_per_rank / (ms_max * 1e-3)


def algorithmic_bytes_per_particle_step(mean_bonds_per_bead: float) -> float:
    """Step kernel's share of the per-particle-step traffic: FP64 x and v read
    and written (96 B) plus the adjacency entries read (4 B per bond end)."""
    return 96.0 + 4.0 * mean_bonds_per_bead


def peak_hbm():
    if os.path.exists(PEAKS):
        return json.load(open(PEAKS))["hbm_gbs"], "MEASURED_PEAKS.json hbm_gbs (burst copy)"
    return 6800.0, "fallback"


def roofline_of(P, g, n: int, intervals: int = 10) -> dict:
    """Roofline of the step kernel (the dominant kernel): per-kernel CUDA-event
    times on the system's stream over `intervals` further reaction intervals
    (kernels launched one by one), algorithmic bytes from the bond count."""
    P.prx_profile_begin(g.h)
    g.run(intervals * THETA)
    prof = P.prx_profile_end(g.h)
    top = max(prof, key=lambda r: r["total_ms"])
    step_rec = next(r for r in prof if r["name"] == "step")
    nb = g.observables()["bonds"]
    bpp = algorithmic_bytes_per_particle_step(2.0 * nb / max(n, 1))
    avg_ms = step_rec["total_ms"] / step_rec["launches"]
    achieved = n * bpp / (avg_ms * 1e-3) / 1e9
    peak, src = peak_hbm()
    return {"bound": "hbm", "kernel": "step", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": None,
            "algorithmic_bytes_per_particle_step": bpp, "avg_launch_ms": avg_ms,
            "peak_source": src, "top_kernel": top["name"],
            "kernel_ms": {r["name"]: round(r["total_ms"], 4) for r in prof},
            "kernel_launches": {r["name"]: r["launches"] for r in prof}}


def step_kernel_traffic():
    """DRAM bytes of one step-kernel launch from an ncu capture, valid only
    while the step kernel's sources are unchanged since the capture."""
    tr_path = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    if not os.path.exists(tr_path):
        return None
    tr = json.load(open(tr_path))
    h = hashlib.sha256()
    for rel in tr.get("digest_of", []):
        # "path" (the whole file) or "path::until::text" (the file up to the
        # first occurrence of text: the step kernel's part of it)
        path, _, until = rel.partition("::until::")
        with open(os.path.join(ROOT, path), "rb") as f:
            src = f.read()
        if until:
            cut = src.find(until.encode())
            src = src[:cut] if cut >= 0 else b""
        h.update(src)
    if tr.get("kernel_source_digest") == h.hexdigest():
        return tr.get("bytes_per_launch")
    return None


# ---------------------------------------------------------------------------
# The oracle on the host cores
# ---------------------------------------------------------------------------
def oracle_timing(inp, sch, cap: int, seed: int, budget_s: float, max_steps: int,
                  threads: int | None = None) -> dict:
    """The oracle as it stands, on a bounded sample of a workload: MD steps
    (with the reaction every Theta steps) from the given state until the
    budget is spent or max_steps are done.  threads=None: orc_run on one
    thread; else the OpenMP driver (same trajectory) on `threads` threads
    (0: all)."""
    import oracle as orc
    o = orc.System(inp.x, inp.v, inp.type, inp.state, cap=cap)
    md = orc.MDParams(L=(inp.L,) * 3, seed=seed)
    rx = orc.Reaction(**sch)
    cores = 1
    t0 = time.perf_counter()
    steps = 0
    while steps < max_steps:
        if threads is None:
            orc.run(o, md, rx, 1)
        else:
            cores = orc.run_omp(o, md, rx, 1, threads)
        steps += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return {"value": inp.n * steps / el, "unit": "particle-steps/s", "cores": cores,
            "kind": "oracle", "steps": steps, "seconds": el}


def cpu_baselines(inp, sch, cap, seed, budget_s, max_steps, what: str) -> dict:
    """Single-thread and all-core timings of the oracle on one workload."""
    one = oracle_timing(inp, sch, cap, seed, budget_s, max_steps)
    out = {"value": one["value"], "unit": one["unit"], "cores": 1, "kind": "oracle",
           "nproc": os.cpu_count(),
           "sample": f"{one['steps']} MD steps of {what} (reaction every {THETA} steps), FP64, "
                     f"one thread, {one['seconds']:.1f} s"}
    try:
        import oracle as orc
        if orc.omp_lib() is not None:
            allc = oracle_timing(inp, sch, cap, seed, budget_s, max_steps, threads=0)
            out["all_cores"] = {"value": allc["value"], "cores": allc["cores"],
                                "sample": f"{allc['steps']} MD steps, OpenMP over the per-particle "
                                          f"force and integration loops, {allc['seconds']:.1f} s"}
    except Exception as e:  # the single-thread number stands alone
        out["all_cores"] = {"unavailable": str(e)}
    return out


# ---------------------------------------------------------------------------
# The other workloads: 1,250-bead FP64 step growth, 33,096-bead chain growth,
# 1M-bead step growth with crosslinkers of functionality 6
# ---------------------------------------------------------------------------
def small_config(P, torch, name: str, inp, sch: dict, cap: int, fp64: bool, md_steps: int,
                 seed: int, args, stream,
                 l2: str = "flushed once before the timed run (the whole state fits in L2)") -> dict:
    """One full run of a workload other than the headline's from its warmed
    liquid: the whole run timed as one region with CUDA events (the L2 is
    flushed once before it), its step kernel's roofline over ten further
    intervals, and the oracle timed on the same start."""
    xw, vw = warmed_liquid(P, inp, cap, seed, fp64=fp64, stream=stream.cuda_stream)
    rx = P.make_reaction(**sch)
    if fp64:  # the FP64 force mode has fixed kernels: skin and interval batching only
        tune, _ = P.prx_autotune(P.make_desc(inp.n, inp.L, adj_cap=cap, seed=seed, fp64=True), xw,
                                 vw, inp.type, inp.state, rx, steps=200, skins=SKINS, shapes=(),
                                 chunks=CHUNKS)
    else:
        tune, _ = P.prx_autotune(P.make_desc(inp.n, inp.L, adj_cap=cap, seed=seed), xw, vw,
                                 inp.type, inp.state, rx, steps=200, skins=SKINS, shapes=SHAPES,
                                 chunks=CHUNKS)
    desc = P.make_desc(inp.n, inp.L, adj_cap=cap, seed=seed, fp64=fp64, skin=tune["skin"])
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=stream.device)
    with P.System(desc, xw, vw, inp.type, inp.state, stream=stream.cuda_stream) as g:
        g.set_reaction(rx)
        g.set_launch_config(tune["step_threads"], tune["step_blocks_per_sm"],
                            tune["chunk_intervals"], tune["step_lanes"])
        g.run(0)  # graphs captured before the timed region
        st0 = g.stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            flush.fill_(1)
            e0.record(stream)
            g.run(md_steps)
            e1.record(stream)
        torch.cuda.synchronize()
        g.sync()
        ms = e0.elapsed_time(e1)
        st1 = g.stats()
        obs = g.observables()
        roof = roofline_of(P, g, inp.n)
    del flush
    line = {"workload": name, "metric": "particle-steps/s",
            "value": inp.n * md_steps / (ms * 1e-3), "unit": "particle-steps/s",
            "md_steps": md_steps, "ms": ms, "beads": inp.n, "k": sch["k"],
            "autotune": {k: v for k, v in tune.items() if k not in ("stage", "cached")},
            "dtype": "f64" if fp64 else "f32 forces / f64 integration",
            "bonds_end": int(obs["bonds"]), "gpu_launches": int(st1["kernel_launches"]
                                                               - st0["kernel_launches"]),
            "rebins": int(st1["rebins"] - st0["rebins"]), "roofline": roof, "l2": l2}
    if not args.no_cpu_baseline:
        class _W:
            pass
        w = _W()
        w.x, w.v, w.type, w.state, w.L, w.n = xw, vw, inp.type, inp.state, inp.L, inp.n
        line["cpu_baseline"] = cpu_baselines(w, sch, cap, seed, args.cpu_budget, md_steps,
                                             f"the {name} workload from the same warmed start")
    return line


def configs_1_2(P, torch, args, stream) -> dict:
    W1 = synth.WORKLOADS["step_growth_1250_fp64"]
    W2 = synth.WORKLOADS["chain_growth_33096"]
    out = {}
    seed = synth.BASE_SEED + 101
    inp = synth.step_growth(W1["n_B"], W1["n_A"], W1["f"], seed, placement="uniform")
    out["step_growth_1250_fp64"] = small_config(
        P, torch, "step_growth_1250_fp64", inp, synth.step_growth_scheme(W1["f"], k=W1["k"]),
        W1["f"], True, W1["steps"], seed, args, stream)
    for k in W2["k"]:
        seed = synth.BASE_SEED + 202
        inp = synth.chain_growth(W2["n_M"], W2["n_init"], seed, placement="uniform")
        nm = f"chain_growth_33096_k{k:g}"
        out[nm] = small_config(P, torch, nm, inp, synth.chain_growth_scheme(k), 2, False,
                               W2["steps"], seed, args, stream)
    # the 1M-bead step growth with crosslinkers of functionality 6 (the
    # same 4:1 B:A site ratio), its full run
    W3 = synth.WORKLOADS["step_growth_1m"]
    seed = synth.BASE_SEED + 303
    inp = synth.step_growth_sites(W3["n_total"], 6, seed, placement="uniform")
    out["step_growth_1m_f6"] = small_config(
        P, torch, "step_growth_1m_f6", inp, synth.step_growth_scheme(6, k=W3["k"], theta=THETA), 6,
        False, W3["steps"], seed, args, stream,
        l2="inputs larger than L2: every step streams the whole system state (129 MB L2); "
           "one 256 MB flush before the timed run")
    return out


# ---------------------------------------------------------------------------
# Batched ensemble and serving stream
# ---------------------------------------------------------------------------
ENSEMBLE = synth.WORKLOADS["ensemble_256"]


def ensemble(P, torch, steps: int, rank: int = 0, world: int = 1, dist=None,
             warmup: int = 3) -> dict:
    """Batched ensemble (256 replicas, sizes log-uniform in 1,024-65,536
    beads, step or chain growth, k log-uniform in [0.01, 1], own seeds)
    advanced together by one prx_batch, against the same replicas run one at
    a time through prx_run (each run to completion and synchronised before
    the next starts).  Both legs time the same number of MD steps per replica
    from the same state; wall clock around each leg.  A sample of replicas is
    then re-run alone from the initial inputs for the same total number of
    steps and compared bit for bit with the replicas that went through the
    batch (same accuracy: identical results).  With several ranks, rank r
    takes replicas r, r + world, ... and the value is all ranks' replica-steps
    over the slowest rank's time."""
    W = ENSEMBLE
    specs = synth.ensemble_specs(W["replicas"], W["n_lo"], W["n_hi"], W["k_lo"], W["k_hi"],
                                 synth.BASE_SEED)[rank::world]
    reps = []
    for sp in specs:
        inp, sch, cap = synth.replica(sp)
        desc = P.make_desc(inp.n, inp.L, adj_cap=cap, seed=sp["seed"])
        g = P.System(desc, inp.x, inp.v, inp.type, inp.state)
        g.set_reaction(P.make_reaction(**sch))
        reps.append((sp, g))
    beads = sum(sp["n"] for sp in specs)
    nrep = len(reps)
    md_steps = steps * THETA
    stream = torch.cuda.Stream()
    b = P.Batch(stream=stream.cuda_stream)
    for _, g in reps:
        b.add(g)
    b.run(warmup * THETA)
    b.sync()
    st0 = b.stats()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    ev0.record(stream)
    b.run(md_steps)
    ev1.record(stream)
    b.sync()
    t_batch = time.perf_counter() - t0
    ms_batch = ev0.elapsed_time(ev1)
    st1 = b.stats()
    b.close()
    # the same replicas, one job at a time
    for _, g in reps:  # untimed: builds each replica's graphs
        g.run(THETA)
        g.sync()
    t0 = time.perf_counter()
    for _, g in reps:
        g.run(md_steps)
        g.sync()
    t_plain = time.perf_counter() - t0
    total = (warmup + steps + 1 + steps) * THETA
    # same accuracy: a sample re-run alone from the initial inputs
    sample = sorted(range(nrep), key=lambda r: specs[r]["n"])[:: max(1, nrep // 4)][:4]
    identical = True
    for r in sample:
        sp, g = reps[r]
        inp, sch, cap = synth.replica(sp)
        desc = P.make_desc(inp.n, inp.L, adj_cap=cap, seed=sp["seed"])
        with P.System(desc, inp.x, inp.v, inp.type, inp.state) as a:
            a.set_reaction(P.make_reaction(**sch))
            a.run(total)
            identical &= bool(np.array_equal(a.positions(), g.positions())
                              and np.array_equal(a.states(), g.states())
                              and np.array_equal(np.sort(a.bonds(), order=["step", "a", "t"]),
                                                 np.sort(g.bonds(), order=["step", "a", "t"])))
    for _, g in reps:
        g.close()
    tb, tp = t_batch, t_plain
    if dist is not None:
        tb = max_over_ranks(t_batch, dist, world)
        tp = max_over_ranks(t_plain, dist, world)
    n_all = W["replicas"] if world > 1 else nrep
    rs_batch = n_all * md_steps / tb
    rs_plain = n_all * md_steps / tp
    return {"workload": "ensemble_256", "replicas": n_all, "replicas_this_rank": nrep,
            "beads_this_rank": beads, "md_steps_per_replica": md_steps,
            "unit": "replica-steps/s",
            "batched": {"value": rs_batch, "particle_steps_per_s": beads * md_steps / t_batch,
                        "device_ms": ms_batch, "wall_s": t_batch,
                        "kernel_launches": int(st1["kernel_launches"] - st0["kernel_launches"]),
                        "rebuild_steps": int(st1["rebuilds"] - st0["rebuilds"])},
            "plain": {"value": rs_plain, "particle_steps_per_s": beads * md_steps / t_plain,
                      "wall_s": t_plain, "how": "each replica through prx_run, synchronised "
                                                "before the next starts"},
            "speedup": rs_batch / rs_plain, "identical": identical,
            "identical_sample": [specs[r]["n"] for r in sample],
            "l2": "not flushed: the ensemble state (~1 GB) exceeds L2"}


def max_over_ranks(v: float, dist, world: int) -> float:
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


SERVING = synth.WORKLOADS["serving_stream"]


def serving(P, torch, arrivals: int, step_scale: float, rank: int = 0, world: int = 1) -> dict:
    """Serving stream: Poisson arrivals (20 jobs/s) of step- or chain-growth
    jobs of 2,048-262,144 beads (log-uniform) and 5,000-50,000 steps
    (log-uniform), replayed in real time through the continuous-batching
    server (admission by device memory through prx_batch_admit, one shared
    batch), then the same trace one job at a time (FIFO, each job created, run
    alone and read back before the next).  Latency = arrival to result
    read-back.  Only the arrival count is bounded; with step_scale = 1 the
    offered load is the workload's (about 2e10 particle-steps/s, above one
    GPU's capacity, so jobs queue and overlap).  Two jobs are re-run alone
    afterwards and compared bit for bit with their served results.  With
    several ranks, rank r serves arrivals r, r + world, ..."""
    from paper_1409_7498_gb300.serve import Job, PolyrxBackend, Server, serve_serial, serve_trace
    W = SERVING
    lo, hi = max(10, int(W["steps_lo"] * step_scale)), max(10, int(W["steps_hi"] * step_scale))
    specs = synth.serving_trace(arrivals, W["rate"], W["n_lo"], W["n_hi"], lo, hi, W["k_lo"],
                                W["k_hi"], synth.BASE_SEED + 5)[rank::world]

    def jobs():
        out = []
        for i, sp in enumerate(specs):
            inp, sch, cap = synth.replica(sp)
            sysd = dict(desc=P.make_desc(inp.n, inp.L, adj_cap=cap, seed=sp["seed"]), pos=inp.x,
                        vel=inp.v, type=inp.type, state=inp.state,
                        reaction=P.make_reaction(**sch))
            out.append(Job(job_id=i, nsteps=sp["nsteps"], arrival=sp["arrival"], system=sysd,
                           n=sp["n"]))
        return out

    free, _ = torch.cuda.mem_get_info()
    budget = int(min(0.5 * free, 64 << 30))
    be = PolyrxBackend(P, mem_budget=budget)
    srv = Server(be, budget, round_steps=200, theta=THETA)
    jb = jobs()
    res_b = serve_trace(srv, jb)
    be.shutdown()
    res_b.update(rounds=srv.rounds, max_resident_jobs=srv.max_members,
                 mean_resident_jobs=srv.mean_members(), peak_admitted_bytes=srv.peak_in_use,
                 budget_bytes=budget)
    be2 = PolyrxBackend(P)
    res_s = serve_serial(be2, jobs())
    be2.shutdown()
    identical = True
    sample = sorted(range(len(jb)), key=lambda i: jb[i].n * jb[i].nsteps)[:2]
    for i in sample:
        j = jb[i]
        sd = j.system
        with P.System(sd["desc"], sd["pos"], sd["vel"], sd["type"], sd["state"]) as g:
            g.set_reaction(sd["reaction"])
            g.run(j.nsteps)
            identical &= bool(np.array_equal(g.states(), j.result["states"]) and np.array_equal(
                np.sort(g.bonds(), order=["step", "a", "t"]),
                np.sort(j.result["bonds"], order=["step", "a", "t"])))
    beads = [sp["n"] for sp in specs]
    offered = W["rate"] / world * float(np.mean(beads)) * float(
        np.mean([sp["nsteps"] for sp in specs]))
    return {"workload": "serving_stream", "arrivals": len(specs), "rate_per_s": W["rate"],
            "beads": [W["n_lo"], W["n_hi"]], "steps": [lo, hi],
            "bounded": f"{arrivals} of {W['arrivals']} arrivals"
                       + ("" if step_scale == 1.0 else f", steps x{step_scale}"),
            "offered_particle_steps_per_s": offered,
            "batched": res_b, "serial": res_s,
            "p50_speedup": res_s["p50_latency_s"] / res_b["p50_latency_s"],
            "p99_speedup": res_s["p99_latency_s"] / res_b["p99_latency_s"],
            "throughput_ratio": res_b["replica_steps_per_s"] / res_s["replica_steps_per_s"],
            "identical": identical}


# ---------------------------------------------------------------------------
# Reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------
def headline_config(world: int = 1) -> dict:
    """The workload's identity, the same in both arms."""
    return {"workload": WORKLOAD, "beads": N_BEADS, "f": FUNC, "k": K_RATE, "theta": THETA,
            "density": synth.DENSITY, "parallelism": f"replicas x{world}"}


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle, timed on all of this host's cores
    (the OpenMP driver of its per-particle loops, the same trajectory as the
    single-threaded oracle; one thread when OpenMP is missing); each bench
    step is one MD step of the same 1M-bead workload (the reaction every
    Theta steps).  The oracle's start is the workload's lattice placement:
    the capped warm-up of a million beads is GPU work this arm does not run."""
    if rank != 0:
        return
    import oracle as orc
    inp = inputs(0, placement="lattice")
    sch = scheme()
    o = orc.System(inp.x, inp.v, inp.type, inp.state, cap=FUNC)
    md = orc.MDParams(L=(inp.L,) * 3, seed=synth.BASE_SEED)
    rx = orc.Reaction(**sch)
    omp = orc.omp_lib() is not None

    def one():
        return orc.run_omp(o, md, rx, 1, 0) if omp else (orc.run(o, md, rx, 1) or 1)

    for _ in range(min(args.warmup, 3)):
        one()
    t0 = time.perf_counter()
    done = 0
    cores = 1
    budget = 120.0
    for _ in range(args.steps):
        cores = one()
        done += 1
        if time.perf_counter() - t0 > budget:
            break
    el = time.perf_counter() - t0
    v = inp.n * done / el
    how = f"OpenMP over {cores} threads" if omp else "one thread"
    line = {"impl": "reference", "metric": "particle-steps/s", "value": v,
            "unit": "particle-steps/s", "n_gpus": args.gpus, "steps": done, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / max(done, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": headline_config(world),
            "run": {"md_steps_per_bench_step": 1, "md_steps_timed": done,
                    "start": "the workload's lattice placement (no warm-up)"},
            "cpu_baseline": {"value": v, "unit": "particle-steps/s", "cores": cores,
                             "kind": "oracle", "nproc": os.cpu_count(),
                             "sample": f"{done} MD steps of the {inp.n}-bead workload from its "
                                       f"lattice placement, {how}"},
            "e2e": {"value": v, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def main():
    args = parse()
    rank, world, local = dist_env()
    if args.gpus != world:
        print(f"bench.py: --gpus {args.gpus} but WORLD_SIZE={world}; launch one rank per GPU "
              f"with torchrun (--nproc-per-node {args.gpus})", file=sys.stderr)
        sys.exit(2)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    from paper_1409_7498_gb300 import build as gbuild
    from paper_1409_7498_gb300 import polyrx as P

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        gbuild.build()
    if world > 1:
        dist.barrier()
    gbuild.build()
    stream = torch.cuda.Stream(device=dev)

    seed = synth.BASE_SEED + rank
    inp = inputs(rank)
    sch = scheme()
    xw, vw = warmed_liquid(P, inp, FUNC, seed, stream=stream.cuda_stream)
    # the library's autotuner picks the Verlet skin for this workload (timed
    # on temporary copies of the warmed system, outside the timed region)
    if args.skin > 0:
        tune = dict(skin=args.skin, step_threads=256, step_blocks_per_sm=0, chunk_intervals=1,
                    step_lanes=1)
        tried = []
    else:
        tune, tried = P.prx_autotune(
            P.make_desc(inp.n, inp.L, adj_cap=FUNC, seed=seed), xw, vw, inp.type, inp.state,
            P.make_reaction(**sch), steps=100, skins=SKINS, shapes=SHAPES, chunks=CHUNKS)
    skin = tune["skin"]
    desc = P.make_desc(inp.n, inp.L, adj_cap=FUNC, seed=seed, skin=skin)
    g = P.System(desc, xw, vw, inp.type, inp.state, stream=stream.cuda_stream)
    g.set_launch_config(tune["step_threads"], tune["step_blocks_per_sm"], tune["chunk_intervals"],
                        tune["step_lanes"])
    # untimed warm-up bench steps: MD on the warmed liquid; then the reaction
    # scheme is set and its graphs are captured, so the timed region is the
    # whole reaction run
    g.run(args.warmup * THETA)
    g.set_reaction(P.make_reaction(**sch))
    g.run(0)
    g.sync()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st0 = g.stats()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = Clocks(local)
    time.sleep(0.3)
    wall0 = time.perf_counter()
    if args.direct:
        P.prx_profile_begin(g.h)
    with torch.cuda.stream(stream):
        # one L2 flush before the timed region; inside it every step streams
        # the whole system state (~270 MB), more than the 129 MB L2
        flush.fill_(1)
        ev0.record(stream)
        g.run(args.steps * THETA)  # graph replays of the autotuned chunk length
        ev1.record(stream)
    torch.cuda.synchronize()
    if args.direct:
        P.prx_profile_end(g.h)
    wall = time.perf_counter() - wall0
    clocks = clk.stop()
    g.sync()
    st1 = g.stats()
    obs_end = g.observables()
    ms = ev0.elapsed_time(ev1)
    ms_max, value = aggregate_throughput(ms, inp.n * THETA * args.steps, world, dist, dev)
    launches = int(st1["kernel_launches"] - st0["kernel_launches"])
    rebins = int(st1["rebins"] - st0["rebins"])
    n_A = int((inp.type == synth.TYPE_A).sum())
    run_info = {"autotune": {"chosen": tune, "tried": [
                    {k: (round(v, 5) if isinstance(v, float) else v) for k, v in t.items()
                     if k != "cached"} for t in tried]},
                "cells": list(st1["cells"]), "rebins_in_timed_region": rebins, "wall_s": wall,
                "bonds_end": int(obs_end["bonds"]),
                "conversion_end": obs_end["bonds"] / (FUNC * n_A),
                "bonds_per_bead_end": 2.0 * obs_end["bonds"] / inp.n}
    if args.profile_roofline:
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
    roof = roofline_of(P, g, inp.n)
    if args.profile_roofline:
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    roof["traffic"] = step_kernel_traffic()
    del flush

    # end to end through the C ABI with host buffers
    e2e = None
    if rank == 0 and not args.no_e2e:
        pin = {k: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
               for k, a in (("x", xw), ("v", vw), ("t", inp.type), ("s", inp.state))}
        h2d = sum(a.nbytes for a in pin.values())
        torch.cuda.synchronize()
        e0 = time.perf_counter()
        ge = P.System(desc, pin["x"], pin["v"], pin["t"], pin["s"], stream=stream.cuda_stream)
        ge.set_reaction(P.make_reaction(**sch))
        ge.set_launch_config(tune["step_threads"], tune["step_blocks_per_sm"],
                             tune["chunk_intervals"], tune["step_lanes"])
        d2h = 0
        ke = max(args.steps, 1)  # the same number of steps as the device-timed region
        ob = None
        for q in range(ke):
            ge.run(THETA)
            # the step's result (the reaction record: populations per (type,
            # state), bonds, step) copied into a pinned slot; the previous
            # step's is read while this one runs
            ge.history_begin(q % 2)
            if q:
                ob = ge.history_end((q - 1) % 2)
            d2h += P.HISTORY_DTYPE.itemsize + 112  # the record and the 112-byte control block
        ob = ge.history_end((ke - 1) % 2)
        stt = ge.states()
        bd = ge.bonds()
        d2h += stt.nbytes + bd.nbytes
        ge.close()
        e_el = time.perf_counter() - e0
        e2e = {"value": inp.n * THETA * ke / e_el, "unit": "particle-steps/s",
               "h2d_bytes_per_step": int(h2d / ke), "d2h_bytes_per_step": int(d2h / ke),
               "steps": ke, "includes": "create from the warmed host state (upload + binning), "
                                        "runs, per-step read-back of the reaction record "
                                        "(populations, bonds; pipelined, one step behind), "
                                        "final states and bonds, destroy"}
        del ob
    g.close()

    ens = None
    if not args.no_ensemble:
        ens = ensemble(P, torch, args.ensemble_steps, rank, world, dist)
    srv = None
    if not args.no_serving:
        srv = serving(P, torch, args.serving_arrivals, args.serving_step_scale, rank, world)
        if world > 1:  # every rank served its share of the arrivals: gather the summaries
            parts = [None] * world
            dist.all_gather_object(parts, srv)
            srv = {"per_rank": parts, "ranks": world,
                   "replica_steps_per_s": sum(p_["batched"]["replica_steps_per_s"] for p_ in parts),
                   "p99_latency_s_max": max(p_["batched"]["p99_latency_s"] for p_ in parts)}
    cfgs = None
    if world == 1 and not args.no_configs:
        cfgs = configs_1_2(P, torch, args, stream)

    if world > 1:
        dist.barrier()
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            class _W:
                pass
            w = _W()
            w.x, w.v, w.type, w.state, w.L, w.n = xw, vw, inp.type, inp.state, inp.L, inp.n
            cpu = cpu_baselines(w, sch, FUNC, seed, args.cpu_budget, 10 * THETA,
                                f"the {inp.n}-bead workload from the same warmed start")
        line = {
            "metric": "particle-steps/s", "value": value, "unit": "particle-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 forces / f64 integration", "data": "synthetic",
            "config": headline_config(world),
            "run": dict(run_info, md_steps_per_bench_step=THETA, md_steps_timed=args.steps * THETA,
                        start=f"uniform placement, {CAP_STEPS} steps with the WCA force capped at "
                              f"{F_CAP:g}, {FREE_STEPS} uncapped steps (untimed)",
                        l2="inputs larger than L2: every step streams the ~270 MB system state "
                           "(129 MB L2); one 256 MB flush before the timed region"),
            "clocks": clocks, "gpu_launches": launches, "roofline": roof,
            "e2e": e2e, "cpu_baseline": cpu, "configs": cfgs, "ensemble": ens,
            "serving": srv,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
