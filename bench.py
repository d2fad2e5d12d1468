"""Benchmark: particle-steps/s of the reactive MD hot path on GB300.

Workload (default): 1,048,576-bead step growth (difunctional B monomers and
A crosslinkers of functionality 4 at a 4:1 B:A site ratio, density 0.85,
WCA + FENE + Langevin, dt = 0.005, reaction every Theta = 10 steps with
r_react = 1.1 and k = 0.1), FP32 forces with FP64 integration.

One bench step = one reaction interval: Theta MD steps (fused force +
integrate kernel, conditional cell-list rebuilds) followed by the reaction
step and its observables record, i.e. every step of the hot path.  The metric
counts particles x MD steps.  Inputs are synthetic (seeded lattice placement,
Maxwell velocities); the L2 cache is flushed between timed bench steps.

Multi-GPU (torchrun): every rank advances its own independent replica (own
seed); there is no data-path collective ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = "step_growth_1m"
N_BEADS = 1_048_576
FUNC = 4
K_RATE = 0.1
THETA = 10
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
SKINS = (0.3, 0.35, 0.4, 0.45, 0.5)  # autotuner candidates


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="polyrx", choices=["polyrx", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0, help="seconds of oracle work")
    ap.add_argument("--direct", action="store_true",
                    help="launch kernels one by one instead of CUDA graphs (for ncu launch lists)")
    ap.add_argument("--no-ensemble", action="store_true",
                    help="skip the batched-ensemble measurement")
    ap.add_argument("--ensemble-steps", type=int, default=20,
                    help="timed reaction intervals of the ensemble measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--skin", type=float, default=0.0,
                    help="Verlet skin to use (default: the library's autotuner picks it)")
    ap.add_argument("--serving-arrivals", type=int, default=64)
    ap.add_argument("--serving-step-scale", type=float, default=0.1)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def inputs(rank: int):
    return synth.step_growth_sites(N_BEADS, FUNC, synth.BASE_SEED + rank)


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


def cpu_baseline(budget_s: float) -> dict:
    """The oracle as it stands, single-threaded on this host, on a bounded
    sample of the same workload: MD steps (with the reaction every Theta
    steps) of the full 1M-bead system until the budget is spent."""
    import oracle as orc
    inp = inputs(0)
    sch = scheme()
    o = orc.System(inp.x, inp.v, inp.type, inp.state, cap=FUNC)
    md = orc.MDParams(L=(inp.L,) * 3, seed=synth.BASE_SEED)
    rx = orc.Reaction(**sch)
    t0 = time.perf_counter()
    steps = 0
    while True:
        orc.run(o, md, rx, 1)
        steps += 1
        el = time.perf_counter() - t0
        if el > budget_s or steps >= 10 * THETA:
            break
    return {"value": inp.n * steps / el, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{steps} MD steps of the {inp.n}-bead step-growth workload "
                      f"(reaction every {THETA} steps), FP64, one thread, {el:.1f} s"}


ENSEMBLE = synth.WORKLOADS["ensemble_256"]


def ensemble(P, torch, steps: int, warmup: int = 3) -> dict:
    """Batched ensemble (256 replicas, sizes log-uniform in 1,024-65,536
    beads, step or chain growth, k log-uniform in [0.01, 1], own seeds)
    advanced together by one prx_batch, against the same replicas run one at
    a time through prx_run (each run to completion and synchronised before
    the next starts).  Both legs time the same number of MD steps per replica
    from the same state; wall clock around each leg.  A sample of replicas is
    then re-run alone from the initial inputs for the same total number of
    steps and compared bit for bit with the replicas that went through the
    batch (same accuracy: identical results)."""
    W = ENSEMBLE
    specs = synth.ensemble_specs(W["replicas"], W["n_lo"], W["n_hi"], W["k_lo"], W["k_hi"],
                                 synth.BASE_SEED)
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
    rs_batch = nrep * md_steps / t_batch
    rs_plain = nrep * md_steps / t_plain
    return {"workload": "ensemble_256", "replicas": nrep, "beads_total": beads,
            "md_steps_per_replica": md_steps, "unit": "replica-steps/s",
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


SERVING = synth.WORKLOADS["serving_stream"]


def serving(P, torch, arrivals: int, step_scale: float) -> dict:
    """Serving stream: Poisson arrivals (20 jobs/s) of step- or chain-growth
    jobs of 2,048-262,144 beads (log-uniform), replayed in real time through
    the continuous-batching server (admission by device memory, one shared
    batch), then the same trace one job at a time (FIFO, each job created,
    run alone and read back before the next).  Latency = arrival to result
    read-back.  The step counts are the workload's (5,000-50,000,
    log-uniform) times `step_scale`, and the arrival count is bounded, so
    that both legs finish in seconds.  Two jobs are re-run alone afterwards
    and compared bit for bit with their served results."""
    from paper_1409_7498_gb300.serve import Job, PolyrxBackend, Server, serve_serial, serve_trace
    W = SERVING
    lo, hi = max(10, int(W["steps_lo"] * step_scale)), max(10, int(W["steps_hi"] * step_scale))
    specs = synth.serving_trace(arrivals, W["rate"], W["n_lo"], W["n_hi"], lo, hi, W["k_lo"],
                                W["k_hi"], synth.BASE_SEED + 5)

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
    be = PolyrxBackend(P)
    srv = Server(be, budget, round_steps=100, theta=THETA)
    jb = jobs()
    res_b = serve_trace(srv, jb)
    be.shutdown()
    res_b.update(rounds=srv.rounds, max_resident_jobs=srv.max_members,
                 peak_admitted_bytes=srv.peak_in_use, budget_bytes=budget)
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
    offered = W["rate"] * float(np.mean(beads)) * float(np.mean([sp["nsteps"] for sp in specs]))
    return {"workload": "serving_stream", "arrivals": arrivals, "rate_per_s": W["rate"],
            "beads": [W["n_lo"], W["n_hi"]], "steps": [lo, hi],
            "scaled": f"steps x{step_scale} and {arrivals} of {W['arrivals']} arrivals, "
                      "so that both legs run in seconds",
            "offered_particle_steps_per_s": offered,
            "batched": res_b, "serial": res_s,
            "p99_speedup": res_s["p99_latency_s"] / res_b["p99_latency_s"],
            "throughput_ratio": res_b["replica_steps_per_s"] / res_s["replica_steps_per_s"],
            "identical": identical}


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle, timed on this host's cores; each bench
    step is one MD step of the same 1M-bead workload (the reaction every
    Theta steps)."""
    if rank != 0:
        return
    import oracle as orc
    inp = inputs(0)
    sch = scheme()
    o = orc.System(inp.x, inp.v, inp.type, inp.state, cap=FUNC)
    md = orc.MDParams(L=(inp.L,) * 3, seed=synth.BASE_SEED)
    rx = orc.Reaction(**sch)
    for _ in range(args.warmup):
        orc.run(o, md, rx, 1)
    t0 = time.perf_counter()
    done = 0
    budget = 150.0
    for _ in range(args.steps):
        orc.run(o, md, rx, 1)
        done += 1
        if time.perf_counter() - t0 > budget:
            break
    el = time.perf_counter() - t0
    v = inp.n * done / el
    line = {"impl": "reference", "metric": "particle-steps/s", "value": v,
            "unit": "particle-steps/s", "n_gpus": args.gpus, "steps": done, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / max(done, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "beads": inp.n, "f": FUNC, "k": K_RATE,
                       "theta": THETA, "sample": "one MD step per bench step"},
            "cpu_baseline": {"value": v, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
                             "sample": f"{done} MD steps of the {inp.n}-bead workload, one thread"},
            "e2e": {"value": v, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    from paper_1409_7498_gb300 import build as gbuild
    from paper_1409_7498_gb300 import polyrx as P

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

    inp = inputs(rank)
    sch = scheme()
    # the library's autotuner picks the Verlet skin for this workload (timed
    # on temporary copies of the system, outside the timed region)
    if args.skin > 0:
        skin, skin_ms = args.skin, {}
    else:
        skin, skin_ms = P.prx_autotune_skin(
            P.make_desc(inp.n, inp.L, adj_cap=FUNC, seed=synth.BASE_SEED + rank), inp.x, inp.v,
            inp.type, inp.state, P.make_reaction(**sch), steps=100, skins=SKINS)
    desc = P.make_desc(inp.n, inp.L, adj_cap=FUNC, seed=synth.BASE_SEED + rank, skin=skin)
    g = P.System(desc, inp.x, inp.v, inp.type, inp.state, stream=stream.cuda_stream)
    g.set_reaction(P.make_reaction(**sch))

    # warm-up (also melts the lattice)
    g.run(args.warmup * THETA)
    g.sync()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
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
        for q in range(args.steps):
            flush.fill_(q & 0xFF)  # L2 flush between timed bench steps (256 MB > 129 MB L2)
            starts[q].record(stream)
            g.run(THETA)
            ends[q].record(stream)
    torch.cuda.synchronize()
    if args.direct:
        P.prx_profile_end(g.h)
    wall = time.perf_counter() - wall0
    clocks = clk.stop()
    g.sync()
    st1 = g.stats()
    ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    ms_max, value = aggregate_throughput(ms, inp.n * THETA * args.steps, world,
                                         dist if world > 1 else None, dev)
    launches = int(st1["kernel_launches"] - st0["kernel_launches"])
    rebins = int(st1["rebins"] - st0["rebins"])

    # roofline of the dominant kernel: per-kernel CUDA-event times on the same
    # stream over a further stretch of the same run (kernels launched one by one)
    P.prx_profile_begin(g.h)
    g.run(10 * THETA)
    prof = P.prx_profile_end(g.h)
    top = max(prof, key=lambda r: r["total_ms"])
    step_rec = next(r for r in prof if r["name"] == "step")
    nb = g.observables()["bonds"]
    bpp = algorithmic_bytes_per_particle_step(2.0 * nb / inp.n)
    avg_ms = step_rec["total_ms"] / step_rec["launches"]
    achieved = inp.n * bpp / (avg_ms * 1e-3) / 1e9
    peak = json.load(open(PEAKS))["hbm_gbs"] if os.path.exists(PEAKS) else 6800.0
    traffic = None
    tr_path = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    if os.path.exists(tr_path):
        # DRAM bytes of one step-kernel launch from an ncu capture, valid only
        # while the step kernel's sources are unchanged since the capture
        tr = json.load(open(tr_path))
        h = hashlib.sha256()
        for rel in tr.get("digest_of", []):
            # "path" (the whole file) or "path::until::text" (the file up to
            # the first occurrence of text: the step kernel's part of it)
            path, _, until = rel.partition("::until::")
            with open(os.path.join(ROOT, path), "rb") as f:
                src = f.read()
            if until:
                cut = src.find(until.encode())
                src = src[:cut] if cut >= 0 else b""
            h.update(src)
        if tr.get("kernel_source_digest") == h.hexdigest():
            traffic = tr.get("bytes_per_launch")

    # end to end through the C ABI with host buffers
    e2e = None
    if rank == 0:
        pin = {k: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
               for k, a in (("x", inp.x), ("v", inp.v), ("t", inp.type), ("s", inp.state))}
        h2d = sum(a.nbytes for a in pin.values())
        torch.cuda.synchronize()
        e0 = time.perf_counter()
        ge = P.System(desc, pin["x"], pin["v"], pin["t"], pin["s"], stream=stream.cuda_stream)
        ge.set_reaction(P.make_reaction(**sch))
        d2h = 0
        ke = max(args.steps, 1)  # the same number of steps as the device-timed region
        for q in range(ke):
            ge.run(THETA)
            # the step's result (populations, bonds, energy) copied into a
            # pinned slot; the previous step's is read while this one runs
            ge.observables_begin(q % 2)
            if q:
                ob = ge.observables_end((q - 1) % 2)
            d2h += 8 * (2 + 8 * 16 + 4)
        ob = ge.observables_end((ke - 1) % 2)
        stt = ge.states()
        bd = ge.bonds()
        d2h += stt.nbytes + bd.nbytes
        ge.close()
        e_el = time.perf_counter() - e0
        e2e = {"value": inp.n * THETA * ke / e_el, "unit": "particle-steps/s",
               "h2d_bytes_per_step": int(h2d / ke), "d2h_bytes_per_step": int(d2h / ke),
               "steps": ke, "includes": "create (upload + binning), runs, per-step observables "
                                        "read-back (pipelined, one step behind), final states "
                                        "and bonds, destroy"}
        del ob

    ens = None
    if world == 1 and not args.no_ensemble:
        ens = ensemble(P, torch, args.ensemble_steps)
    srv = None
    if world == 1 and not args.no_serving:
        srv = serving(P, torch, args.serving_arrivals, args.serving_step_scale)

    if world > 1:
        dist.barrier()
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline(args.cpu_budget)
        line = {
            "metric": "particle-steps/s", "value": value, "unit": "particle-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 forces / f64 integration", "data": "synthetic",
            "config": {"workload": WORKLOAD, "beads": inp.n, "f": FUNC, "k": K_RATE,
                       "theta": THETA, "md_steps_per_bench_step": THETA, "box": inp.L,
                       "cells": list(st1["cells"]), "parallelism": f"replicas x{world}",
                       "l2": "flushed between bench steps (256 MB write)",
                       "rebins_in_timed_region": rebins, "wall_s": wall, "skin": skin,
                       "autotune_ms_per_step": {str(k): round(v, 4) for k, v in skin_ms.items()}},
            "clocks": clocks, "gpu_launches": launches,
            "roofline": {"bound": "hbm", "kernel": "step", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                         "algorithmic_bytes_per_particle_step": bpp,
                         "avg_launch_ms": avg_ms, "peak_source": "MEASURED_PEAKS.json hbm_gbs"
                         if os.path.exists(PEAKS) else "fallback",
                         "top_kernel": top["name"],
                         "kernel_ms": {r["name"]: round(r["total_ms"], 4) for r in prof},
                         "kernel_launches": {r["name"]: r["launches"] for r in prof}},
            "e2e": e2e, "cpu_baseline": cpu, "ensemble": ens, "serving": srv,
        }
        print(json.dumps(line), flush=True)
    g.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
