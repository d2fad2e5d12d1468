"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds no arithmetic of the method: it only places particles,
draws thermal velocities and assigns types and initial states.  Both the
oracle and the CUDA path receive its arrays unchanged.

Recipe (stated once here, used everywhere):
  * box: cubic, edge L = (N / rho)^(1/3) at rho = 0.85;
  * positions: the N particles occupy a random subset of the sites of a
    simple cubic lattice of m = ceil(N^(1/3)) sites per edge (spacing L/m,
    about 1.03-1.05 sigma at rho = 0.85), each displaced by a uniform jitter
    of +-jitter/2 lattice spacings, so no two particles start closer than
    about 0.95 sigma and no capped warm-up is needed;
    or (placement="uniform", the benchmark workloads' recipe) uniformly at
    random in the box, which needs the capped-force WCA warm-up before
    production (the warm-up runs in the library; this module only places);
  * velocities: Maxwell-Boltzmann at kT with the centre-of-mass velocity
    removed;
  * types: 0 = B (difunctional monomer / chain monomer M), 1 = A
    (crosslinker of functionality f, or chain initiator), assigned to a
    random permutation of the particles.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

TYPE_B = 0
TYPE_A = 1
TYPE_E = 2   # chain end unit E of an E-P_n-E chain (Sec. II.B)
TYPE_P = 3   # repeat unit P of an E-P_n-E chain (does not react)
TYPE_X6 = 4  # second crosslinker type (functionality 6) of the concurrent-reaction inputs
DENSITY = 0.85
BASE_SEED = 14097498


@dataclass
class Inputs:
    """One system's initial data, by particle id."""
    L: float
    x: np.ndarray       # (n, 3) float64
    v: np.ndarray       # (n, 3) float64
    type: np.ndarray    # (n,) uint8
    state: np.ndarray   # (n,) int8
    scheme: str         # "step" or "chain"
    f: int              # crosslinker functionality (step growth), 1 for chain growth
    seed: int

    @property
    def n(self) -> int:
        return len(self.type)


def box_edge(n: int, rho: float = DENSITY) -> float:
    return (n / rho) ** (1.0 / 3.0)


def lattice_positions(n: int, L: float, rng: np.random.Generator, jitter: float = 0.05):
    if n == 0:
        return np.zeros((0, 3))
    m = max(1, math.ceil(round(n ** (1.0 / 3.0), 9)))
    while m ** 3 < n:
        m += 1
    a = L / m
    sites = rng.choice(m ** 3, size=n, replace=False)
    ijk = np.stack([sites % m, (sites // m) % m, sites // (m * m)], axis=1).astype(np.float64)
    pos = (ijk + 0.5 + jitter * (rng.random((n, 3)) - 0.5)) * a
    pos = np.where(pos >= L, pos - L, pos)
    pos = np.where(pos < 0.0, pos + L, pos)
    return np.ascontiguousarray(pos)


def uniform_positions(n: int, L: float, rng: np.random.Generator):
    """Uniform random placement (the paper's first protocol step, App. A);
    such inputs need the capped-force warm-up before production."""
    return np.ascontiguousarray(rng.random((n, 3)) * L)


def maxwell_velocities(n: int, kT: float, mass: float, rng: np.random.Generator):
    if n == 0:
        return np.zeros((0, 3))
    v = rng.standard_normal((n, 3)) * math.sqrt(kT / mass)
    v -= v.mean(axis=0, keepdims=True)
    return np.ascontiguousarray(v)


def _place(n: int, L: float, rng: np.random.Generator, jitter: float, placement: str):
    if placement == "uniform":
        return uniform_positions(n, L, rng)
    if placement != "lattice":
        raise ValueError(f"unknown placement {placement!r}")
    return lattice_positions(n, L, rng, jitter)


def step_growth(n_B: int, n_A: int, f: int, seed: int, rho: float = DENSITY, kT: float = 1.0,
                jitter: float = 0.05, placement: str = "lattice") -> Inputs:
    """Difunctional B monomers (state 0) and A crosslinkers of functionality
    f (state f)."""
    rng = np.random.default_rng(seed)
    n = n_B + n_A
    L = box_edge(n, rho)
    x = _place(n, L, rng, jitter, placement)
    v = maxwell_velocities(n, kT, 1.0, rng)
    typ = np.full(n, TYPE_B, np.uint8)
    st = np.zeros(n, np.int8)
    a_ids = rng.permutation(n)[:n_A]
    typ[a_ids] = TYPE_A
    st[a_ids] = f
    return Inputs(L, x, v, typ, st, "step", f, seed)


def ep_chains(n_chains: int, n_rep: int, f: int, seed: int, rho: float = DENSITY,
              kT: float = 1.0, jitter: float = 0.05):
    """Step growth of Sec. II.B: E-P_n-E chains (n = n_rep repeat units,
    chain bonds FENE) and crosslinkers X of functionality f in the
    stoichiometric ratio f n_X = 2 n_chains (two end units per chain).

    Simple cubic lattice with the chain length along x: each x-run of
    n_rep + 2 consecutive sites is either one chain (bond length = the
    lattice spacing, 1.06 sigma at rho = 0.85) or n_rep + 2 crosslinkers;
    which runs hold chains is seeded.  Returns (Inputs, box edges, chain
    bonds): Inputs.L is the x edge only, the box is the 3-tuple; the bonds
    are an (m, 2) array (lower id first)."""
    rng = np.random.default_rng(seed)
    run = n_rep + 2
    n_x_runs = int(math.ceil(2 * n_chains / f / run))
    n_runs = n_chains + n_x_runs
    # lattice of (run * mx) x my x mz sites with mx * my * mz >= n_runs
    m = max(1, int(math.ceil((n_runs * run) ** (1.0 / 3.0) / run)))
    my = mz = max(1, int(math.ceil(math.sqrt(n_runs / m))))
    while m * my * mz < n_runs:
        my += 1
    n = n_runs * run
    a = (n / rho / (m * run * my * mz)) ** (1.0 / 3.0)
    dims = (m * run * a, my * a, mz * a)  # box edges (not cubic in general)
    runs = rng.permutation(m * my * mz)[:n_runs]
    is_chain = np.zeros(n_runs, bool)
    is_chain[rng.permutation(n_runs)[:n_chains]] = True
    x = np.zeros((n, 3))
    typ = np.full(n, TYPE_A, np.uint8)
    st = np.full(n, f, np.int8)
    bonds = []
    for r in range(n_runs):
        q = runs[r]
        ix, iy, iz = q % m, (q // m) % my, q // (m * my)
        for u in range(run):
            p = r * run + u
            x[p] = ((ix * run + u + 0.5) * a, (iy + 0.5) * a, (iz + 0.5) * a)
        if is_chain[r]:
            base = r * run
            typ[base:base + run] = TYPE_P
            typ[base] = typ[base + run - 1] = TYPE_E
            st[base:base + run] = 0
            bonds += [(base + u, base + u + 1) for u in range(run - 1)]
    x += jitter * a * (rng.random((n, 3)) - 0.5)
    box = np.array(dims)
    x = np.where(x >= box, x - box, x)
    x = np.where(x < 0.0, x + box, x)
    v = maxwell_velocities(n, kT, 1.0, rng)
    return (Inputs(dims[0], np.ascontiguousarray(x), v, typ, st, "ep", f, seed),
            dims, np.array(bonds, np.int64).reshape(-1, 2))


def ep_scheme(f: int, k: float, theta: int = 10, r_react: float = 1.1,
              bond_style: int = 0, selection: int = 0) -> dict:
    """Sec. II.B: X^s (s in 1..f) + E^0 -> bond, X to s - 1 (delta_A = -1),
    E to 1 (delta_T = +1).  Valences: X f, E 2 (chain bond + one X), P 2."""
    mv = [0] * 8
    mv[TYPE_A] = f
    mv[TYPE_E] = 2
    mv[TYPE_P] = 2
    return dict(mask_A=1 << TYPE_A, mask_T=1 << TYPE_E, a_lo=1, a_hi=f, t_lo=0, t_hi=0, dA=-1,
                dT=+1, k=k, theta=theta, r_react=r_react, bond_style=bond_style,
                max_valence=tuple(mv), selection=selection)


def step_growth_sites(n_total: int, f: int, seed: int, **kw) -> Inputs:
    """N beads at a 4:1 B:A reactive-site ratio: 2 n_B = 4 f n_A, so
    n_A = round(N / (1 + 2 f))."""
    n_A = int(round(n_total / (1 + 2 * f)))
    return step_growth(n_total - n_A, n_A, f, seed, **kw)


def chain_growth(n_M: int, n_init: int, seed: int, rho: float = DENSITY, kT: float = 1.0,
                 jitter: float = 0.05, placement: str = "lattice") -> Inputs:
    """Monomers M (type B, state 0) and initiators (type A, state 2 = P*)."""
    rng = np.random.default_rng(seed)
    n = n_M + n_init
    L = box_edge(n, rho)
    x = _place(n, L, rng, jitter, placement)
    v = maxwell_velocities(n, kT, 1.0, rng)
    typ = np.full(n, TYPE_B, np.uint8)
    st = np.zeros(n, np.int8)
    ids = rng.permutation(n)[:n_init]
    typ[ids] = TYPE_A
    st[ids] = 2
    return Inputs(L, x, v, typ, st, "chain", 1, seed)


def log_uniform_int(rng: np.random.Generator, lo: int, hi: int, size=None):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size)).astype(np.int64)


# ---------------------------------------------------------------------------
# Reaction schemes as plain parameter sets (no arithmetic).  Both the oracle
# and the CUDA library turn one of these into their own parameter struct.
# ---------------------------------------------------------------------------
def step_growth_scheme(f: int, k: float, theta: int = 10, r_react: float = 1.1,
                       bond_style: int = 0, selection: int = 0) -> dict:
    """Step growth, Sec. II.B, with difunctional single-bead targets:
    A crosslinkers start at state f and react while in states 1..f
    (delta_A = -1); B targets react while in states 0..1 (delta_T = +1), so a
    B forms at most two bonds and an A at most f."""
    mv = [0] * 8
    mv[TYPE_B] = 2
    mv[TYPE_A] = f
    return dict(mask_A=1 << TYPE_A, mask_T=1 << TYPE_B, a_lo=1, a_hi=f, t_lo=0, t_hi=1, dA=-1,
                dT=+1, k=k, theta=theta, r_react=r_react, bond_style=bond_style,
                max_valence=tuple(mv), selection=selection)


def chain_growth_scheme(k: float, theta: int = 10, r_react: float = 1.1,
                        bond_style: int = 0, selection: int = 0) -> dict:
    """Chain growth, Sec. II.A: states M = 0, P = 1, P* = 2.  The active end
    P* (an initiator of type A or a monomer of type B) binds a monomer M of
    type B; the old end becomes P (delta_A = -1) and the monomer becomes the
    new end P* (delta_T = +2)."""
    mv = [0] * 8
    mv[TYPE_B] = 2
    mv[TYPE_A] = 1
    return dict(mask_A=(1 << TYPE_A) | (1 << TYPE_B), mask_T=1 << TYPE_B, a_lo=2, a_hi=2, t_lo=0,
                t_hi=0, dA=-1, dT=+2, k=k, theta=theta, r_react=r_react, bond_style=bond_style,
                max_valence=tuple(mv), selection=selection)


def step_growth_mixed(n_B: int, n_A: int, n_X6: int, seed: int, **kw) -> Inputs:
    """Step growth with two crosslinker types: n_A of functionality 4 (type A,
    state 4) and n_X6 of functionality 6 (type X6, state 6), with difunctional
    B targets; the input of the concurrent-reaction scheme below."""
    inp = step_growth(n_B, n_A + n_X6, 4, seed, **kw)
    rng = np.random.default_rng(seed + 1)
    x6 = rng.permutation(np.flatnonzero(inp.type == TYPE_A))[:n_X6]
    inp.type[x6] = TYPE_X6
    inp.state[x6] = 6
    return inp


def concurrent_schemes(k_first: float, k_later: float, k_x6: float, theta: int = 10,
                       r_react: float = 1.1, r_react_x6: float = 1.05) -> list:
    """Three concurrent reactions on the same B targets (a substitution
    effect and a second crosslinker type): a 4-functional crosslinker's first
    bond at k_first, its later bonds at k_later, and the 6-functional
    crosslinker's bonds at k_x6 with its own cutoff."""
    mv = [0] * 8
    mv[TYPE_B], mv[TYPE_A], mv[TYPE_X6] = 2, 4, 6
    base = dict(mask_T=1 << TYPE_B, t_lo=0, t_hi=1, dA=-1, dT=+1, theta=theta, bond_style=0,
                max_valence=tuple(mv), selection=0)
    return [dict(base, mask_A=1 << TYPE_A, a_lo=4, a_hi=4, k=k_first, r_react=r_react),
            dict(base, mask_A=1 << TYPE_A, a_lo=1, a_hi=3, k=k_later, r_react=r_react),
            dict(base, mask_A=1 << TYPE_X6, a_lo=1, a_hi=6, k=k_x6, r_react=r_react_x6)]


CHAIN_PHI0 = 328 / 33_096  # initiator fraction of the chain-growth workload


def ensemble_specs(replicas: int, n_lo: int, n_hi: int, k_lo: float, k_hi: float,
                   seed: int) -> list:
    """Replicas of the batched-ensemble workload: size and rate log-uniform,
    step growth (f = 4) or chain growth with equal odds, one seed each."""
    rng = np.random.default_rng(seed)
    n = log_uniform_int(rng, n_lo, n_hi, replicas)
    k = np.exp(rng.uniform(math.log(k_lo), math.log(k_hi), replicas))
    kind = rng.integers(0, 2, replicas)
    return [dict(kind="step" if kind[r] == 0 else "chain", n=int(n[r]), k=float(k[r]),
                 seed=seed + 1 + r) for r in range(replicas)]


def replica(spec: dict, theta: int = 10):
    """(Inputs, scheme, adjacency capacity) of one ensemble replica."""
    if spec["kind"] == "step":
        return (step_growth_sites(spec["n"], 4, spec["seed"]),
                step_growth_scheme(4, spec["k"], theta), 4)
    n_init = max(1, int(round(CHAIN_PHI0 * spec["n"])))
    return (chain_growth(spec["n"] - n_init, n_init, spec["seed"]),
            chain_growth_scheme(spec["k"], theta), 2)


def serving_trace(arrivals: int, rate: float, n_lo: int, n_hi: int, steps_lo: int, steps_hi: int,
                  k_lo: float, k_hi: float, seed: int) -> list:
    """Jobs of the serving workload: Poisson arrivals (exponential gaps of
    mean 1/rate seconds), sizes and step counts log-uniform, step or chain
    growth with equal odds, rate k log-uniform, one seed each."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, arrivals))
    n = log_uniform_int(rng, n_lo, n_hi, arrivals)
    steps = log_uniform_int(rng, steps_lo, steps_hi, arrivals)
    k = np.exp(rng.uniform(math.log(k_lo), math.log(k_hi), arrivals))
    kind = rng.integers(0, 2, arrivals)
    return [dict(kind="step" if kind[r] == 0 else "chain", n=int(n[r]), k=float(k[r]),
                 seed=seed + 1 + r, arrival=float(t[r]), nsteps=int(steps[r]))
            for r in range(arrivals)]


# The five workloads, by size.  Physical parameters shared by all of them:
# sigma = eps = m = 1, kT = 1, gamma = 1, dt = 0.005, FENE k = 30, R0 = 1.5,
# r_react = 1.1, Theta = 10, rho = 0.85.
WORKLOADS = {
    "step_growth_1250_fp64": dict(n_B=1000, n_A=250, f=4, k=0.1, steps=10_000, fp64=True),
    "chain_growth_33096": dict(n_M=32_768, n_init=328, k=(0.01, 0.1, 1.0), steps=50_000),
    "step_growth_1m": dict(n_total=1_048_576, f=4, k=0.1, steps=20_000),
    "ensemble_256": dict(replicas=256, n_lo=1024, n_hi=65_536, k_lo=0.01, k_hi=1.0, steps=20_000),
    "serving_stream": dict(rate=20.0, n_lo=2048, n_hi=262_144, steps_lo=5000, steps_hi=50_000,
                           arrivals=512, k_lo=0.01, k_hi=1.0),
}
