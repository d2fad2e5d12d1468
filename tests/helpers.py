"""Test helpers: build systems for both sides from the same seeded inputs.

The oracle and the CUDA binding never see each other; only these helpers
(test code) hold both.
"""
from __future__ import annotations

import numpy as np

import oracle as orc
import synth


def gpu():
    from paper_1409_7498_gb300 import build, polyrx
    build.build()
    return polyrx


def md_params(L, seed, **kw) -> orc.MDParams:
    return orc.MDParams(L=(L,) * 3, seed=seed, **kw)


def orc_reaction(scheme: dict) -> orc.Reaction:
    return orc.Reaction(**scheme)


def gpu_reaction(P, scheme: dict):
    return P.make_reaction(**scheme)


def oracle_system(x, v, types, states, cap, bonds=None) -> orc.System:
    s = orc.System(x, v, types, states, cap=cap)
    if bonds is not None:
        for r in bonds:
            s.add_bond(int(r["a"]), int(r["t"]), int(r["style"]), int(r["step"]))
    return s


def bonds_of_oracle(s: orc.System) -> np.ndarray:
    from paper_1409_7498_gb300.polyrx import BOND_DTYPE
    b = s.bonds()
    out = np.zeros(len(b), BOND_DTYPE)
    if len(b):
        out["step"], out["a"], out["t"], out["style"] = b[:, 0], b[:, 1], b[:, 2], b[:, 3]
    return out


def gpu_system(P, L, x, v, types, states, *, cap=4, fp64=False, seed=synth.BASE_SEED, bonds=None,
               gamma=1.0, skin=-1.0, eps=1.0, force_cap=0.0, dt=0.005):
    desc = P.make_desc(len(types), L, adj_cap=cap, fp64=fp64, seed=seed, gamma=gamma, skin=skin,
                       wca_eps=eps, force_cap=force_cap, dt=dt)
    return P.System(desc, x, v, types, states, bonds=bonds)


def canonical(bonds: np.ndarray) -> np.ndarray:
    """Bonds as an (m, 4) int array (step, a, t, style) sorted canonically."""
    if len(bonds) == 0:
        return np.zeros((0, 4), np.int64)
    b = np.stack([bonds["step"].astype(np.int64), bonds["a"].astype(np.int64),
                  bonds["t"].astype(np.int64), bonds["style"].astype(np.int64)], axis=1)
    return b[np.lexsort((b[:, 2], b[:, 1], b[:, 0]))]


def force_errors(f_gpu: np.ndarray, f_ref: np.ndarray) -> dict:
    """c16 reading: max_i |df_i| / RMS_i |f_i|, plus the RMS relative error."""
    df = np.sqrt(((f_gpu - f_ref) ** 2).sum(1))
    rms = np.sqrt(((f_ref ** 2).sum(1)).mean())
    return dict(max_over_rms=float(df.max() / rms), rms_rel=float(np.sqrt((df ** 2).mean()) / rms))


def chain_ree2(x, bonds, types, states, L):
    """Squared end-to-end distances of the chains (initiator to active end),
    bond vectors summed under the minimum image."""
    n = len(types)
    adj = [[] for _ in range(n)]
    for a, t in bonds:
        adj[a].append(t)
        adj[t].append(a)
    out = []
    for s in np.nonzero(types == synth.TYPE_A)[0]:
        if not adj[s]:
            continue
        prev, cur, r, length = -1, s, np.zeros(3), 0
        while True:
            nxt = [q for q in adj[cur] if q != prev]
            if not nxt:
                break
            d = x[nxt[0]] - x[cur]
            r += d - L * np.round(d / L)
            prev, cur, length = cur, nxt[0], length + 1
        if length >= 3:
            out.append(float(r @ r))
    return out
