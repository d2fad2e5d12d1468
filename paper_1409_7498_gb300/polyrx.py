"""Python binding of the polyrx C ABI (include/polyrx.h): argument marshalling only.

Every function keeps the C name and forwards to libpolyrx.so, which runs the
whole path in hand-written CUDA kernels.  There is no CPU fallback: if the
library is missing or fails to load, the import-time call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpolyrx.so")

PRX_OK = 0
PRX_EINVAL, PRX_ENOMEM, PRX_ECAPACITY, PRX_EOVERSTRETCH = -1, -2, -3, -4
PRX_ENONFINITE, PRX_ETIMEOUT, PRX_ECUDA, PRX_EIO = -5, -6, -7, -8
PRX_BOND_FENE, PRX_BOND_MIRROR_LJ = 0, 1
PRX_SELECT_RANDOM, PRX_SELECT_NEAREST = 0, 1
PRX_FORCE_FP32, PRX_FORCE_FP64 = 0, 1
PRX_MAX_TYPES, PRX_MAX_STATES, PRX_MAX_ADJ = 8, 16, 8
PRX_OBS_SLOTS = 4  # pinned slots of the pipelined observables


class PolyrxError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"polyrx status {code}: {msg}")
        self.code = code


class prx_system_desc(C.Structure):
    _fields_ = [("n", C.c_uint32), ("adj_cap", C.c_uint32), ("box", C.c_double * 3),
                ("dt", C.c_double), ("kT", C.c_double), ("gamma", C.c_double),
                ("mass", C.c_double), ("wca_eps", C.c_double), ("wca_sigma", C.c_double),
                ("fene_k", C.c_double), ("fene_r0", C.c_double), ("force_cap", C.c_double),
                ("skin", C.c_double), ("force_precision", C.c_int32), ("reserved", C.c_int32),
                ("seed", C.c_uint64)]


class prx_reaction_desc(C.Structure):
    _fields_ = [("type_mask_A", C.c_uint32), ("type_mask_T", C.c_uint32), ("a_lo", C.c_int32),
                ("a_hi", C.c_int32), ("t_lo", C.c_int32), ("t_hi", C.c_int32), ("dA", C.c_int32),
                ("dT", C.c_int32), ("k", C.c_double), ("r_react", C.c_double),
                ("theta", C.c_uint32), ("bond_style", C.c_int32), ("selection", C.c_int32),
                ("max_valence", C.c_uint8 * PRX_MAX_TYPES)]


class prx_bond(C.Structure):
    _fields_ = [("a", C.c_uint32), ("t", C.c_uint32), ("step", C.c_int64), ("style", C.c_uint32),
                ("reaction", C.c_uint32)]


BOND_DTYPE = np.dtype([("a", "<u4"), ("t", "<u4"), ("step", "<i8"), ("style", "<u4"),
                       ("reaction", "<u4")])


class prx_rx_trace(C.Structure):
    _fields_ = [("candidates", C.c_int64), ("retained", C.c_int64), ("a_winners", C.c_int64),
                ("formed", C.c_int64)]


class prx_observables(C.Structure):
    _fields_ = [("step", C.c_int64), ("bonds", C.c_int64),
                ("counts", (C.c_int64 * PRX_MAX_STATES) * PRX_MAX_TYPES),
                ("ke_half", C.c_double), ("momentum", C.c_double * 3)]


HISTORY_DTYPE = np.dtype([("step", "<i8"), ("bonds", "<i8"),
                          ("counts", "<i4", (PRX_MAX_TYPES, PRX_MAX_STATES))])


class prx_stats(C.Structure):
    _fields_ = [("steps", C.c_uint64), ("reactions", C.c_uint64), ("rebins", C.c_uint64),
                ("step_launches", C.c_uint64), ("kernel_launches", C.c_uint64),
                ("cells", C.c_uint32 * 3), ("cell_edge", C.c_double * 3)]


class prx_batch_stats(C.Structure):
    _fields_ = [("members", C.c_uint32), ("active", C.c_uint32), ("particles", C.c_uint64),
                ("steps", C.c_uint64), ("rebuilds", C.c_uint64), ("reactions", C.c_uint64),
                ("kernel_launches", C.c_uint64), ("graph_launches", C.c_uint64),
                ("max_slots", C.c_uint32), ("slots_used", C.c_uint32),
                ("mem_budget", C.c_uint64), ("bytes_admitted", C.c_uint64),
                ("epochs", C.c_uint64)]


class prx_launch_config(C.Structure):
    _fields_ = [("step_threads", C.c_uint32), ("step_blocks_per_sm", C.c_uint32),
                ("chunk_intervals", C.c_uint32), ("step_lanes", C.c_uint32)]


class prx_tune_choice(C.Structure):
    _fields_ = [("skin", C.c_double), ("launch", prx_launch_config), ("ms_per_step", C.c_double),
                ("stage", C.c_uint32), ("cached", C.c_uint32)]


class prx_class(C.Structure):
    _fields_ = [("type_mask", C.c_uint32), ("s_lo", C.c_int32), ("s_hi", C.c_int32)]


class prx_kernel_time(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_uint64), ("total_ms", C.c_double)]


_lib = None


def lib():
    """Loads libpolyrx.so (built by paper_1409_7498_gb300.build); raises when absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_1409_7498_gb300.build.build() first")
    L = C.CDLL(LIB_PATH)
    P, VP, U64, I = C.POINTER, C.c_void_p, C.c_uint64, C.c_int
    sig = {
        "prx_create": ([P(prx_system_desc), VP, VP, VP, VP, VP, U64, VP, P(VP)], I),
        "prx_destroy": ([VP], None),
        "prx_estimate_bytes": ([P(prx_system_desc), P(prx_reaction_desc), P(U64)], I),
        "prx_set_reaction": ([VP, P(prx_reaction_desc)], I),
        "prx_set_reactions": ([VP, P(prx_reaction_desc), C.c_uint32], I),
        "prx_run": ([VP, U64], I),
        "prx_sync": ([VP], I),
        "prx_react_once": ([VP, U64, P(prx_rx_trace)], I),
        "prx_compute_forces": ([VP, VP, P(C.c_double)], I),
        "prx_get_step": ([VP, P(U64)], I),
        "prx_get_positions": ([VP, VP], I),
        "prx_get_velocities": ([VP, VP], I),
        "prx_get_states": ([VP, VP], I),
        "prx_get_types": ([VP, VP], I),
        "prx_get_bonds": ([VP, VP, U64, P(U64)], I),
        "prx_get_observables": ([VP, P(prx_observables)], I),
        "prx_observables_begin": ([VP, I], I),
        "prx_observables_end": ([VP, I, P(prx_observables)], I),
        "prx_get_history": ([VP, VP, U64, P(U64)], I),
        "prx_history_begin": ([VP, I], I),
        "prx_history_end": ([VP, I, VP], I),
        "prx_get_stats": ([VP, P(prx_stats)], I),
        "prx_save": ([VP, C.c_char_p], I),
        "prx_load": ([C.c_char_p, VP, P(VP)], I),
        "prx_profile_begin": ([VP], I),
        "prx_profile_end": ([VP, P(prx_kernel_time), C.c_uint32, P(C.c_uint32)], I),
        "prx_react_noalloc": ([P(prx_reaction_desc), P(C.c_double), C.c_double, U64, U64,
                               C.c_uint32, VP, VP, VP, C.c_uint32, VP, VP, VP, C.c_uint32, VP,
                               VP, P(prx_rx_trace)], I),
        "prx_pair_histogram": ([VP, P(prx_class), P(prx_class), C.c_double, C.c_uint32, VP,
                                P(U64), P(U64)], I),
        "prx_autotune_skin": ([P(prx_system_desc), VP, VP, VP, VP, P(prx_reaction_desc),
                               C.c_uint32, P(C.c_double), C.c_uint32, P(C.c_double),
                               P(C.c_double)], I),
        "prx_set_launch_config": ([VP, P(prx_launch_config)], I),
        "prx_get_launch_config": ([VP, P(prx_launch_config)], I),
        "prx_autotune": ([P(prx_system_desc), VP, VP, VP, VP, P(prx_reaction_desc), C.c_uint32,
                          P(C.c_double), C.c_uint32, P(C.c_uint32), P(C.c_uint32),
                          P(C.c_uint32), C.c_uint32, P(C.c_uint32), C.c_uint32, C.c_char_p,
                          P(prx_tune_choice),
                          P(prx_tune_choice), C.c_uint32, P(C.c_uint32)], I),
        "prx_batch_create": ([C.c_uint32, U64, VP, P(VP)], I),
        "prx_batch_admit": ([VP, VP, U64, P(C.c_int32)], I),
        "prx_batch_step_epoch": ([VP, U64, P(U64)], I),
        "prx_batch_poll": ([VP, P(C.c_int32), C.c_int32, P(C.c_int32)], I),
        "prx_batch_destroy": ([VP], None),
        "prx_batch_add": ([VP, VP], I),
        "prx_batch_remove": ([VP, VP], I),
        "prx_batch_run": ([VP, U64], I),
        "prx_batch_sync": ([VP, P(C.c_int32)], I),
        "prx_batch_stats_get": ([VP, P(prx_batch_stats)], I),
        "prx_batch_last_error": ([VP], C.c_char_p),
        "prx_last_error": ([VP], C.c_char_p),
        "prx_status_string": ([I], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(rc: int, handle=None):
    if rc != PRX_OK:
        msg = lib().prx_last_error(handle)
        raise PolyrxError(rc, (msg or b"").decode() or lib().prx_status_string(rc).decode())


def make_desc(n, box, *, adj_cap=4, dt=0.005, kT=1.0, gamma=1.0, mass=1.0, wca_eps=1.0,
              wca_sigma=1.0, fene_k=30.0, fene_r0=1.5, force_cap=0.0, skin=-1.0, fp64=False,
              seed=14097498) -> prx_system_desc:
    b = (box,) * 3 if np.isscalar(box) else tuple(box)
    return prx_system_desc(int(n), int(adj_cap), (C.c_double * 3)(*map(float, b)), dt, kT, gamma,
                           mass, wca_eps, wca_sigma, fene_k, fene_r0, force_cap, skin,
                           PRX_FORCE_FP64 if fp64 else PRX_FORCE_FP32, 0,
                           int(seed) & 0xFFFFFFFFFFFFFFFF)


def make_reaction(mask_A, mask_T, a_lo, a_hi, t_lo, t_hi, dA, dT, k, theta=10, r_react=1.1,
                  bond_style=PRX_BOND_FENE, max_valence=(8,) * 8,
                  selection=PRX_SELECT_RANDOM) -> prx_reaction_desc:
    mv = list(max_valence) + [0] * (8 - len(max_valence))
    return prx_reaction_desc(mask_A, mask_T, a_lo, a_hi, t_lo, t_hi, dA, dT, float(k),
                             float(r_react), int(theta), int(bond_style), int(selection),
                             (C.c_uint8 * 8)(*mv[:8]))


# ---- the C entry points -----------------------------------------------------

def prx_create(desc: prx_system_desc, pos, vel, type_, state, bonds=None, stream=None):
    n = desc.n
    pos = np.ascontiguousarray(pos, np.float64).reshape(n, 3)
    vel = None if vel is None else np.ascontiguousarray(vel, np.float64).reshape(n, 3)
    type_ = np.ascontiguousarray(type_, np.uint8)
    state = np.ascontiguousarray(state, np.int8)
    nb = 0
    if bonds is not None and len(bonds):
        bonds = np.ascontiguousarray(bonds, BOND_DTYPE)
        nb = len(bonds)
    else:
        bonds = None
    out = C.c_void_p()
    rc = lib().prx_create(C.byref(desc), _ptr(pos), _ptr(vel), _ptr(type_), _ptr(state),
                          _ptr(bonds), nb, C.c_void_p(stream) if stream else None, C.byref(out))
    _check(rc, None)
    return out


def prx_destroy(h):
    lib().prx_destroy(h)


def prx_estimate_bytes(desc: prx_system_desc, rx: prx_reaction_desc | None = None) -> int:
    b = C.c_uint64()
    _check(lib().prx_estimate_bytes(C.byref(desc), C.byref(rx) if rx is not None else None,
                                    C.byref(b)))
    return b.value


def prx_set_reaction(h, rx):
    _check(lib().prx_set_reaction(h, C.byref(rx) if rx is not None else None), h)


def prx_set_reactions(h, rxs):
    """Sets the concurrent reactions `rxs` (a sequence of prx_reaction_desc;
    empty clears the scheme)."""
    arr = (prx_reaction_desc * max(1, len(rxs)))(*rxs)
    _check(lib().prx_set_reactions(h, arr, len(rxs)), h)


def prx_run(h, nsteps: int):
    _check(lib().prx_run(h, int(nsteps)), h)


def prx_sync(h):
    _check(lib().prx_sync(h), h)


def prx_react_once(h, step: int) -> dict:
    t = prx_rx_trace()
    _check(lib().prx_react_once(h, int(step), C.byref(t)), h)
    return dict(candidates=t.candidates, retained=t.retained, a_winners=t.a_winners,
                formed=t.formed)


def prx_compute_forces(h, n: int):
    f = np.zeros((n, 3), np.float64)
    e = C.c_double()
    _check(lib().prx_compute_forces(h, _ptr(f), C.byref(e)), h)
    return f, e.value


def prx_get_step(h) -> int:
    s = C.c_uint64()
    _check(lib().prx_get_step(h, C.byref(s)), h)
    return s.value


def prx_get_positions(h, n: int):
    out = np.zeros((n, 3), np.float64)
    _check(lib().prx_get_positions(h, _ptr(out)), h)
    return out


def prx_get_velocities(h, n: int):
    out = np.zeros((n, 3), np.float64)
    _check(lib().prx_get_velocities(h, _ptr(out)), h)
    return out


def prx_get_states(h, n: int):
    out = np.zeros(n, np.int8)
    _check(lib().prx_get_states(h, _ptr(out)), h)
    return out


def prx_get_types(h, n: int):
    out = np.zeros(n, np.uint8)
    _check(lib().prx_get_types(h, _ptr(out)), h)
    return out


def prx_get_bonds(h):
    n = C.c_uint64()
    rc = lib().prx_get_bonds(h, None, 0, C.byref(n))
    if rc not in (PRX_OK, PRX_ECAPACITY):
        _check(rc, h)
    out = np.zeros(n.value, BOND_DTYPE)
    _check(lib().prx_get_bonds(h, _ptr(out), n.value, C.byref(n)), h)
    return out


def prx_observables_begin(h, slot: int):
    _check(lib().prx_observables_begin(h, int(slot)), h)


def prx_observables_end(h, slot: int) -> dict:
    o = prx_observables()
    _check(lib().prx_observables_end(h, int(slot), C.byref(o)), h)
    return _obs_dict(o)


def prx_get_observables(h) -> dict:
    o = prx_observables()
    _check(lib().prx_get_observables(h, C.byref(o)), h)
    return _obs_dict(o)


def _obs_dict(o) -> dict:
    return dict(step=o.step, bonds=o.bonds,
                counts=np.ctypeslib.as_array(o.counts).astype(np.int64),
                ke_half=o.ke_half, momentum=np.ctypeslib.as_array(o.momentum).copy())


def prx_get_history(h, cap: int = 1 << 20):
    n = C.c_uint64()
    _check(lib().prx_get_history(h, None, 0, C.byref(n)), h)
    out = np.zeros(cap, HISTORY_DTYPE)
    _check(lib().prx_get_history(h, _ptr(out), cap, C.byref(n)), h)
    return out[: n.value]


def prx_history_begin(h, slot: int):
    _check(lib().prx_history_begin(h, int(slot)), h)


def prx_history_end(h, slot: int):
    """The newest reaction record (step, bonds, counts) as a one-element array."""
    out = np.zeros(1, HISTORY_DTYPE)
    _check(lib().prx_history_end(h, int(slot), _ptr(out)), h)
    return out[0]


def prx_get_stats(h) -> dict:
    s = prx_stats()
    _check(lib().prx_get_stats(h, C.byref(s)), h)
    return dict(steps=s.steps, reactions=s.reactions, rebins=s.rebins,
                step_launches=s.step_launches, kernel_launches=s.kernel_launches,
                cells=tuple(s.cells), cell_edge=tuple(s.cell_edge))


def prx_save(h, path: str):
    _check(lib().prx_save(h, path.encode()), h)


def prx_load(path: str, stream=None):
    out = C.c_void_p()
    _check(lib().prx_load(path.encode(), C.c_void_p(stream) if stream else None, C.byref(out)),
           None)
    return out


def prx_profile_begin(h):
    _check(lib().prx_profile_begin(h), h)


def prx_profile_end(h) -> list:
    out = (prx_kernel_time * 64)()
    n = C.c_uint32()
    _check(lib().prx_profile_end(h, out, 64, C.byref(n)), h)
    return [dict(name=out[i].name.decode(), launches=out[i].launches, total_ms=out[i].total_ms)
            for i in range(min(n.value, 64))]


PRX_NOALLOC_MAX_N = 16384


def prx_react_noalloc(rx, box, dt, seed, step, n, d_pos, d_type, d_state, adj_cap, d_nadj, d_adj,
                      d_bonds_out, bonds_cap, d_nbonds_out, stream=None, check=True):
    """Reaction step on caller-owned device buffers (integer device
    addresses), allocating nothing; see prx_react_noalloc in polyrx.h.
    Returns the trace counts; with check=False, (status, trace) instead of
    raising on a non-zero status (the outputs are written either way)."""
    b = (C.c_double * 3)(*([float(box)] * 3 if np.isscalar(box) else [float(v) for v in box]))
    t = prx_rx_trace()
    rc = lib().prx_react_noalloc(C.byref(rx), b, float(dt), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                 int(step), int(n), C.c_void_p(d_pos), C.c_void_p(d_type),
                                 C.c_void_p(d_state), int(adj_cap), C.c_void_p(d_nadj),
                                 C.c_void_p(d_adj), C.c_void_p(d_bonds_out), int(bonds_cap),
                                 C.c_void_p(d_nbonds_out), C.c_void_p(stream) if stream else None,
                                 C.byref(t))
    tr = dict(candidates=t.candidates, retained=t.retained, a_winners=t.a_winners,
              formed=t.formed)
    if not check:
        return rc, tr
    if rc != PRX_OK:
        raise PolyrxError(rc, lib().prx_status_string(rc).decode())
    return tr


def prx_pair_histogram(h, a, b, r_max: float, nbins: int):
    """Pair-distance histogram between classes a and b, each (type_mask,
    state_lo, state_hi); returns (counts, n_a, n_b)."""
    counts = np.zeros(int(nbins), np.uint64)
    na, nb = C.c_uint64(), C.c_uint64()
    _check(lib().prx_pair_histogram(h, C.byref(prx_class(*a)), C.byref(prx_class(*b)),
                                    float(r_max), int(nbins), _ptr(counts), C.byref(na),
                                    C.byref(nb)), h)
    return counts.astype(np.int64), na.value, nb.value


def prx_autotune_skin(desc: prx_system_desc, pos, vel, type_, state, rx=None, steps: int = 100,
                      skins=(0.25, 0.3, 0.35, 0.4, 0.45, 0.5)):
    """Fastest skin among the candidates; returns (best, {skin: ms per step})."""
    n = desc.n
    pos = np.ascontiguousarray(pos, np.float64).reshape(n, 3)
    vel = None if vel is None else np.ascontiguousarray(vel, np.float64).reshape(n, 3)
    type_ = np.ascontiguousarray(type_, np.uint8)
    state = np.ascontiguousarray(state, np.int8)
    sk = (C.c_double * len(skins))(*map(float, skins))
    ms = (C.c_double * len(skins))()
    best = C.c_double()
    rc = lib().prx_autotune_skin(C.byref(desc), _ptr(pos), _ptr(vel), _ptr(type_), _ptr(state),
                                 C.byref(rx) if rx is not None else None, int(steps), sk,
                                 len(skins), C.byref(best), ms)
    _check(rc, None)
    return best.value, {float(skins[q]): ms[q] for q in range(len(skins))}


def _choice(c: prx_tune_choice) -> dict:
    return dict(skin=c.skin, step_threads=c.launch.step_threads,
                step_blocks_per_sm=c.launch.step_blocks_per_sm,
                chunk_intervals=c.launch.chunk_intervals, step_lanes=c.launch.step_lanes,
                ms_per_step=c.ms_per_step, stage=c.stage, cached=bool(c.cached))


def prx_set_launch_config(h, step_threads=0, step_blocks_per_sm=0, chunk_intervals=0,
                          step_lanes=0):
    cfg = prx_launch_config(int(step_threads), int(step_blocks_per_sm), int(chunk_intervals),
                            int(step_lanes))
    _check(lib().prx_set_launch_config(h, C.byref(cfg)), h)


def prx_get_launch_config(h) -> dict:
    cfg = prx_launch_config()
    _check(lib().prx_get_launch_config(h, C.byref(cfg)), h)
    return dict(step_threads=cfg.step_threads, step_blocks_per_sm=cfg.step_blocks_per_sm,
                chunk_intervals=cfg.chunk_intervals, step_lanes=cfg.step_lanes)


def prx_autotune(desc: prx_system_desc, pos, vel, type_, state, rx=None, steps: int = 100,
                 skins=(0.3, 0.35, 0.4, 0.45, 0.5), shapes=((128, 0), (256, 0), (512, 0)),
                 chunks=(1, 2, 4), cache_path=None):
    """The library's autotuner (skin, step-kernel shape as (threads, blocks
    per SM[, lanes per particle]), reaction intervals per graph replay).
    Returns (best, tried): dicts with skin, step_threads, step_blocks_per_sm,
    step_lanes, chunk_intervals, ms_per_step, stage and cached."""
    shapes = [tuple(sh) + (1,) * (3 - len(sh)) for sh in shapes]
    n = desc.n
    pos = np.ascontiguousarray(pos, np.float64).reshape(n, 3)
    vel = None if vel is None else np.ascontiguousarray(vel, np.float64).reshape(n, 3)
    type_ = np.ascontiguousarray(type_, np.uint8)
    state = np.ascontiguousarray(state, np.int8)
    sk = (C.c_double * max(1, len(skins)))(*skins)
    th = (C.c_uint32 * max(1, len(shapes)))(*[int(a) for a, _, _ in shapes])
    bp = (C.c_uint32 * max(1, len(shapes)))(*[int(b) for _, b, _ in shapes])
    ln = (C.c_uint32 * max(1, len(shapes)))(*[int(c) for _, _, c in shapes])
    ch = (C.c_uint32 * max(1, len(chunks)))(*chunks)
    cap = len(skins) + len(shapes) + len(chunks)
    tried = (prx_tune_choice * max(1, cap))()
    best = prx_tune_choice()
    nt = C.c_uint32()
    rc = lib().prx_autotune(C.byref(desc), _ptr(pos), _ptr(vel), _ptr(type_), _ptr(state),
                            C.byref(rx) if rx is not None else None, int(steps), sk, len(skins),
                            th, bp, ln, len(shapes), ch, len(chunks),
                            cache_path.encode() if cache_path else None, C.byref(best), tried,
                            cap, C.byref(nt))
    _check(rc, None)
    return _choice(best), [_choice(tried[q]) for q in range(min(nt.value, cap))]


def _bcheck(rc: int, b=None):
    if rc != PRX_OK:
        msg = lib().prx_batch_last_error(b)
        raise PolyrxError(rc, (msg or b"").decode() or lib().prx_status_string(rc).decode())


def prx_batch_create(max_slots: int = 0, mem_budget: int = 0, stream=None):
    h = C.c_void_p()
    _bcheck(lib().prx_batch_create(int(max_slots), int(mem_budget),
                                   C.c_void_p(stream) if stream else None, C.byref(h)))
    return h.value


def prx_batch_admit(b, h, nsteps: int):
    """The system's slot, or None when the batch refused it (PRX_ENOMEM)."""
    slot = C.c_int32(-1)
    rc = lib().prx_batch_admit(b, h, int(nsteps), C.byref(slot))
    if rc == PRX_ENOMEM:
        return None
    _bcheck(rc, b)
    return slot.value


def prx_batch_step_epoch(b, max_steps: int) -> int:
    run = C.c_uint64()
    _bcheck(lib().prx_batch_step_epoch(b, int(max_steps), C.byref(run)), b)
    return run.value


def prx_batch_poll(b, cap: int = 256) -> list:
    out = (C.c_int32 * max(1, cap))()
    n = C.c_int32()
    _bcheck(lib().prx_batch_poll(b, out, int(cap), C.byref(n)), b)
    return [out[i] for i in range(n.value)]


def prx_batch_destroy(b):
    lib().prx_batch_destroy(b)


def prx_batch_add(b, h):
    _bcheck(lib().prx_batch_add(b, h), b)


def prx_batch_remove(b, h):
    _bcheck(lib().prx_batch_remove(b, h), b)


def prx_batch_run(b, nsteps: int):
    _bcheck(lib().prx_batch_run(b, int(nsteps)), b)


def prx_batch_sync(b):
    """Waits for the batch; raises PolyrxError (with .member set) on a member's status."""
    failed = C.c_int32(-1)
    rc = lib().prx_batch_sync(b, C.byref(failed))
    if rc != PRX_OK:
        msg = lib().prx_batch_last_error(b)
        e = PolyrxError(rc, (msg or b"").decode() or lib().prx_status_string(rc).decode())
        e.member = failed.value
        raise e


def prx_batch_stats_get(b) -> dict:
    st = prx_batch_stats()
    _bcheck(lib().prx_batch_stats_get(b, C.byref(st)), b)
    return {k: getattr(st, k) for k, _ in prx_batch_stats._fields_}


class Batch:
    """Owning handle over one prx_batch.  Members are System objects; the
    batch keeps them alive while they are members."""

    def __init__(self, stream=None, max_slots: int = 0, mem_budget: int = 0):
        self.h = prx_batch_create(max_slots, mem_budget, stream)
        self.members = []
        self.admitted = {}  # slot -> System, until poll reports it

    def add(self, system):
        prx_batch_add(self.h, system.h)
        self.members.append(system)

    def admit(self, system, nsteps: int):
        """Admits `system` for exactly nsteps more steps; returns its slot, or
        None when no slot or memory is free."""
        slot = prx_batch_admit(self.h, system.h, nsteps)
        if slot is not None:
            self.admitted[slot] = system
        return slot

    def step_epoch(self, max_steps: int) -> int:
        return prx_batch_step_epoch(self.h, max_steps)

    def poll(self) -> list:
        """Slots of the admitted systems that finished since the last poll
        (they are back in standalone use)."""
        slots = prx_batch_poll(self.h)
        for q in slots:
            self.admitted.pop(q, None)
        return slots

    def remove(self, system):
        prx_batch_remove(self.h, system.h)
        self.members.remove(system)

    def run(self, nsteps):
        prx_batch_run(self.h, nsteps)

    def sync(self):
        prx_batch_sync(self.h)

    def stats(self):
        return prx_batch_stats_get(self.h)

    def close(self):
        if getattr(self, "h", None):
            prx_batch_destroy(self.h)
            self.h = None
            self.members = []
            self.admitted = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class System:
    """Owning handle over one prx_system (calls prx_destroy when closed)."""

    def __init__(self, desc: prx_system_desc, pos, vel, type_, state, bonds=None, stream=None,
                 _handle=None):
        self.n = desc.n
        self.desc = desc
        self.h = _handle if _handle is not None else prx_create(desc, pos, vel, type_, state,
                                                                bonds, stream)

    @classmethod
    def load(cls, path: str, stream=None):
        desc = prx_system_desc()
        with open(path, "rb") as f:
            f.read(8)  # magic
            C.memmove(C.byref(desc), f.read(C.sizeof(desc)), C.sizeof(desc))
        obj = cls.__new__(cls)
        obj.h = prx_load(path, stream)
        obj.desc = desc
        obj.n = desc.n
        return obj

    def close(self):
        if getattr(self, "h", None):
            prx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_reaction(self, rx):
        prx_set_reaction(self.h, rx)

    def set_reactions(self, rxs):
        prx_set_reactions(self.h, list(rxs))

    def set_launch_config(self, step_threads=0, step_blocks_per_sm=0, chunk_intervals=0,
                          step_lanes=0):
        prx_set_launch_config(self.h, step_threads, step_blocks_per_sm, chunk_intervals,
                              step_lanes)

    def launch_config(self) -> dict:
        return prx_get_launch_config(self.h)

    def run(self, nsteps):
        prx_run(self.h, nsteps)

    def sync(self):
        prx_sync(self.h)

    def react_once(self, step):
        return prx_react_once(self.h, step)

    def forces(self):
        return prx_compute_forces(self.h, self.n)

    def step(self):
        return prx_get_step(self.h)

    def positions(self):
        return prx_get_positions(self.h, self.n)

    def velocities(self):
        return prx_get_velocities(self.h, self.n)

    def states(self):
        return prx_get_states(self.h, self.n)

    def types(self):
        return prx_get_types(self.h, self.n)

    def bonds(self):
        return prx_get_bonds(self.h)

    def observables(self):
        return prx_get_observables(self.h)

    def observables_begin(self, slot: int):
        """Enqueues the observables into pinned slot `slot` (no wait)."""
        prx_observables_begin(self.h, slot)

    def observables_end(self, slot: int) -> dict:
        """Waits for slot `slot` and returns its observables."""
        return prx_observables_end(self.h, slot)

    def history(self):
        return prx_get_history(self.h)

    def history_begin(self, slot: int):
        """Enqueues the copy of the newest reaction record into pinned slot `slot`."""
        prx_history_begin(self.h, slot)

    def history_end(self, slot: int):
        """Waits for slot `slot`; returns the newest reaction record."""
        return prx_history_end(self.h, slot)

    def stats(self):
        return prx_get_stats(self.h)

    def save(self, path):
        prx_save(self.h, path)

    def pair_histogram(self, a, b, r_max, nbins):
        return prx_pair_histogram(self.h, a, b, r_max, nbins)
