"""polyrx oracle: plain FP64 CPU restatement of de Buyl & Nies (arXiv:1409.7498).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users of this package; the CUDA
library and its Python binding never import it, and it never imports them.

The arithmetic lives in ``oracle.c`` (compiled with ``-ffp-contract=off``);
this module only builds it, loads it and marshals numpy arrays.
``timing_omp.c`` includes ``oracle.c`` unchanged and adds an OpenMP driver
of the per-particle loops, used only to time the oracle on all host cores.  The rate
equations of Secs. II.A and II.B live in ``rate_equations.py``.

Citations name the paper's sections, equations and tables.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

OK, EINVAL, ENOMEM, ECAPACITY, EOVERSTRETCH, ENONFINITE = 0, -1, -2, -3, -4, -5
BOND_FENE, BOND_MIRROR_LJ = 0, 1
SELECT_RANDOM, SELECT_NEAREST = 0, 1
TAG_THERMO, TAG_ACCEPT, TAG_SEL_A, TAG_SEL_T = 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so beside it (gcc, no contraction)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))
    ):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(
        ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
         "-o", tmp, _SRC, "-lm"]
    )
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_OMP_SRC = os.path.join(_HERE, "timing_omp.c")
_OMP_LIB_PATH = os.path.join(_HERE, "liboracle_omp.so")


def build_omp(force: bool = False):
    """Compile timing_omp.c (oracle.c unchanged plus an OpenMP driver of the
    per-particle loops) into liboracle_omp.so; returns its path, or None when
    the host compiler has no OpenMP."""
    srcs = [_SRC, _OMP_SRC, os.path.join(_HERE, "oracle.h")]
    if not force and os.path.exists(_OMP_LIB_PATH) and os.path.getmtime(_OMP_LIB_PATH) >= max(
        os.path.getmtime(p) for p in srcs
    ):
        return _OMP_LIB_PATH
    tmp = _OMP_LIB_PATH + f".tmp{os.getpid()}"
    try:
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
             "-fopenmp", "-I", _HERE, "-o", tmp, _OMP_SRC, "-lm"],
            stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
    except (OSError, subprocess.CalledProcessError):
        return None
    os.replace(tmp, _OMP_LIB_PATH)
    return _OMP_LIB_PATH


class _MD(C.Structure):
    _fields_ = [
        ("L", C.c_double * 3), ("dt", C.c_double), ("kT", C.c_double), ("gamma", C.c_double),
        ("mass", C.c_double), ("eps", C.c_double), ("sigma", C.c_double), ("fene_k", C.c_double),
        ("fene_r0", C.c_double), ("force_cap", C.c_double), ("seed", C.c_uint64),
    ]


class _CLASS(C.Structure):
    _fields_ = [("type_mask", C.c_uint32), ("s_lo", C.c_int32), ("s_hi", C.c_int32)]


class _RX(C.Structure):
    _fields_ = [
        ("mask_A", C.c_uint32), ("mask_T", C.c_uint32), ("a_lo", C.c_int32), ("a_hi", C.c_int32),
        ("t_lo", C.c_int32), ("t_hi", C.c_int32), ("dA", C.c_int32), ("dT", C.c_int32),
        ("k", C.c_double), ("theta", C.c_int64), ("r_react", C.c_double),
        ("bond_style", C.c_int32), ("selection", C.c_int32), ("max_valence", C.c_uint8 * 8),
    ]


class _SYS(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("cap", C.c_int32), ("pad_", C.c_int32),
        ("x", C.c_void_p), ("v", C.c_void_p), ("type", C.c_void_p), ("state", C.c_void_p),
        ("nadj", C.c_void_p), ("adj", C.c_void_p), ("adj_style", C.c_void_p),
        ("nb", C.c_int64), ("nb_cap", C.c_int64), ("bond_a", C.c_void_p), ("bond_t", C.c_void_p),
        ("bond_step", C.c_void_p), ("bond_style", C.c_void_p), ("step", C.c_int64),
        ("bond_rx", C.c_void_p),
    ]


class _TRACE(C.Structure):
    _fields_ = [("candidates", C.c_int64), ("retained", C.c_int64), ("a_winners", C.c_int64),
                ("formed", C.c_int64)]


class _OBS(C.Structure):
    _fields_ = [("counts", (C.c_int64 * 16) * 8), ("bonds", C.c_int64), ("ke_half", C.c_double),
                ("epot", C.c_double), ("momentum", C.c_double * 3)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.POINTER
        _lib.orc_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
        _lib.orc_philox4x32_10.restype = None
        _lib.orc_u53.argtypes = [C.c_uint32, C.c_uint32]
        _lib.orc_u53.restype = C.c_double
        _lib.orc_u24.argtypes = [C.c_uint32]
        _lib.orc_u24.restype = C.c_double
        _lib.orc_forces.argtypes = [P(_SYS), P(_MD), C.c_int, C.c_void_p, P(C.c_double)]
        _lib.orc_step.argtypes = [P(_SYS), P(_MD), C.c_int, P(C.c_double)]
        _lib.orc_check_reaction.argtypes = [P(_RX)]
        _lib.orc_react.argtypes = [P(_SYS), P(_MD), P(_RX), C.c_int, C.c_int64, P(_TRACE)]
        _lib.orc_observables.argtypes = [P(_SYS), P(_MD), P(_OBS)]
        _lib.orc_run.argtypes = [P(_SYS), P(_MD), P(_RX), C.c_int64, C.c_int, P(_OBS), C.c_int64]
        _lib.orc_pair_histogram.argtypes = [P(_SYS), P(_MD), P(_CLASS), P(_CLASS), C.c_double,
                                            C.c_int32, P(C.c_int64), P(C.c_int64),
                                            P(C.c_int64)]
        _lib.orc_check_reactions.argtypes = [P(_RX), C.c_int]
        _lib.orc_react_set.argtypes = [P(_SYS), P(_MD), P(_RX), C.c_int, C.c_int, C.c_int64,
                                       P(_TRACE), P(C.c_int64)]
        _lib.orc_run_set.argtypes = [P(_SYS), P(_MD), P(_RX), C.c_int, C.c_int64, C.c_int]
    return _lib


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


def _check(rc: int, what: str):
    if rc != OK:
        raise OracleError(rc, what)


@dataclass
class MDParams:
    """MD parameters: Sec. II.C (WCA Eq. 15, FENE) plus the Langevin thermostat."""
    L: tuple
    dt: float = 0.005
    kT: float = 1.0
    gamma: float = 1.0
    mass: float = 1.0
    eps: float = 1.0
    sigma: float = 1.0
    fene_k: float = 30.0
    fene_r0: float = 1.5
    force_cap: float = 0.0
    seed: int = 14097498

    def _c(self) -> _MD:
        return _MD((C.c_double * 3)(*[float(v) for v in self.L]), self.dt, self.kT, self.gamma,
                   self.mass, self.eps, self.sigma, self.fene_k, self.fene_r0, self.force_cap,
                   int(self.seed) & 0xFFFFFFFFFFFFFFFF)


@dataclass
class Reaction:
    """Reaction scheme T^t + A^a -> T^(t+dT)-A^(a+dA), Eq. 2, with the type
    masks and state windows that select A and T (AR parameters, Sec. III)."""
    mask_A: int
    mask_T: int
    a_lo: int
    a_hi: int
    t_lo: int
    t_hi: int
    dA: int
    dT: int
    k: float
    theta: int = 10
    r_react: float = 1.1
    bond_style: int = BOND_FENE
    max_valence: tuple = (8,) * 8
    selection: int = 0  # SELECT_RANDOM (Table I) or SELECT_NEAREST (LAMMPS rule, Sec. IV.A)

    def _c(self) -> _RX:
        mv = list(self.max_valence) + [0] * (8 - len(self.max_valence))
        return _RX(self.mask_A, self.mask_T, self.a_lo, self.a_hi, self.t_lo, self.t_hi, self.dA,
                   self.dT, self.k, self.theta, self.r_react, self.bond_style, self.selection,
                   (C.c_uint8 * 8)(*mv[:8]))


@dataclass
class System:
    """Particle state by id: positions, velocities, types, states, adjacency
    and the append-only bond list (the FixedPairList of Sec. III.A)."""
    x: np.ndarray
    v: np.ndarray
    type: np.ndarray
    state: np.ndarray
    cap: int = 8
    bond_capacity: int = -1
    step: int = 0
    nadj: np.ndarray = field(default=None)
    adj: np.ndarray = field(default=None)
    adj_style: np.ndarray = field(default=None)
    nb: int = 0

    def __post_init__(self):
        n = len(self.type)
        self.x = np.ascontiguousarray(self.x, dtype=np.float64).reshape(n, 3).copy()
        self.v = np.ascontiguousarray(self.v, dtype=np.float64).reshape(n, 3).copy()
        self.type = np.ascontiguousarray(self.type, dtype=np.uint8).copy()
        self.state = np.ascontiguousarray(self.state, dtype=np.int8).copy()
        if self.nadj is None:
            self.nadj = np.zeros(n, np.uint8)
            self.adj = np.zeros((n, self.cap), np.uint32)
            self.adj_style = np.zeros((n, self.cap), np.uint8)
        if self.bond_capacity < 0:
            self.bond_capacity = max(1, (n * self.cap) // 2)
        self.bond_a = np.zeros(self.bond_capacity, np.uint32)
        self.bond_t = np.zeros(self.bond_capacity, np.uint32)
        self.bond_step = np.zeros(self.bond_capacity, np.int64)
        self.bond_style = np.zeros(self.bond_capacity, np.uint8)
        self.bond_rx = np.zeros(self.bond_capacity, np.uint8)

    @property
    def n(self) -> int:
        return len(self.type)

    def add_bond(self, a: int, t: int, style: int = BOND_FENE, step: int = 0):
        """Insert an initial bond (both adjacency rows and the bond list)."""
        for p, q in ((a, t), (t, a)):
            if self.nadj[p] >= self.cap:
                raise OracleError(ECAPACITY, "add_bond")
            self.adj[p, self.nadj[p]] = q
            self.adj_style[p, self.nadj[p]] = style
            self.nadj[p] += 1
        self.bond_a[self.nb], self.bond_t[self.nb] = a, t
        self.bond_step[self.nb], self.bond_style[self.nb] = step, style
        self.nb += 1

    def bonds(self) -> np.ndarray:
        """Bonds as rows (step, a, t, style) in canonical order."""
        b = np.stack([self.bond_step[: self.nb], self.bond_a[: self.nb].astype(np.int64),
                      self.bond_t[: self.nb].astype(np.int64),
                      self.bond_style[: self.nb].astype(np.int64)], axis=1)
        if len(b):
            b = b[np.lexsort((b[:, 2], b[:, 1], b[:, 0]))]
        return b

    def bond_reactions(self) -> np.ndarray:
        """Bonds as rows (step, a, t, reaction) in canonical order; reaction is
        the index in the scheme of react_set that formed the bond (0 for
        initial bonds and for the single-reaction step)."""
        b = np.stack([self.bond_step[: self.nb], self.bond_a[: self.nb].astype(np.int64),
                      self.bond_t[: self.nb].astype(np.int64),
                      self.bond_rx[: self.nb].astype(np.int64)], axis=1)
        if len(b):
            b = b[np.lexsort((b[:, 2], b[:, 1], b[:, 0]))]
        return b

    def _c(self) -> _SYS:
        def p(a):
            return a.ctypes.data_as(C.c_void_p)
        return _SYS(self.n, self.cap, 0, p(self.x), p(self.v), p(self.type), p(self.state),
                    p(self.nadj), p(self.adj), p(self.adj_style), self.nb, self.bond_capacity,
                    p(self.bond_a), p(self.bond_t), p(self.bond_step), p(self.bond_style), self.step,
                    p(self.bond_rx))

    def _sync_back(self, cs: _SYS):
        self.nb = int(cs.nb)
        self.step = int(cs.step)


def philox4x32_10(ctr, key):
    """Philox4x32-10 block function (Salmon et al., SC'11)."""
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def u53(hi: int, lo: int) -> float:
    return lib().orc_u53(hi, lo)


def u24(w: int) -> float:
    return lib().orc_u24(w)


def forces(sys: System, md: MDParams, use_cells: bool = False):
    """Conservative forces (WCA on all pairs + bond potentials), by id."""
    f = np.zeros((sys.n, 3), np.float64)
    e = C.c_double(0.0)
    cs = sys._c()
    _check(lib().orc_forces(C.byref(cs), C.byref(md._c()), int(use_cells),
                            f.ctypes.data_as(C.c_void_p), C.byref(e)), "forces")
    return f, e.value


def step(sys: System, md: MDParams, use_cells: bool = True) -> float:
    """One Langevin velocity-Verlet step; returns the full-step kinetic energy."""
    cs = sys._c()
    ke = C.c_double(0.0)
    rc = lib().orc_step(C.byref(cs), C.byref(md._c()), int(use_cells), C.byref(ke))
    sys._sync_back(cs)
    _check(rc, "step")
    return ke.value


def check_reaction(rx: Reaction) -> int:
    return lib().orc_check_reaction(C.byref(rx._c()))


def react(sys: System, md: MDParams, rx: Reaction, step: int, use_cells: bool = False):
    """Reaction step, Table I steps 1-9.  Returns the trace counts."""
    cs = sys._c()
    tr = _TRACE()
    rc = lib().orc_react(C.byref(cs), C.byref(md._c()), C.byref(rx._c()), int(use_cells),
                         int(step), C.byref(tr))
    sys._sync_back(cs)
    _check(rc, "react")
    return dict(candidates=tr.candidates, retained=tr.retained, a_winners=tr.a_winners,
                formed=tr.formed)


def _rx_array(rxs):
    arr = (_RX * max(1, len(rxs)))()
    for q, r in enumerate(rxs):
        arr[q] = r._c()
    return arr


def check_reactions(rxs) -> int:
    """Status of a set of concurrent reactions (0 when valid)."""
    return lib().orc_check_reactions(_rx_array(rxs), len(rxs))


def react_set(sys: System, md: MDParams, rxs, step: int, use_cells: bool = False):
    """Reaction step with several concurrent reactions (see orc_react_set).
    Returns (trace counts, final pairs per reaction)."""
    cs = sys._c()
    tr = _TRACE()
    per = (C.c_int64 * max(1, len(rxs)))()
    rc = lib().orc_react_set(C.byref(cs), C.byref(md._c()), _rx_array(rxs), len(rxs),
                             int(use_cells), int(step), C.byref(tr), per)
    sys._sync_back(cs)
    _check(rc, "react_set")
    return (dict(candidates=tr.candidates, retained=tr.retained, a_winners=tr.a_winners,
                 formed=tr.formed), [int(per[q]) for q in range(len(rxs))])


def run_set(sys: System, md: MDParams, rxs, nsteps: int, use_cells: bool = True):
    """nsteps MD steps with the concurrent reactions every Theta steps."""
    cs = sys._c()
    rc = lib().orc_run_set(C.byref(cs), C.byref(md._c()), _rx_array(rxs), len(rxs), int(nsteps),
                           int(use_cells))
    sys._sync_back(cs)
    _check(rc, "run_set")


def _obs_dict(o: _OBS) -> dict:
    return dict(counts=np.array([[o.counts[t][s] for s in range(16)] for t in range(8)],
                                dtype=np.int64),
                bonds=int(o.bonds), ke_half=o.ke_half, epot=o.epot,
                momentum=np.array(list(o.momentum)))


def observables(sys: System, md: MDParams) -> dict:
    cs = sys._c()
    o = _OBS()
    _check(lib().orc_observables(C.byref(cs), C.byref(md._c()), C.byref(o)), "observables")
    return _obs_dict(o)


def run(sys: System, md: MDParams, rx: Reaction | None, nsteps: int, use_cells: bool = True):
    """nsteps MD steps with the reaction every Theta steps; observables after each reaction."""
    nrx = (sys.step + nsteps) // rx.theta - sys.step // rx.theta if rx else 0
    obs = (_OBS * max(1, nrx))()
    cs = sys._c()
    rxc = C.byref(rx._c()) if rx else None
    rc = lib().orc_run(C.byref(cs), C.byref(md._c()), rxc, int(nsteps), int(use_cells), obs,
                       int(nrx))
    sys._sync_back(cs)
    _check(rc, "run")
    return [_obs_dict(obs[i]) for i in range(nrx)]


_omp = None


def omp_lib():
    """The OpenMP timing driver, or None when it cannot be built here."""
    global _omp
    if _omp is None:
        path = build_omp()
        if path is None:
            return None
        _omp = C.CDLL(path)
        _omp.orc_run_omp.argtypes = [C.POINTER(_SYS), C.POINTER(_MD), C.POINTER(_RX), C.c_int64,
                                     C.c_int]
        _omp.orc_omp_max_threads.restype = C.c_int
    return _omp


def run_omp(sys: System, md: MDParams, rx: Reaction | None, nsteps: int, threads: int = 0) -> int:
    """The MD steps and reactions of run(), with the per-particle force and
    integration loops on `threads` host threads (0: all); the same trajectory
    bit for bit.  Returns the thread count used."""
    L = omp_lib()
    if L is None:
        raise OracleError(EINVAL, "run_omp (no OpenMP compiler)")
    cs = sys._c()
    rxc = C.byref(rx._c()) if rx else None
    used = threads if threads > 0 else L.orc_omp_max_threads()
    rc = L.orc_run_omp(C.byref(cs), C.byref(md._c()), rxc, int(nsteps), int(threads))
    sys._sync_back(cs)
    _check(rc, "run_omp")
    return used


def pair_histogram(sys: System, md: MDParams, a: tuple, b: tuple, r_max: float, nbins: int):
    """Pair-distance histogram between class a and class b, each given as
    (type_mask, state_lo, state_hi); returns (counts, n_a, n_b)."""
    cs = sys._c()
    counts = (C.c_int64 * nbins)()
    na, nb = C.c_int64(), C.c_int64()
    rc = lib().orc_pair_histogram(C.byref(cs), C.byref(md._c()), C.byref(_CLASS(*a)),
                                  C.byref(_CLASS(*b)), float(r_max), int(nbins), counts,
                                  C.byref(na), C.byref(nb))
    _check(rc, "pair_histogram")
    return np.array(list(counts), dtype=np.int64), na.value, nb.value
