"""prx_react_noalloc: the reaction step for callers that cannot allocate
device memory themselves (a fixed memory budget handed out by a host
framework, an allocator hook that must not re-enter the allocator).

The caller owns every input and output buffer; the only scratch is a static
device array inside the library.  Through the C ABI, two calls in a row are
compared with prx_react_once on a library-owned system and with the oracle
(Table I steps 1-9, or the nearest-partner rule of Sec. IV.A) on the same
state: the same bonds, states, adjacency and Table I counts.  The reaction
step is integer and FP64-decision work, so the tolerance is zero.  The cases
cover both selection rules, certain (p = 1) and rare (p = 0.005) acceptance,
a valence limit below the scheme's (pairs refused with PRX_ECAPACITY) and a
bond buffer shorter than the bonds formed.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import oracle as orc
import synth
from helpers import canonical, gpu, gpu_reaction, gpu_system, md_params, oracle_system

pytestmark = pytest.mark.gpu

SEED, CAP = 2718, 4
STEPS = (10, 20)


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _inputs():
    # 3,600 difunctional B + 400 crosslinkers (f = 4), positions jittered by
    # a quarter spacing so that pair distances spread around r_react
    return synth.step_growth(3600, 400, 4, SEED, jitter=0.5)


class _DeviceState:
    """Caller-owned device buffers of one system (particle-id order)."""

    def __init__(self, torch, P, inp, bonds_cap):
        dev = torch.device("cuda")
        n = inp.n
        self.n = n
        self.torch = torch
        self.P = P
        self.pos = torch.tensor(inp.x, dtype=torch.float64, device=dev).contiguous()
        self.typ = torch.tensor(inp.type, dtype=torch.uint8, device=dev)
        self.st = torch.tensor(inp.state, dtype=torch.int8, device=dev)
        self.nadj = torch.zeros(n, dtype=torch.uint8, device=dev)
        self.adj = torch.zeros(n * CAP, dtype=torch.int32, device=dev)
        self.bonds_cap = bonds_cap
        self.bonds = torch.zeros(max(1, bonds_cap) * P.BOND_DTYPE.itemsize, dtype=torch.uint8,
                                 device=dev)
        self.nb = torch.zeros(1, dtype=torch.int32, device=dev)

    def react(self, rx, box, step):
        """One call; returns (status, trace, bonds written by this call)."""
        P = self.P
        stream = self.torch.cuda.current_stream().cuda_stream
        status, trace = P.prx_react_noalloc(rx, box, 0.005, SEED, step, self.n,
                                            self.pos.data_ptr(), self.typ.data_ptr(),
                                            self.st.data_ptr(), CAP, self.nadj.data_ptr(),
                                            self.adj.data_ptr(), self.bonds.data_ptr(),
                                            self.bonds_cap, self.nb.data_ptr(), stream,
                                            check=False)
        k = int(self.nb.item())
        b = self.bonds.cpu().numpy().view(P.BOND_DTYPE)[:k].copy()
        return status, trace, b

    def adjacency(self):
        """Sorted partner ids of every particle's row (style bit dropped)."""
        nadj = self.nadj.cpu().numpy().astype(np.int64)
        adj = (self.adj.cpu().numpy().view(np.uint32) & 0x7FFFFFFF).reshape(self.n, CAP)
        return nadj, [sorted(adj[i, :nadj[i]].tolist()) for i in range(self.n)]


def _oracle_adjacency(o):
    return o.nadj.astype(np.int64), [sorted(o.adj[i, :o.nadj[i]].tolist()) for i in range(o.n)]


def _oracle_react(o, md, scheme, step):
    """Oracle reaction step; its state is updated even when it reports a
    capacity limit.  Returns (status, trace)."""
    nb0 = o.nb
    try:
        tr = orc.react(o, md, orc.Reaction(**scheme), step=step, use_cells=True)
        status = orc.OK
    except orc.OracleError as e:
        status, tr = e.code, None
    return status, tr, nb0


@pytest.mark.parametrize("selection", [0, 1], ids=["random", "nearest"])
@pytest.mark.parametrize("k", [0.1, 20.0], ids=["p0.005", "p1"])
def test_noalloc_matches_react_once_and_oracle_twice(selection, k):
    torch = _torch()
    P = gpu()
    inp = _inputs()
    sch = synth.step_growth_scheme(4, k=k, selection=selection)
    rx = gpu_reaction(P, sch)
    assert inp.n <= P.PRX_NOALLOC_MAX_N

    # the existing entry point on a library-owned system
    with gpu_system(P, inp.L, inp.x, inp.v, inp.type, inp.state, cap=CAP, seed=SEED) as g:
        g.set_reaction(rx)
        ref_traces = [g.react_once(s) for s in STEPS]
        ref_bonds = canonical(g.bonds())
        ref_states = g.states()

    # the oracle on the same state
    o = oracle_system(inp.x, inp.v, inp.type, inp.state, CAP)
    md = md_params(inp.L, SEED)
    orc_traces = [_oracle_react(o, md, sch, s)[1] for s in STEPS]

    d = _DeviceState(torch, P, inp, bonds_cap=inp.n)
    got, traces = [], []
    for s in STEPS:
        status, tr, b = d.react(rx, inp.L, s)
        assert status == P.PRX_OK
        traces.append(tr)
        got.append(b)
    got = canonical(np.concatenate(got))

    assert traces == ref_traces == orc_traces
    assert np.array_equal(got, ref_bonds)
    ob = o.bonds()
    assert np.array_equal(got[:, :3], ob[:, :3])
    assert np.array_equal(d.st.cpu().numpy(), ref_states)
    assert np.array_equal(d.st.cpu().numpy(), o.state)
    nadj, rows = d.adjacency()
    onadj, orows = _oracle_adjacency(o)
    assert np.array_equal(nadj, onadj) and rows == orows
    if k > 1.0:
        assert len(got) > 100  # the case is not vacuous
    else:
        assert traces[0]["candidates"] > 1000


@pytest.mark.parametrize("selection", [0, 1], ids=["random", "nearest"])
def test_noalloc_valence_limit(selection):
    """Crosslinkers limited to one bond (below the scheme's f = 4): on the
    second call every pair of an already-bonded crosslinker is refused with
    PRX_ECAPACITY, forms no bond and leaves no hole in the output."""
    torch = _torch()
    P = gpu()
    inp = _inputs()
    sch = synth.step_growth_scheme(4, k=20.0, selection=selection)
    mv = list(sch["max_valence"])
    mv[synth.TYPE_A] = 1
    sch["max_valence"] = tuple(mv)
    rx = gpu_reaction(P, sch)
    o = oracle_system(inp.x, inp.v, inp.type, inp.state, CAP)
    md = md_params(inp.L, SEED)
    d = _DeviceState(torch, P, inp, bonds_cap=inp.n)
    statuses = []
    for s in STEPS:
        status, tr, b = d.react(rx, inp.L, s)
        ostatus, otr, nb0 = _oracle_react(o, md, sch, s)
        statuses.append(status)
        assert status == ostatus
        ob = o.bonds()
        ob = ob[ob[:, 0] == s]
        assert np.array_equal(canonical(b)[:, :3], ob[:, :3])
        assert len(b) == o.nb - nb0  # the count matches the bonds written
        if otr is not None:
            assert tr == otr
        assert np.array_equal(d.st.cpu().numpy(), o.state)
        nadj, rows = d.adjacency()
        onadj, orows = _oracle_adjacency(o)
        assert np.array_equal(nadj, onadj) and rows == orows
    assert statuses[0] == P.PRX_OK and statuses[1] == P.PRX_ECAPACITY


def test_noalloc_bond_buffer_shorter_than_bonds_formed():
    """bonds_cap below the bonds formed: PRX_ECAPACITY, the first bonds_cap
    bonds in ascending id of A applied and written, the rest not applied."""
    torch = _torch()
    P = gpu()
    inp = _inputs()
    sch = synth.step_growth_scheme(4, k=20.0)
    rx = gpu_reaction(P, sch)
    cap_b = 50
    o = orc.System(inp.x, inp.v, inp.type, inp.state, cap=CAP, bond_capacity=cap_b)
    md = md_params(inp.L, SEED)
    ostatus, otr, _ = _oracle_react(o, md, sch, 10)
    assert ostatus == orc.ECAPACITY
    d = _DeviceState(torch, P, inp, bonds_cap=cap_b)
    status, tr, b = d.react(rx, inp.L, 10)
    assert status == P.PRX_ECAPACITY
    assert len(b) == cap_b == o.nb
    assert np.array_equal(canonical(b)[:, :3], o.bonds()[:, :3])
    assert np.array_equal(d.st.cpu().numpy(), o.state)
    nadj, rows = d.adjacency()
    onadj, orows = _oracle_adjacency(o)
    assert np.array_equal(nadj, onadj) and rows == orows


def test_noalloc_rejects_bad_arguments():
    torch = _torch()
    P = gpu()
    nb = torch.zeros(1, dtype=torch.int32, device="cuda")
    rx = gpu_reaction(P, synth.step_growth_scheme(4, k=0.1))
    with pytest.raises(P.PolyrxError) as e:
        P.prx_react_noalloc(rx, 50.0, 0.005, 1, 10, P.PRX_NOALLOC_MAX_N + 1, 0, 0, 0, 4, 0, 0, 0,
                            0, 0, None)
    assert e.value.code == P.PRX_ECAPACITY
    bad = gpu_reaction(P, synth.step_growth_scheme(4, k=0.1, selection=7))
    with pytest.raises(P.PolyrxError) as e:
        P.prx_react_noalloc(bad, 50.0, 0.005, 1, 10, 0, 0, 0, 0, 4, 0, 0, 0, 0, nb.data_ptr(),
                            None)
    assert e.value.code == P.PRX_EINVAL
