"""prx_react_noalloc: the reaction step for callers that cannot allocate
device memory themselves (a fixed memory budget handed out by a host
framework, an allocator hook that must not re-enter the allocator).

The caller owns every input and output buffer; the only scratch is a static
device array inside the library.  This checks, through the C ABI, that two
calls in a row give exactly what prx_react_once gives on the same state: the
same bonds, states and Table I counts (the reaction step is bit-exact, so the
tolerance is zero).
"""
import numpy as np
import pytest

import synth
from helpers import canonical, gpu, gpu_reaction, gpu_system

pytestmark = pytest.mark.gpu


def test_noalloc_matches_react_once_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P = gpu()
    seed, cap = 2718, 4
    inp = synth.step_growth(3600, 400, 4, seed, jitter=0.5)
    sch = synth.step_growth_scheme(4, k=20.0)  # p = 1: every candidate is retained
    rx = gpu_reaction(P, sch)
    n = inp.n
    assert n <= P.PRX_NOALLOC_MAX_N

    # the existing entry point on a library-owned system
    with gpu_system(P, inp.L, inp.x, inp.v, inp.type, inp.state, cap=cap, seed=seed) as g:
        g.set_reaction(rx)
        ref_traces = [g.react_once(10), g.react_once(20)]
        ref_bonds = canonical(g.bonds())
        ref_states = g.states()

    # the same two reaction steps on caller-owned device buffers
    dev = torch.device("cuda")
    pos = torch.tensor(inp.x, dtype=torch.float64, device=dev).contiguous()
    typ = torch.tensor(inp.type, dtype=torch.uint8, device=dev)
    st = torch.tensor(inp.state, dtype=torch.int8, device=dev)
    nadj = torch.zeros(n, dtype=torch.uint8, device=dev)
    adj = torch.zeros(n * cap, dtype=torch.int32, device=dev)
    bonds_cap = n
    bonds = torch.zeros(bonds_cap * P.BOND_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    nb = torch.zeros(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    got_bonds, traces = [], []
    for step in (10, 20):
        traces.append(P.prx_react_noalloc(rx, inp.L, 0.005, seed, step, n, pos.data_ptr(),
                                          typ.data_ptr(), st.data_ptr(), cap, nadj.data_ptr(),
                                          adj.data_ptr(), bonds.data_ptr(), bonds_cap,
                                          nb.data_ptr(), stream))
        k = int(nb.item())
        got_bonds.append(bonds.cpu().numpy().view(P.BOND_DTYPE)[:k].copy())
    got = canonical(np.concatenate(got_bonds))

    assert traces == ref_traces
    assert len(ref_bonds) > 100
    assert np.array_equal(got, ref_bonds)
    assert np.array_equal(st.cpu().numpy(), ref_states)
    # adjacency rows hold the partner ids of every new bond
    deg = np.bincount(np.concatenate([got[:, 1], got[:, 2]]), minlength=n)
    assert np.array_equal(nadj.cpu().numpy().astype(np.int64), deg)


def test_noalloc_rejects_oversized_systems():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P = gpu()
    rx = gpu_reaction(P, synth.step_growth_scheme(4, k=0.1))
    with pytest.raises(P.PolyrxError) as e:
        P.prx_react_noalloc(rx, 50.0, 0.005, 1, 10, P.PRX_NOALLOC_MAX_N + 1, 0, 0, 0, 4, 0, 0, 0,
                            0, 0, None)
    assert e.value.code == P.PRX_ECAPACITY
