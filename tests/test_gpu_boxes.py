"""Non-cubic boxes on the GPU against the FP64 oracle.

Two cases the cubic workloads do not reach:
  * a box with unequal edges: the step kernel's general path (per-axis
    scales) instead of the unit-space path of cubic boxes;
  * a long thin box whose cell rows hold more particles than the list
    build's shared-memory buffer: the neighbour rows of a tile are staged in
    several chunks, and every tile takes several passes of its threads.
Bars as in test_gpu_parity: FP32 forces within 1e-5 (max_i |df_i| / RMS |f|
and RMS |df| / RMS |f|), FP64 forces within 1e-12.
"""
import numpy as np
import pytest

import oracle as orc
from helpers import force_errors, gpu

pytestmark = pytest.mark.gpu

SPACING = 0.85 ** (-1.0 / 3.0)  # simple cubic lattice at density 0.85


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return gpu()


def lattice_box(counts, seed, jitter=0.05):
    """Jittered simple cubic lattice of counts[0] x counts[1] x counts[2]
    sites filling the box exactly (seeded)."""
    L = tuple(c * SPACING for c in counts)
    g = np.stack(np.meshgrid(*[np.arange(c) for c in counts], indexing="ij"), -1).reshape(-1, 3)
    rng = np.random.default_rng(seed)
    x = (g + 0.5) * SPACING + rng.uniform(-jitter, jitter, g.shape)
    return L, np.ascontiguousarray(x, np.float64)


def melted_box(counts, seed, steps=100):
    L, x = lattice_box(counts, seed)
    n = len(x)
    o = orc.System(x, np.zeros((n, 3)), np.zeros(n, np.uint8), np.zeros(n, np.int8), cap=4)
    md = orc.MDParams(L=L, seed=seed)
    orc.run(o, md, None, steps)  # the oracle melts the lattice
    return L, o, md


def gpu_from(P, L, o, seed, fp64):
    desc = P.make_desc(o.n, L, adj_cap=4, fp64=fp64, seed=seed)
    return P.System(desc, o.x, o.v, o.type, o.state)


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("counts", [(19, 13, 10), (662, 5, 5)])
def test_forces_in_non_cubic_boxes(P, counts, fp64):
    # (662, 5, 5): 16,550 beads in a 699 x 5.3 x 5.3 box, 3 x 3 cells across,
    # ~1,840 beads per cell row: a tile's nine neighbour rows (~16,600
    # staged entries) exceed the staging buffer (at most ~10,000)
    L, o, md = melted_box(counts, 29)
    f_ref, e_ref = orc.forces(o, md, use_cells=True)
    with gpu_from(P, L, o, 29, fp64) as g:
        f, e = g.forces()
    err = force_errors(f, f_ref)
    if fp64:
        assert err["max_over_rms"] < 1e-12, err
        assert e == pytest.approx(e_ref, rel=1e-12)
    else:
        assert err["max_over_rms"] < 1e-5, err
        assert err["rms_rel"] < 1e-5, err
        assert e == pytest.approx(e_ref, rel=1e-5)


def test_run_with_rebuilds_in_a_long_box(P):
    """The FP32 trajectory stays on the oracle's (FP64, same random draws)
    as in the cubic runs, and rebuilds with chunked staging keep going."""
    L, o, md = melted_box((662, 5, 5), 31)
    with gpu_from(P, L, o, 31, False) as g:
        g.run(40)
        x = g.positions()
        # the same state at step 0 on the oracle (the melt advanced its step
        # counter, and the random draws are keyed by step)
        o2 = orc.System(o.x, o.v, o.type, o.state, cap=4)
        orc.run(o2, md, None, 40)
        d = x - o2.x
        for k in range(3):
            d[:, k] -= L[k] * np.round(d[:, k] / L[k])
        assert np.abs(d).max() < 1e-4, np.abs(d).max()
        g.run(400)
        g.sync()
        assert np.isfinite(g.positions()).all()
        assert g.stats()["rebins"] >= 5
