"""Thermoneutral bonding on the GPU (mirror LJ, Eq. 17; Sec. II): without a
thermostat (gamma = 0), forming mirror-LJ bonds at r <= r_react <= sigma_c
leaves the total energy on the same track as a run with no reaction, while
FENE bonds add their potential at the moment of reaction (about 17 eps per
bond formed inside the cutoff here)."""
import numpy as np
import pytest

import synth
from helpers import gpu, gpu_reaction, gpu_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return gpu()


def energy_track(P, style):
    inp = synth.step_growth(1600, 400, 4, 13)  # lattice start: no overlaps
    with gpu_system(P, inp.L, inp.x, inp.v, inp.type, inp.state, cap=4, seed=13, gamma=0.0,
                    fp64=True) as g:
        if style is not None:
            g.set_reaction(gpu_reaction(P, synth.step_growth_scheme(4, k=2.0, bond_style=style)))
        e = []
        for _ in range(40):
            g.run(10)
            e.append(g.observables()["ke_half"] + g.forces()[1])
        return np.array(e), (g.bonds().shape[0] if style is not None else 0)


def test_mirror_lj_bonds_are_thermoneutral(P):
    e_none, _ = energy_track(P, None)
    e_mlj, nb_mlj = energy_track(P, P.PRX_BOND_MIRROR_LJ)
    e_fene, nb_fene = energy_track(P, P.PRX_BOND_FENE)
    assert nb_mlj > 100 and nb_fene > 100
    drift_none = np.abs(e_none - e_none[0]).max()
    drift_mlj = np.abs(e_mlj - e_mlj[0]).max()
    gain_fene = e_fene[-1] - e_fene[0]
    # the no-reaction run fixes the scale of the integration error
    assert drift_mlj < 3 * drift_none + 1.0, (drift_mlj, drift_none)
    assert gain_fene > 10.0 * nb_fene * 0.5, (gain_fene, nb_fene)
