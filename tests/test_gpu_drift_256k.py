"""Configuration 1 (LJ, N = 256,000, FCC 4*40^3, density 0.84, T = 1,
r_c = 2.5 sigma shifted, skin 0.3, dt = 0.005): the FP32 velocity-Verlet
run's energy series against the FP64 oracle run from the same start over
the first 100 steps (Sec. 3.3.1), with the int32-row engine and the tile
engine."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import dev, status_word, to_dev

pytestmark = pytest.mark.gpu

NSTEPS = 100


@pytest.fixture(scope="module")
def P():
    import paper_1912_04232_b300 as P
    return P


@pytest.fixture(scope="module")
def reference():
    c = W.lj_large()
    _, _, PEo, KEo = O.nve(c.r, c.v, c.L, "lj", dt=c.dt, nsteps=NSTEPS)
    return c, PEo, KEo


@pytest.mark.parametrize("tiles", [False, True])
def test_energy_series_256k_tracks_oracle(P, reference, tiles):
    import torch
    c, PEo, KEo = reference
    s = P.md_space_periodic(3, [c.L] * 3)
    nl = P.NeighborList(s, c.N, c.r_cut, c.skin, 128, tiles=tiles)
    rd, vd = to_dev(c.r, torch.float32), to_dev(c.v, torch.float32)
    f = torch.zeros_like(rd)
    st = status_word()
    pot = P.lj_pot()
    nl.build(rd, st)
    P.md_energy_forces(s, pot, rd, nl.plan, f, None, st)
    PE = torch.zeros(NSTEPS, dtype=torch.float64, device=dev())
    KE = torch.zeros_like(PE)
    P.md_integrate_nve(s, pot, rd, vd, f, c.mass, c.dt, NSTEPS, nl.plan, PE, KE, True, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    assert nl.stats()[0] >= 5          # rebuilds inside the run
    E, Eo = (PE + KE).cpu().numpy(), PEo[1:] + KEo[1:]
    # pointwise, per particle
    assert np.abs(E - Eo).max() / c.N <= 1e-4
    # the drift of the FP32 run matches the FP64 run's
    drift, drift_o = np.abs(E - E[0]).max() / c.N, np.abs(Eo - Eo[0]).max() / c.N
    assert abs(drift - drift_o) <= 1e-4
