"""Pins of the Nose-Hoover chain oracle (Sec. 3.3.1; Martyna, Klein,
Tuckerman 1992; half-step sweep of Martyna, Tuckerman, Tobias, Klein 1996).

Each test checks the oracle against something other than its own code: the
velocity-Verlet NVE oracle it must reduce to as the thermostat masses grow,
the time reversibility and second order of the symmetric splitting (the
conserved extended energy H'), and equipartition at the target temperature."""
import numpy as np

import oracle as O
import workloads as W


def _lj216(seed=0):
    return W.lj_fluid("sc", 6, seed=seed, steps=10)


def test_nhc_reduces_to_nve_for_heavy_thermostats():
    # tau -> infinity: Q -> infinity, the chain stays at rest and the step is
    # plain velocity Verlet
    c = _lj216()
    x, v, PE, KE, H, th = O.nhc(c.r, c.v, c.L, "lj", dt=0.005, kT=1.0, tau=1e9, nsteps=50)
    xn, vn, PEn, KEn = O.nve(c.r, c.v, c.L, "lj", dt=0.005, nsteps=50)
    np.testing.assert_allclose(x, xn, rtol=0, atol=1e-9)
    np.testing.assert_allclose(v, vn, rtol=0, atol=1e-9)
    np.testing.assert_allclose(PE, PEn, rtol=1e-12)


def test_nhc_time_reversible():
    # forward n steps, flip particle and thermostat velocities, n steps back:
    # positions and the chain positions xi return, velocities return flipped
    c = _lj216(1)
    n = 60
    x, v, _, _, _, (xi, w) = O.nhc(c.r, c.v, c.L, "lj", dt=0.004, kT=1.5, nsteps=n)
    xb, vb, _, _, _, (xib, wb) = O.nhc(x, -v, c.L, "lj", dt=0.004, kT=1.5, nsteps=n, therm=(xi, -w))
    d = xb - O._pos(c.r)
    d -= c.L * np.round(d / c.L)
    assert np.abs(d).max() < 1e-9
    np.testing.assert_allclose(-vb, O._pos(c.v), rtol=0, atol=1e-9)
    np.testing.assert_allclose(xib, 0.0, atol=1e-9)
    np.testing.assert_allclose(wb, 0.0, atol=1e-9)


def test_nhc_extended_energy_is_second_order():
    # the largest deviation of H' over a fixed time shrinks ~4x when dt halves
    # (the thermostat time scale tau is held fixed)
    c = _lj216(2)
    dev = []
    for dt in (0.004, 0.002):
        n = int(round(0.8 / dt))
        _, _, _, _, H, _ = O.nhc(c.r, c.v, c.L, "lj", dt=dt, kT=1.5, tau=0.4, nsteps=n)
        dev.append(np.abs(H - H[0]).max())
    assert dev[0] / dev[1] > 3.0
    assert dev[0] / c.N < 2e-3


def test_nhc_equipartition():
    # the time-averaged kinetic energy approaches g kT / 2 (g = 3N)
    c = _lj216(3)
    kT = 1.2
    _, _, _, KE, _, _ = O.nhc(c.r, c.v, c.L, "lj", dt=0.005, kT=kT, tau=0.25, nsteps=12000)
    mean = KE[4000:].mean()
    assert abs(mean / (1.5 * c.N * kT) - 1.0) < 0.03
