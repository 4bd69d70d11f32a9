"""Pins of the FIRE oracle (Bitzek et al. 2006; Sec. 3.3.1 minimisers).

Each test checks the oracle against something other than its own code: the
velocity-Verlet NVE oracle (FIRE's MD step is one velocity-Verlet step), a
closed-form first step of a head-on disk pair, the published time-step
schedule, the freeze rule once the power vanishes, rotation invariance,
convergence of a disk packing, and the shape of the paper's averaged
packing-energy curve (Sec. 4.2, Fig. 3(b))."""
import numpy as np
import pytest

import oracle as O
import workloads as W

FP = O.FIRE_DEFAULTS


def _disks(N, L, seed, overlap=True):
    rng = np.random.Generator(np.random.PCG64(seed))
    r = np.zeros((N, 3))
    r[:, :2] = rng.uniform(0.0, L, size=(N, 2))
    diam = np.where(np.arange(N) < N // 2, 1.4, 1.0)
    return r, diam


def test_fire_step_is_velocity_verlet_then_mixing():
    # one FIRE step from rest = one unit-mass velocity-Verlet step (positions
    # identical), after which the velocity changes only along F by the
    # published mixing: v_fire = (1 - a) v_md + a |v_md| F/|F|
    r, diam = _disks(60, 7.0, 3)
    a = FP["alpha_start"]
    x, v, E, dts, st = O.fire(r, 7.0, "soft", nsteps=1, dim=2, diam=diam)
    xn, vn, PE, KE = O.nve(r, np.zeros_like(r), 7.0, "soft", dt=FP["dt_start"], nsteps=1, dim=2, diam=diam, mass=1.0)
    # (the NVE oracle wraps positions into the box, FIRE keeps them unwrapped)
    dx = x[:, :2] - xn[:, :2]
    np.testing.assert_allclose(dx - 7.0 * np.round(dx / 7.0), 0.0, rtol=0, atol=1e-13)
    _, F, _ = O.soft(xn, diam, 7.0, dim=2)
    F = F[:, :2].ravel()
    vmd = vn[:, :2].ravel()
    assert float(F @ vmd) > 0.0     # the power is positive: no freeze
    d = v[:, :2].ravel() - (1.0 - a) * vmd
    Fh = F / np.linalg.norm(F)
    np.testing.assert_allclose(d, a * np.linalg.norm(vmd) * Fh, rtol=0, atol=1e-13)
    assert st == (FP["dt_start"], a, 1)


def test_fire_head_on_pair_first_step_closed_form():
    # unit disks 0.6 apart, eps = 1, alpha = 2: |F| = 1 - r, along the axis
    r = np.array([[0.0, 0.0, 0.0], [0.6, 0.0, 0.0]])
    x, v, E, dts, st = O.fire(r, 10.0, "soft", nsteps=1, dim=2, diam=np.ones(2))
    dt = FP["dt_start"]
    f0 = 0.4
    d1 = 0.6 + dt * dt * f0                  # each disk moves dt * (dt/2) f0
    f1 = 1.0 - d1
    v1 = 0.5 * dt * (f0 + f1)                # v is parallel to F: mixing keeps it
    np.testing.assert_allclose(x[:, 0], [-0.5 * dt * dt * f0, 0.6 + 0.5 * dt * dt * f0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(v[:, 0], [-v1, v1], rtol=0, atol=1e-15)
    np.testing.assert_allclose(E[:2], [0.5 * 0.4 ** 2, 0.5 * f1 ** 2], rtol=1e-14)


def test_fire_time_step_schedule():
    # while the power stays positive: dt_start for the first n_min steps,
    # then x f_inc per step up to dt_max (alpha x f_alpha alongside); once
    # the pair separates, F = P = 0 and every further step halves dt
    prm = dict(dt_start=0.02, dt_max=0.05)
    r = np.array([[0.0, 0.0, 0.0], [0.3, 0.0, 0.0]])
    x, v, E, dts, st = O.fire(r, 10.0, "soft", nsteps=200, dim=2, diam=np.ones(2), fire_params=prm)
    n_min, f_inc = FP["n_min"], FP["f_inc"]
    sep = int(np.argmax(E[1:] == 0.0))       # first step after which the disks no longer touch
    assert sep > 20
    want = [0.02 * min(f_inc ** max(k + 1 - n_min, 0), 2.5) for k in range(sep)]
    want = np.minimum(want, 0.05)
    got = dts[:sep]
    np.testing.assert_allclose(got, want, rtol=1e-12)
    # after separation: halving
    np.testing.assert_allclose(dts[sep:sep + 5], dts[sep - 1] * 0.5 ** np.arange(1, 6), rtol=1e-12)


def test_fire_freezes_once_separated():
    r = np.array([[0.0, 0.0, 0.0], [0.6, 0.0, 0.0]])
    x, v, E, dts, st = O.fire(r, 10.0, "soft", nsteps=40, dim=2, diam=np.ones(2))
    assert E[-1] == 0.0 and np.all(v == 0.0) and st[2] == 0
    assert x[1, 0] - x[0, 0] >= 1.0
    x2, _, _, _, _ = O.fire(r, 10.0, "soft", nsteps=60, dim=2, diam=np.ones(2))
    np.testing.assert_array_equal(x, x2)     # frozen: later steps move nothing


def test_fire_rotation_invariance():
    # a quarter turn maps the square periodic box onto itself
    L = 6.0
    r, diam = _disks(40, L, 5)
    rot = np.zeros_like(r)
    rot[:, 0] = np.mod(-r[:, 1], L)
    rot[:, 1] = r[:, 0]
    _, _, Ea, dta, _ = O.fire(r, L, "soft", nsteps=60, dim=2, diam=diam)
    _, _, Eb, dtb, _ = O.fire(rot, L, "soft", nsteps=60, dim=2, diam=diam)
    np.testing.assert_allclose(Ea, Eb, rtol=1e-9, atol=1e-14)
    np.testing.assert_allclose(dta, dtb, rtol=1e-12)


def test_fire_relaxes_a_packing():
    # the App. A system: 128 bidisperse disks at packing fraction 0.9,
    # 300 FIRE steps
    pk = W.packing_2d(N=128, D=1.4, phi=0.9, seed=0)
    L = W.packing_box(pk.N, pk.D, pk.phi)
    r = np.zeros((pk.N, 3))
    r[:, :2] = pk.s0 * L
    x, v, E, dts, st = O.fire(r, L, "soft", nsteps=300, dim=2, diam=pk.diam)
    assert E[-1] < 0.02 * E[0]
    _, F, _ = O.soft(x, pk.diam, L, dim=2)
    assert np.abs(F).max() < 0.05 * np.abs(O.soft(r, pk.diam, L, dim=2)[1]).max()


def _packing_energy_means(Ds, nseed):
    # ensemble mean of the minimised energy of the App. A system (128 disks,
    # half of diameter D and half of diameter 1, box at packing fraction
    # 0.9, 300 FIRE steps from uniform random positions)
    out = {}
    for D in Ds:
        Es = []
        for seed in range(nseed):
            pk = W.packing_2d(N=128, D=D, phi=0.9, seed=seed)
            L = W.packing_box(pk.N, pk.D, pk.phi)
            r = np.zeros((pk.N, 3))
            r[:, :2] = pk.s0 * L
            Es.append(O.fire(r, L, "soft", nsteps=300, dim=2, diam=pk.diam)[2][-1])
        out[D] = (float(np.mean(Es)), float(np.std(Es) / np.sqrt(nseed)))
    return out


def test_packing_energy_curve_has_the_papers_shape():
    # Sec. 4.2, Fig. 3(b): averaged over random starts, the minimised energy
    # is lowest for equal disks (D = 1), rises as the small disks shrink and
    # peaks at the maximally frustrated ratio D ~ 0.8, then falls again.  At
    # fixed packing fraction the energy is scale invariant, so a ratio D and
    # its reciprocal describe the same mixture: the peak shows again at
    # 1/0.8 = 1.25 with the same height.  Seeds are fixed; every margin below
    # is several standard errors of the ensemble means.
    m = _packing_energy_means([0.65, 0.8, 0.9, 1.0, 1.25], 24)
    E = {D: v[0] for D, v in m.items()}
    assert E[1.0] < 0.6 * min(E[0.65], E[0.8], E[0.9], E[1.25])
    assert E[0.8] > E[0.65] + 3 * (m[0.8][1] + m[0.65][1])
    assert E[0.8] > E[0.9] + 3 * (m[0.8][1] + m[0.9][1])
    assert abs(E[1.25] - E[0.8]) < 0.1 * E[0.8]
