"""Pins of the flocking oracle (Sec. 4.3 and its appendix): closed-form
pair and single-boid energies, gradients against central finite
differences (with the displacement stop-gradients of alignment and
cohesion), invariance under a quarter turn and translation, and the free
swimming of a lone boid."""
import numpy as np

import oracle as O

FP = O.FLOCK_DEFAULTS


def _rho(r, Rc, a=2.0):
    return (1.0 - r / Rc) ** a / a if r < Rc else 0.0


def test_pair_closed_forms():
    L = 200.0
    R = np.array([[10.0, 10.0], [30.0, 10.0]])
    # anti-aligned: (1 - N.N)^2 = 4; cohesion zero (each faces the other)
    E, gR, gth, (al, av, co, ob) = O.flock_grad(R, np.array([0.0, np.pi]), L)
    assert abs(al - FP["J_align"] * _rho(20.0, FP["R_align"]) * 4.0) < 1e-12
    assert abs(av - FP["J_avoid"] * _rho(20.0, FP["R_avoid"])) < 1e-12
    assert co == 0.0 and ob == 0.0
    # aligned, both facing +x: no alignment energy; boid 1 faces away from
    # its only neighbour: cohesion 1/2 J (1 - (-1))^2 = 2 J
    E, gR, gth, (al, av, co, ob) = O.flock_grad(R, np.array([0.0, 0.0]), L)
    assert al == 0.0
    assert abs(co - 2.0 * FP["J_cohesion"]) < 1e-12
    # across the periodic boundary: same pair, shifted
    R2 = np.array([[195.0, 10.0], [15.0, 10.0]])
    _, _, _, parts2 = O.flock_grad(R2, np.array([0.0, np.pi]), L)
    assert abs(parts2[0] - FP["J_align"] * _rho(20.0, FP["R_align"]) * 4.0) < 1e-12


def test_obstacle_closed_form():
    # boid at distance 5 from an obstacle of radius 10, facing it: w = N,
    # (1 + 1)^2 = 4; facing away: 0
    L = 200.0
    obs = [[50.0, 50.0, 10.0]]
    R = np.array([[45.0, 50.0]])
    _, _, _, (al, av, co, ob) = O.flock_grad(R, np.array([0.0]), L, obstacles=obs)
    assert abs(ob - FP["J_obstacle"] * _rho(5.0, 10.0) * 4.0) < 1e-12
    _, _, _, (al, av, co, ob) = O.flock_grad(R, np.array([np.pi]), L, obstacles=obs)
    assert abs(ob) < 1e-12


def _flock(N, L, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(0, L, size=(N, 2)), rng.uniform(-np.pi, np.pi, size=N)


def test_gradients_match_finite_differences():
    L = 150.0
    R, th = _flock(60, L, 1)
    obs = [[40.0, 60.0, 20.0], [100.0, 100.0, 15.0]]
    E, gR, gth, _ = O.flock_grad(R, th, L, obstacles=obs)
    h = 1e-6
    for i in range(0, 60, 7):
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (O.flock_grad(R, tp, L, obstacles=obs)[0] - O.flock_grad(R, tm, L, obstacles=obs)[0]) / (2 * h)
        assert abs(fd - gth[i]) < 1e-6 * max(1.0, abs(gth[i]))
        for k in range(2):
            Rp, Rm = R.copy(), R.copy()
            Rp[i, k] += h
            Rm[i, k] -= h
            # alignment and cohesion take no gradient through the positions
            ep = O.flock_grad(Rp, th, L, obstacles=obs)[3]
            em = O.flock_grad(Rm, th, L, obstacles=obs)[3]
            fd = ((ep[1] + ep[3]) - (em[1] + em[3])) / (2 * h)
            assert abs(fd - gR[i, k]) < 1e-6 * max(1.0, abs(gR[i, k]))


def test_quarter_turn_and_translation_invariance():
    L = 150.0
    R, th = _flock(80, L, 2)
    obs = np.array([[40.0, 60.0, 20.0]])
    E, _, _, parts = O.flock_grad(R, th, L, obstacles=obs)
    rot = np.stack([np.mod(-R[:, 1], L), R[:, 0]], axis=1)
    orot = np.array([[np.mod(-obs[0, 1], L), obs[0, 0], obs[0, 2]]])
    E2, _, _, parts2 = O.flock_grad(rot, th + np.pi / 2, L, obstacles=orot)
    np.testing.assert_allclose(parts2, parts, rtol=1e-10, atol=1e-12)
    sh = np.mod(R + np.array([17.3, -41.9]), L)
    osh = obs.copy()
    osh[0, :2] = np.mod(obs[0, :2] + np.array([17.3, -41.9]), L)
    E3, _, _, parts3 = O.flock_grad(sh, th, L, obstacles=osh)
    np.testing.assert_allclose(parts3, parts, rtol=1e-10, atol=1e-12)


def test_lone_boid_swims_straight():
    L = 500.0
    R0 = np.array([[100.0, 200.0]])
    th0 = np.array([0.7])
    R, th, E = O.flock_run(R0, th0, L, dt=0.25, nsteps=40)
    np.testing.assert_allclose(R[0], R0[0] + 0.25 * 40 * FP["speed"] * np.array([np.cos(0.7), np.sin(0.7)]),
                               rtol=0, atol=1e-10)
    assert th[0] == 0.7 and np.all(E == 0.0)
