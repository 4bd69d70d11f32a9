"""Pins of the flocking oracle (Sec. 4.3 and its appendix): closed-form
pair, obstacle and predator energies, gradients against central finite
differences (with the displacement stop-gradients of alignment, cohesion
and chasing), invariance under a quarter turn and translation, the free
swimming of a lone boid, and Reynolds' rules emerging from the energy
dynamics."""
import numpy as np

import oracle as O
import workloads as W

FP = O.FLOCK_DEFAULTS


def _rho(r, Rc, a=2.0):
    return (1.0 - r / Rc) ** a / a if r < Rc else 0.0


def test_pair_closed_forms():
    L = 200.0
    R = np.array([[10.0, 10.0], [30.0, 10.0]])
    # anti-aligned: (1 - N.N)^2 = 4; cohesion zero (each faces the other)
    E, gR, gth, _, (al, av, co, ob, fl, ch) = O.flock_grad(R, np.array([0.0, np.pi]), L)
    assert abs(al - FP["J_align"] * _rho(20.0, FP["R_align"]) * 4.0) < 1e-12
    assert abs(av - FP["J_avoid"] * _rho(20.0, FP["R_avoid"])) < 1e-12
    assert co == 0.0 and ob == 0.0
    # aligned, both facing +x: no alignment energy; boid 1 faces away from
    # its only neighbour: cohesion 1/2 J (1 - (-1))^2 = 2 J
    E, gR, gth, _, (al, av, co, ob, fl, ch) = O.flock_grad(R, np.array([0.0, 0.0]), L)
    assert al == 0.0
    assert abs(co - 2.0 * FP["J_cohesion"]) < 1e-12
    # across the periodic boundary: same pair, shifted
    R2 = np.array([[195.0, 10.0], [15.0, 10.0]])
    _, _, _, _, parts2 = O.flock_grad(R2, np.array([0.0, np.pi]), L)
    assert abs(parts2[0] - FP["J_align"] * _rho(20.0, FP["R_align"]) * 4.0) < 1e-12


def test_obstacle_closed_form():
    # boid at distance 5 from an obstacle of radius 10, facing it: w = N,
    # (1 + 1)^2 = 4; facing away: 0
    L = 200.0
    obs = [[50.0, 50.0, 10.0]]
    R = np.array([[45.0, 50.0]])
    _, _, _, _, (al, av, co, ob, fl, ch) = O.flock_grad(R, np.array([0.0]), L, obstacles=obs)
    assert abs(ob - FP["J_obstacle"] * _rho(5.0, 10.0) * 4.0) < 1e-12
    _, _, _, _, (al, av, co, ob, fl, ch) = O.flock_grad(R, np.array([np.pi]), L, obstacles=obs)
    assert abs(ob) < 1e-12


def _flock(N, L, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(0, L, size=(N, 2)), rng.uniform(-np.pi, np.pi, size=N)


def test_gradients_match_finite_differences():
    L = 150.0
    R, th = _flock(60, L, 1)
    obs = [[40.0, 60.0, 20.0], [100.0, 100.0, 15.0]]
    pred = [[70.0, 80.0, 0.4], [20.0, 130.0, -2.0]]
    E, gR, gth, gP, _ = O.flock_grad(R, th, L, obstacles=obs, predators=pred)
    h = 1e-6
    g = lambda R_, th_, p_: O.flock_grad(R_, th_, L, obstacles=obs, predators=p_)
    for i in range(0, 60, 7):
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (g(R, tp, pred)[0] - g(R, tm, pred)[0]) / (2 * h)
        assert abs(fd - gth[i]) < 1e-6 * max(1.0, abs(gth[i]))
        for k in range(2):
            Rp, Rm = R.copy(), R.copy()
            Rp[i, k] += h
            Rm[i, k] -= h
            # alignment and cohesion take no gradient through the positions
            ep, em = g(Rp, th, pred)[4], g(Rm, th, pred)[4]
            fd = ((ep[1] + ep[3] + ep[4]) - (em[1] + em[3] + em[4])) / (2 * h)
            assert abs(fd - gR[i, k]) < 1e-6 * max(1.0, abs(gR[i, k]))
    # predators minimise their own energy: chase (heading only) + obstacles
    for p in range(2):
        for k in range(3):
            pp, pm = np.array(pred), np.array(pred)
            pp[p, k] += h
            pm[p, k] -= h
            ep, em = g(R, th, pp)[4], g(R, th, pm)[4]
            if k == 2:
                fd = ((ep[3] + ep[5]) - (em[3] + em[5])) / (2 * h)
            else:
                fd = (ep[3] - em[3]) / (2 * h)
            assert abs(fd - gP[p, k]) < 1e-6 * max(1.0, abs(gP[p, k]))


def test_predator_closed_forms():
    L = 400.0
    FPd = O.FLOCK_DEFAULTS
    # a boid 20 from a predator, facing it: flee = J rho(20; R_flee) 4
    R = np.array([[100.0, 100.0]])
    _, _, _, _, parts = O.flock_grad(R, np.array([0.0]), L, predators=[[120.0, 100.0, 0.0]])
    assert abs(parts[4] - FPd["J_flee"] * _rho(20.0, FPd["R_flee"]) * 4.0) < 1e-12
    # the predator faces along +x while its only boid lies along +y:
    # chase = J/2 (1 - 0)^2
    _, _, _, gP, parts = O.flock_grad(np.array([[120.0, 150.0]]), np.array([1.0]), L,
                                      predators=[[120.0, 100.0, 0.0]])
    assert abs(parts[5] - 0.5 * FPd["J_chase"]) < 1e-12
    assert gP[0, 2] < 0.0     # it turns towards the boid (theta increases)


def test_quarter_turn_and_translation_invariance():
    L = 150.0
    R, th = _flock(80, L, 2)
    obs = np.array([[40.0, 60.0, 20.0]])
    pred = np.array([[90.0, 30.0, 1.1]])
    E, _, _, _, parts = O.flock_grad(R, th, L, obstacles=obs, predators=pred)
    rot = np.stack([np.mod(-R[:, 1], L), R[:, 0]], axis=1)
    orot = np.array([[np.mod(-obs[0, 1], L), obs[0, 0], obs[0, 2]]])
    prot = np.array([[np.mod(-pred[0, 1], L), pred[0, 0], pred[0, 2] + np.pi / 2]])
    E2, _, _, _, parts2 = O.flock_grad(rot, th + np.pi / 2, L, obstacles=orot, predators=prot)
    np.testing.assert_allclose(parts2, parts, rtol=1e-10, atol=1e-12)
    shift = np.array([17.3, -41.9])
    sh = np.mod(R + shift, L)
    osh = obs.copy()
    osh[0, :2] = np.mod(obs[0, :2] + shift, L)
    psh = pred.copy()
    psh[0, :2] = np.mod(pred[0, :2] + shift, L)
    E3, _, _, _, parts3 = O.flock_grad(sh, th, L, obstacles=osh, predators=psh)
    np.testing.assert_allclose(parts3, parts, rtol=1e-10, atol=1e-12)


def test_lone_boid_swims_straight():
    L = 500.0
    R0 = np.array([[100.0, 200.0]])
    th0 = np.array([0.7])
    R, th, _, E = O.flock_run(R0, th0, L, dt=0.25, nsteps=40)
    np.testing.assert_allclose(R[0], R0[0] + 0.25 * 40 * FP["speed"] * np.array([np.cos(0.7), np.sin(0.7)]),
                               rtol=0, atol=1e-10)
    assert th[0] == 0.7 and np.all(E == 0.0)


def test_lone_predator_sprints():
    # no boids in chase range and no obstacles: the predator swims straight,
    # at twice its speed in the first sprint_steps of every sprint_period
    L = 2000.0
    R0 = np.array([[10.0, 10.0]])
    p0 = np.array([[1000.0, 1000.0, -0.4]])
    prm = dict(sprint_period=7, sprint_steps=3, sprint_factor=2.0)
    n, dt = 23, 0.5
    _, _, p, _ = O.flock_run(R0, np.array([0.0]), L, dt=dt, nsteps=n, params=prm, predators=p0)
    fast = sum(1 for s in range(n) if s % 7 < 3)
    dist = dt * FP["predator_speed"] * (2.0 * fast + (n - fast))
    np.testing.assert_allclose(p[0, :2], p0[0, :2] + dist * np.array([np.cos(-0.4), np.sin(-0.4)]), rtol=0,
                               atol=1e-9)
    assert p[0, 2] == -0.4
    # sprints off: plain speed
    _, _, p, _ = O.flock_run(R0, np.array([0.0]), L, dt=dt, nsteps=n, params=dict(sprint_period=0),
                             predators=p0)
    np.testing.assert_allclose(p[0, :2], p0[0, :2] + dt * n * FP["predator_speed"] *
                               np.array([np.cos(-0.4), np.sin(-0.4)]), rtol=0, atol=1e-9)


def _order_and_spacing(R, th, L, r_align):
    # mean cos(theta_i - theta_j) over pairs within the alignment range, and
    # the smallest pair distance (minimum image)
    d = R[:, None, :2] - R[None, :, :2]
    d -= L * np.round(d / L)
    r = np.sqrt((d ** 2).sum(-1))
    np.fill_diagonal(r, np.inf)
    c = np.cos(th[:, None] - th[None, :])
    return float(c[r < r_align].mean()), float(r.min())


def test_energy_descent_makes_the_rules_emerge():
    # Sec. 4.3: each term is built so that lowering it produces one of
    # Reynolds' rules.  From uniform random headings, 300 steps of the energy
    # dynamics with the alignment term alone turn the boids towards their
    # neighbours' headings (local order 0 -> > 0.6) while nothing keeps them
    # apart; with the avoidance and cohesion terms on, the order still grows
    # and no two boids come closer than a few units.  A sign error in either
    # update would show here though the gradients match finite differences.
    f = W.flock(N=400, n_obs=0, seed=3)
    o0, m0 = _order_and_spacing(f.R.astype(np.float64), f.theta.astype(np.float64), f.L, 45.0)
    assert abs(o0) < 0.1
    R, th, _, E = O.flock_run(f.R, f.theta, f.L, dt=0.1, nsteps=300, params=dict(J_avoid=0.0, J_cohesion=0.0))
    o1, m1 = _order_and_spacing(R, th, f.L, 45.0)
    assert o1 > 0.6 and E[-1] < 0.1 * E[0]
    assert m1 < 2.0
    R, th, _, E = O.flock_run(f.R, f.theta, f.L, dt=0.1, nsteps=300)
    o2, m2 = _order_and_spacing(R, th, f.L, 45.0)
    assert o2 > 0.6 and E[-1] < E[0]
    assert m2 > 5.0 > m0
