"""GPU parity of the flocking energy model (Sec. 4.3 and its appendix)
against the FP64 oracle: energies, one step, a 100-step trajectory with
obstacles and list rebuilds, predators chasing the flock, and a lone boid
swimming across the boundary."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import dev, status_word, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1912_04232_b300 as P
    return P


def _run(P, fl, dt, nsteps, obstacles=True, predators=False, skin=4.0):
    import torch
    prm = P.flock_params()
    rmax = max(prm.R_align, prm.R_avoid, prm.R_cohesion)
    s = P.md_space_periodic(2, [fl.L, fl.L])
    nl = P.NeighborList(s, fl.N, rmax, skin, 128)
    b = np.zeros((fl.N, 4), np.float32)
    b[:, :2] = fl.R
    bd = to_dev(b, torch.float32)
    th = to_dev(fl.theta, torch.float32)
    alt = torch.zeros_like(bd)
    obs = to_dev(fl.obstacles, torch.float32) if obstacles else None
    n_obs = fl.obstacles.shape[0] if obstacles else 0
    n_p = fl.predators.shape[0] if predators else 0
    pr = np.zeros((max(n_p, 1), 4), np.float32)
    if n_p:
        pr[:n_p, :3] = fl.predators
    prd = to_dev(pr, torch.float32)
    pr_alt = torch.zeros_like(prd)
    st = status_word()
    E = torch.zeros(max(nsteps, 1), dtype=torch.float64, device=dev())
    nl.build(bd, st)
    P.md_flock_run(s, prm, obs, n_obs, prd if n_p else None, pr_alt if n_p else None, n_p, bd, th, alt, dt, nsteps,
                   nl.plan, E, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    return bd.cpu().numpy(), th.cpu().numpy(), E.cpu().numpy(), nl, prd.cpu().numpy()[:n_p]


def _wrapdiff(a, b, L):
    d = a - b
    return d - L * np.round(d / L)


def test_flock_energy_and_one_step(P):
    fl = W.flock(2000, seed=1)
    b, th, E, _, _ = _run(P, fl, 0.5, 1)
    Eo, gR, gth, gP, parts = O.flock_grad(fl.R, fl.theta, fl.L, obstacles=fl.obstacles)
    assert abs(E[0] - Eo) <= 2e-5 * abs(Eo)
    Ro, tho, _, _ = O.flock_run(fl.R, fl.theta, fl.L, dt=0.5, nsteps=1, obstacles=fl.obstacles)
    assert np.abs(_wrapdiff(b[:, :2], Ro, fl.L)).max() < 5e-4
    assert np.abs(th - tho).max() < 2e-5
    np.testing.assert_allclose(b[:, 2], np.cos(th), rtol=0, atol=1e-6)
    np.testing.assert_allclose(b[:, 3], np.sin(th), rtol=0, atol=1e-6)


def test_predators_energy_and_one_step(P):
    fl = W.flock(2000, seed=5, n_pred=6)
    b, th, E, _, pr = _run(P, fl, 0.5, 1, predators=True)
    Eo, gR, gth, gP, parts = O.flock_grad(fl.R, fl.theta, fl.L, obstacles=fl.obstacles, predators=fl.predators)
    assert parts[4] > 0.0 and parts[5] > 0.0     # boids in flight range, predators off their course
    assert abs(E[0] - Eo) <= 2e-5 * abs(Eo)
    Ro, tho, po, _ = O.flock_run(fl.R, fl.theta, fl.L, dt=0.5, nsteps=1, obstacles=fl.obstacles,
                                 predators=fl.predators)
    assert np.abs(_wrapdiff(b[:, :2], Ro, fl.L)).max() < 5e-4
    assert np.abs(th - tho).max() < 2e-5
    assert np.abs(_wrapdiff(pr[:, :2], po[:, :2], fl.L)).max() < 5e-4
    assert np.abs(pr[:, 2] - po[:, 2]).max() < 2e-5


def _spread_run(fl, dt, n, obstacles, predators):
    # the cohesion and chase sets have hard edges, so FP32 and FP64 runs
    # part where an agent crosses R_cohesion or R_chase; the bound is the
    # oracle's own spread from a start perturbed at the size of FP32
    # rounding (coordinates ~800)
    rng = np.random.Generator(np.random.PCG64(9))
    Rp = fl.R.astype(np.float64) + rng.uniform(-3e-5, 3e-5, size=fl.R.shape)
    thp = fl.theta.astype(np.float64) + rng.uniform(-1e-7, 1e-7, size=fl.N)
    pp = None
    if predators:
        pp = fl.predators.astype(np.float64)
        pp[:, :2] += rng.uniform(-3e-5, 3e-5, size=(pp.shape[0], 2))
    return O.flock_run(Rp, thp, fl.L, dt=dt, nsteps=n, obstacles=fl.obstacles if obstacles else None,
                       predators=pp)


@pytest.mark.parametrize("obstacles,predators", [(False, False), (True, False), (True, True)])
def test_flock_trajectory_matches_oracle(P, obstacles, predators):
    fl = W.flock(1500, seed=2, n_pred=4 if predators else 0)
    n, dt = 100, 0.1
    b, th, E, nl, pr = _run(P, fl, dt, n, obstacles=obstacles, predators=predators)
    Ro, tho, po, Eo = O.flock_run(fl.R, fl.theta, fl.L, dt=dt, nsteps=n,
                                  obstacles=fl.obstacles if obstacles else None,
                                  predators=fl.predators if predators else None)
    assert nl.stats()[0] >= 2            # the boids moved far enough to rebuild
    Rq, thq, pq, Eq = _spread_run(fl, dt, n, obstacles, predators)
    e_spread = np.maximum(np.abs(Eq - Eo)[:n], 1e-6 * np.abs(Eo[:n]))
    assert np.all(np.abs(E - Eo[:n]) <= 4 * e_spread + 1e-6 * np.abs(Eo[:n]))
    r_spread = max(np.abs(_wrapdiff(Rq, Ro, fl.L)).max(), 1e-3)
    t_spread = max(np.abs(thq - tho).max(), 1e-4)
    assert np.abs(_wrapdiff(b[:, :2], Ro, fl.L)).max() < 4 * r_spread
    assert np.abs(th - tho).max() < 4 * t_spread
    if predators:
        p_spread = max(np.abs(_wrapdiff(pq[:, :2], po[:, :2], fl.L)).max(), 1e-3)
        pt_spread = max(np.abs(pq[:, 2] - po[:, 2]).max(), 1e-4)
        assert np.abs(_wrapdiff(pr[:, :2], po[:, :2], fl.L)).max() < 4 * p_spread
        assert np.abs(pr[:, 2] - po[:, 2]).max() < 4 * pt_spread


def test_lone_boid_crosses_the_boundary(P):
    fl = W.Flock(N=1, L=W.f32(400.0), R=np.array([[395.0, 10.0]], np.float32), theta=np.array([0.3], np.float32),
                 obstacles=np.zeros((0, 3), np.float32))
    b, th, E, _, _ = _run(P, fl, 0.5, 40, obstacles=False)
    want = np.mod(np.array([395.0, 10.0]) + 0.5 * 40 * np.array([np.cos(0.3), np.sin(0.3)]), 400.0)
    np.testing.assert_allclose(b[0, :2], want, rtol=0, atol=1e-3)
    assert th[0] == np.float32(0.3) and np.all(E == 0.0)


@pytest.mark.parametrize("predators", [False, True])
def test_flock_graph_loop_equals_host_launches_bitwise(P, predators):
    # 41 steps: 20 graph iterations of two steps and one host-launched step
    fl = W.flock(1500, seed=4, n_pred=3 if predators else 0)
    P.md_set_loop_graphs(False)
    try:
        a = _run(P, fl, 0.1, 41, predators=predators)
    finally:
        P.md_set_loop_graphs(True)
    b = _run(P, fl, 0.1, 41, predators=predators)
    for x, y in zip(a[:3] + a[4:], b[:3] + b[4:]):
        np.testing.assert_array_equal(x, y)
    assert a[3].stats()[0] == b[3].stats()[0]


def test_predator_sprints_without_energy_series(P):
    # a lone predator far from the boids: the sprint schedule is followed
    # with and without the energy series (the step count is kept either way)
    import torch
    fl = W.Flock(N=64, L=W.f32(2000.0), R=np.random.Generator(np.random.PCG64(3)).uniform(0, 100, (64, 2))
                 .astype(np.float32), theta=np.zeros(64, np.float32), obstacles=np.zeros((0, 3), np.float32),
                 predators=np.array([[1000.0, 1000.0, -0.4]], np.float32))
    prm = dict(sprint_period=7, sprint_steps=3, sprint_factor=2.0)
    _, _, po, _ = O.flock_run(fl.R, fl.theta, fl.L, dt=0.5, nsteps=23, params=prm, predators=fl.predators)
    for with_E in (True, False):
        s = P.md_space_periodic(2, [fl.L, fl.L])
        pp = P.flock_params(**prm)
        nl = P.NeighborList(s, fl.N, 45.0, 4.0, 128)
        b = np.zeros((fl.N, 4), np.float32)
        b[:, :2] = fl.R
        bd = to_dev(b, torch.float32)
        th = to_dev(fl.theta, torch.float32)
        pr = np.zeros((1, 4), np.float32)
        pr[0, :3] = fl.predators[0]
        prd = to_dev(pr, torch.float32)
        st = status_word()
        E = torch.zeros(23, dtype=torch.float64, device=dev()) if with_E else None
        nl.build(bd, st)
        P.md_flock_run(s, pp, None, 0, prd, torch.zeros_like(prd), 1, bd, th, torch.zeros_like(bd), 0.5, 23, nl.plan,
                       E, st)
        torch.cuda.synchronize()
        assert P.md_status_poll(st) == 0
        got = prd.cpu().numpy()[0]
        np.testing.assert_allclose(got[:2], po[0, :2], rtol=0, atol=2e-3)
        assert got[2] == np.float32(-0.4)


def _order_and_spacing(R, th, L, r_align):
    d = R[:, None, :2].astype(np.float64) - R[None, :, :2].astype(np.float64)
    d -= L * np.round(d / L)
    r = np.sqrt((d ** 2).sum(-1))
    np.fill_diagonal(r, np.inf)
    c = np.cos(th[:, None].astype(np.float64) - th[None, :].astype(np.float64))
    return float(c[r < r_align].mean()), float(r.min())


@pytest.mark.parametrize("terms", ["align", "all"])
def test_rules_emerge_as_in_the_oracle(P, terms):
    # 300 steps from uniform random headings: alignment alone orders the
    # headings locally with nothing keeping boids apart; with avoidance and
    # cohesion the order still grows and boids keep their distance.  The
    # trajectories themselves part from the FP64 oracle's (chaos), so the
    # GPU's order parameter is compared with the oracle's within 0.1.
    import torch
    fl = W.flock(N=400, n_obs=0, seed=3)
    kw = dict(J_avoid=0.0, J_cohesion=0.0) if terms == "align" else {}
    prm = P.flock_params(**kw)
    s = P.md_space_periodic(2, [fl.L, fl.L])
    nl = P.NeighborList(s, fl.N, max(prm.R_align, prm.R_avoid, prm.R_cohesion), 4.0, 128)
    b = np.zeros((fl.N, 4), np.float32)
    b[:, :2] = fl.R
    bd = to_dev(b, torch.float32)
    th = to_dev(fl.theta, torch.float32)
    alt = torch.zeros_like(bd)
    st = status_word()
    E = torch.zeros(300, dtype=torch.float64, device=dev())
    nl.build(bd, st)
    P.md_flock_run(s, prm, None, 0, None, None, 0, bd, th, alt, 0.1, 300, nl.plan, E, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    og, mg = _order_and_spacing(bd.cpu().numpy(), th.cpu().numpy(), fl.L, 45.0)
    Ro, tho, _, _ = O.flock_run(fl.R, fl.theta, fl.L, dt=0.1, nsteps=300, params=kw)
    oo, mo = _order_and_spacing(Ro, tho, fl.L, 45.0)
    assert og > 0.6 and abs(og - oo) < 0.1, (og, oo)
    if terms == "align":
        assert mg < 2.0
    else:
        assert mg > 5.0, (mg, mo)
