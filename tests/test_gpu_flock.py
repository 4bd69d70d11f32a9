"""GPU parity of the flocking energy model (Sec. 4.3 and its appendix)
against the FP64 oracle: energies, one step, a 20-step trajectory with
obstacles and list rebuilds, and a lone boid swimming across the boundary."""
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


def _run(P, fl, dt, nsteps, obstacles=True, skin=4.0):
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
    st = status_word()
    E = torch.zeros(max(nsteps, 1), dtype=torch.float64, device=dev())
    nl.build(bd, st)
    P.md_flock_run(s, prm, obs, n_obs, bd, th, alt, dt, nsteps, nl.plan, E, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    return bd.cpu().numpy(), th.cpu().numpy(), E.cpu().numpy(), nl


def _wrapdiff(a, b, L):
    d = a - b
    return d - L * np.round(d / L)


def test_flock_energy_and_one_step(P):
    fl = W.flock(2000, seed=1)
    b, th, E, _ = _run(P, fl, 0.5, 1)
    Eo, gR, gth, parts = O.flock_grad(fl.R, fl.theta, fl.L, obstacles=fl.obstacles)
    assert abs(E[0] - Eo) <= 2e-5 * abs(Eo)
    Ro, tho, _ = O.flock_run(fl.R, fl.theta, fl.L, dt=0.5, nsteps=1, obstacles=fl.obstacles)
    assert np.abs(_wrapdiff(b[:, :2], Ro, fl.L)).max() < 5e-4
    assert np.abs(th - tho).max() < 2e-5
    np.testing.assert_allclose(b[:, 2], np.cos(th), rtol=0, atol=1e-6)
    np.testing.assert_allclose(b[:, 3], np.sin(th), rtol=0, atol=1e-6)


@pytest.mark.parametrize("obstacles", [False, True])
def test_flock_trajectory_matches_oracle(P, obstacles):
    fl = W.flock(1500, seed=2)
    n, dt = 100, 0.1
    b, th, E, nl = _run(P, fl, dt, n, obstacles=obstacles)
    Ro, tho, Eo = O.flock_run(fl.R, fl.theta, fl.L, dt=dt, nsteps=n,
                              obstacles=fl.obstacles if obstacles else None)
    assert nl.stats()[0] >= 2            # the boids moved far enough to rebuild
    # the cohesion set has a hard edge, so FP32 and FP64 runs part where a
    # boid crosses R_cohesion; the bound is the oracle's own spread from a
    # start perturbed at the size of FP32 rounding (coordinates ~800)
    rng = np.random.Generator(np.random.PCG64(9))
    Rp = fl.R.astype(np.float64) + rng.uniform(-3e-5, 3e-5, size=fl.R.shape)
    thp = fl.theta.astype(np.float64) + rng.uniform(-1e-7, 1e-7, size=fl.N)
    Rq, thq, Eq = O.flock_run(Rp, thp, fl.L, dt=dt, nsteps=n, obstacles=fl.obstacles if obstacles else None)
    e_spread = np.maximum(np.abs(Eq - Eo)[:n], 1e-6 * np.abs(Eo[:n]))
    assert np.all(np.abs(E - Eo[:n]) <= 4 * e_spread + 1e-6 * np.abs(Eo[:n]))
    r_spread = max(np.abs(_wrapdiff(Rq, Ro, fl.L)).max(), 1e-3)
    t_spread = max(np.abs(thq - tho).max(), 1e-4)
    assert np.abs(_wrapdiff(b[:, :2], Ro, fl.L)).max() < 4 * r_spread
    assert np.abs(th - tho).max() < 4 * t_spread


def test_lone_boid_crosses_the_boundary(P):
    fl = W.Flock(N=1, L=W.f32(400.0), R=np.array([[395.0, 10.0]], np.float32), theta=np.array([0.3], np.float32),
                 obstacles=np.zeros((0, 3), np.float32))
    b, th, E, _ = _run(P, fl, 0.5, 40, obstacles=False)
    want = np.mod(np.array([395.0, 10.0]) + 0.5 * 40 * np.array([np.cos(0.3), np.sin(0.3)]), 400.0)
    np.testing.assert_allclose(b[0, :2], want, rtol=0, atol=1e-3)
    assert th[0] == np.float32(0.3) and np.all(E == 0.0)


def test_flock_graph_loop_equals_host_launches_bitwise(P):
    # 41 steps: 20 graph iterations of two steps and one host-launched step
    fl = W.flock(1500, seed=4)
    P.md_set_loop_graphs(False)
    try:
        a = _run(P, fl, 0.1, 41)
    finally:
        P.md_set_loop_graphs(True)
    b = _run(P, fl, 0.1, 41)
    for x, y in zip(a[:3], b[:3]):
        np.testing.assert_array_equal(x, y)
    assert a[3].stats()[0] == b[3].stats()[0]
