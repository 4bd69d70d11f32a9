"""GPU parity of the tile engine (MD_NBR_TILES, Sec. 3.2.3 lists, Sec. 3.3.1
NVE, Sec. 3.3.2 LJ and soft spheres): its rows, forces, energies and
velocity-Verlet trajectories through the C ABI against the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import dev, force_error, rows_equal_off_cutoff, status_word, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1912_04232_b300 as P
    return P


def _setup(P, r, L, r_cut=2.5, skin=0.3, cap=128):
    import torch
    s = P.md_space_periodic(3, [L] * 3)
    nl = P.NeighborList(s, r.shape[0], r_cut, skin, cap, tiles=True)
    return s, nl, to_dev(r, torch.float32), status_word()


def _tile_forces(P, s, nl, rd, pot, st, tpp=0):
    """Import, one force evaluation on the tiles, export forces and rows."""
    import torch
    N = rd.shape[0]
    f = torch.zeros((N, 4), dtype=torch.float32, device=dev())
    E = torch.zeros(1, dtype=torch.float64, device=dev())
    P.md_set_tile_tpp(tpp)
    try:
        P.md_tiles_import(s, rd, None, None, nl.plan, st)
        P.md_tiles_forces(s, pot, nl.plan, E, st)
        P.md_tiles_export(s, nl.plan, None, None, f, rows=True)
        torch.cuda.synchronize()
    finally:
        P.md_set_tile_tpp(0)   # the library default: chosen by tile size
    return f.cpu().numpy(), E.item()


def _liquid(n_side=10, jitter=0.3, seed=3):
    # FCC lattice with large uniform jitter: a disordered start in which
    # particles sit at arbitrary offsets inside their cells
    return W.lj_fluid("fcc", n_side, jitter=jitter, seed=seed)


@pytest.mark.parametrize("tpp", [1, 4, 8])
@pytest.mark.parametrize("case", ["lj4096", "liquid4000"])
def test_tiles_rows_forces_energies(P, case, tpp):
    c = W.lj_small() if case == "lj4096" else _liquid()
    s, nl, rd, st = _setup(P, c.r, c.L)
    f, E = _tile_forces(P, s, nl, rd, P.lj_pot(), st, tpp)
    assert P.md_status_poll(st) == 0
    # rows: the oracle's FP32-decision sets at r_list, except pairs within
    # 1e-6 sigma of r_list (the tile build decides on image-shifted staged
    # positions with FMAs)
    cnt_o, nb_o = O.neighbor_list(c.r, c.L, float(nl.plan.r_list), cap=128, fp32_decision=True)
    rows_equal_off_cutoff(nl.cnt.cpu().numpy(), nl.nbr.cpu().numpy(), cnt_o, nb_o, c.r, c.L, float(nl.plan.r_list))
    U, F, e = O.lj(c.r, c.L)
    assert force_error(f, F) <= 1e-4
    np.testing.assert_allclose(f[:, 3], e, rtol=0, atol=2e-5 * np.abs(e).max())
    assert abs(E - U) <= 1e-5 * abs(U)


@pytest.mark.parametrize("ncell", [3, 4, 5])
def test_tiles_rows_small_grids(P, ncell):
    # 6, 8 and 10 half-cells per axis: every tile's region wraps the box,
    # so most rows carry partners across the boundary
    r_list = 2.8
    L = ncell * r_list * 1.01
    N = int(0.8 * L ** 3)
    rng = np.random.Generator(np.random.PCG64(500 + ncell))
    r = np.zeros((N, 4), np.float32)
    r[:, :3] = W.uniform_box_positions(N, L, 3, rng)
    s, nl, rd, st = _setup(P, r, L, cap=256)
    assert list(nl.plan.ncell) == [ncell] * 3
    _tile_forces(P, s, nl, rd, P.lj_pot(), st)
    assert P.md_status_poll(st) & ~P.MD_ERR_NONFINITE == 0
    cnt_o, nb_o = O.neighbor_list(r, L, float(nl.plan.r_list), cap=256, fp32_decision=True)
    rows_equal_off_cutoff(nl.cnt.cpu().numpy(), nl.nbr.cpu().numpy(), cnt_o, nb_o, r, L, float(nl.plan.r_list))


def test_tiles_soft_spheres_3d(P):
    # bidisperse 3-D soft spheres (diameters 1.0 / 1.4, 50/50, w column),
    # number density 0.8, uniform random start (overlapping)
    import torch
    N = 3000
    L = W.f32((N / 0.8) ** (1.0 / 3.0))
    rng = np.random.Generator(np.random.PCG64(11))
    r = np.zeros((N, 4), np.float32)
    r[:, :3] = W.uniform_box_positions(N, L, 3, rng)
    diam = np.where(np.arange(N) < N // 2, 1.0, 1.4)
    r[:, 3] = diam
    s, nl, rd, st = _setup(P, r, L, r_cut=1.4, skin=0.3)
    f, E = _tile_forces(P, s, nl, rd, P.soft_pot(), st)
    assert P.md_status_poll(st) == 0
    U, F, e = O.soft(r, diam, L, dim=3)
    assert force_error(f, F) <= 1e-4
    np.testing.assert_allclose(f[:, 3], e, rtol=0, atol=2e-5 * np.abs(e).max())
    assert abs(E - U) <= 1e-5 * abs(U)


@pytest.mark.parametrize("tpp", [0, 4])
def test_tiles_rows_forces_lj256k(P, tpp):
    c = W.lj_large()
    s, nl, rd, st = _setup(P, c.r, c.L)
    info = P.md_tiles_info(s, nl.plan)
    assert info["H"] == (48, 48, 48) and info["tile"] == (2, 8, 6) and info["ntiles"] == 1152
    f, E = _tile_forces(P, s, nl, rd, P.lj_pot(), st, tpp)
    assert P.md_status_poll(st) == 0
    cnt_o, nb_o = O.neighbor_list(c.r, c.L, float(nl.plan.r_list), cap=128, fp32_decision=True)
    rows_equal_off_cutoff(nl.cnt.cpu().numpy(), nl.nbr.cpu().numpy(), cnt_o, nb_o, c.r, c.L, float(nl.plan.r_list))
    U, F, e = O.lj(c.r, c.L)
    assert force_error(f, F) <= 1e-4
    assert abs(E - U) <= 1e-5 * abs(U)


def _run_nve(P, c, nsteps, use_graph, dt=None, tiles=True):
    import torch
    s = P.md_space_periodic(3, [c.L] * 3)
    nl = P.NeighborList(s, c.N, c.r_cut, c.skin, 128, tiles=tiles)
    rd = to_dev(c.r, torch.float32)
    vd = to_dev(c.v, torch.float32)
    st = status_word()
    f = torch.zeros((c.N, 4), dtype=torch.float32, device=dev())
    pot = P.lj_pot()
    nl.build(rd, st)
    P.md_energy_forces(s, pot, rd, nl.plan, f, None, st)
    PE = torch.zeros(nsteps, dtype=torch.float64, device=dev())
    KE = torch.zeros(nsteps, dtype=torch.float64, device=dev())
    P.md_integrate_nve(s, pot, rd, vd, f, 1.0, c.dt if dt is None else dt, nsteps, nl.plan, PE, KE, use_graph, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    return rd.cpu().numpy(), vd.cpu().numpy(), f.cpu().numpy(), PE.cpu().numpy(), KE.cpu().numpy(), nl


@pytest.mark.parametrize("use_graph", [False, True])
def test_tiles_nve_short_trajectory_matches_oracle(P, use_graph):
    c = W.lj_small()
    n = 20
    r, v, f, PE, KE, nl = _run_nve(P, c, n, use_graph)
    ro, vo, PEo, KEo = O.nve(c.r, c.v, c.L, "lj", dt=c.dt, nsteps=n)
    d = r[:, :3] - ro
    d -= c.L * np.round(d / c.L)
    assert np.abs(d).max() < 2e-4
    assert np.abs(v[:, :3] - vo).max() < 2e-3
    np.testing.assert_allclose(PE, PEo[1:], rtol=2e-5)
    np.testing.assert_allclose(KE, KEo[1:], rtol=2e-5)
    # returned positions are wrapped into the box
    assert r[:, :3].min() >= 0.0 and r[:, :3].max() < c.L
    # the forces returned belong to the returned positions
    U, F, _ = O.lj(r, c.L)
    assert force_error(f, F) <= 1e-4


def test_tiles_nve_zero_dt_keeps_forces(P):
    # dt = 0: nothing moves, the forces returned are those of the start
    c = _liquid(8)
    r, v, f, PE, KE, nl = _run_nve(P, c, 3, True, dt=0.0)
    np.testing.assert_array_equal(r, c.r)
    U, F, _ = O.lj(c.r, c.L)
    assert force_error(f, F) <= 1e-4
    np.testing.assert_allclose(PE, U, rtol=1e-5)


def test_tiles_graph_equals_host_launches_bitwise(P):
    c = W.lj_small()
    a = _run_nve(P, c, 100, False)
    b = _run_nve(P, c, 100, True)
    for x, y in zip(a[:5], b[:5]):
        np.testing.assert_array_equal(x, y)
    assert a[5].stats()[0] == b[5].stats()[0] >= 3
    np.testing.assert_array_equal(a[5].nbr.cpu().numpy(), b[5].nbr.cpu().numpy())


def test_tiles_run_to_run_bitwise(P):
    c = _liquid(jitter=0.1)   # close pairs of the 0.3 jitter would blow up under dynamics
    a = _run_nve(P, c, 60, True)
    b = _run_nve(P, c, 60, True)
    for x, y in zip(a[:5], b[:5]):
        np.testing.assert_array_equal(x, y)


def test_tiles_nve_energy_series_tracks_oracle(P):
    c = W.lj_small()
    r, v, f, PE, KE, nl = _run_nve(P, c, c.steps, True)
    _, _, PEo, KEo = O.nve(c.r, c.v, c.L, "lj", dt=c.dt, nsteps=c.steps)
    E, Eo = PE + KE, PEo[1:] + KEo[1:]
    assert np.abs(E - Eo).max() / c.N < 1e-4
    assert nl.stats()[0] >= 3


@pytest.mark.parametrize("workload", ["lj4096", "lj256k"])
def test_tiles_rows_after_dynamics(P, workload):
    # the rows handed back after a run are the last in-loop build's: equal to
    # the oracle's FP32-decision sets at that build's positions, and they
    # hold every pair inside r_cut at the final positions
    c = W.lj_small() if workload == "lj4096" else W.lj_large()
    r, v, f, PE, KE, nl = _run_nve(P, c, 60 if workload == "lj4096" else 30, True)
    assert nl.stats()[0] >= 3
    rref = nl.rref.cpu().numpy()
    cnt_o, nb_o = O.neighbor_list(rref, c.L, float(nl.plan.r_list), cap=128, fp32_decision=True)
    cnt_g, nb_g = nl.cnt.cpu().numpy(), nl.nbr.cpu().numpy()
    rows_equal_off_cutoff(cnt_g, nb_g, cnt_o, nb_o, rref, c.L, float(nl.plan.r_list))
    cnt_c, nb_c = O.neighbor_list(r, c.L, 2.5, cap=128)
    for i in range(0, c.N, 97 if c.N > 10000 else 7):
        assert set(nb_c[i, : cnt_c[i]].tolist()) <= set(nb_g[i, : cnt_g[i]].tolist()), i


def test_tiles_equal_int32_rows_engine_within_rounding(P):
    # the tile engine and the int32-row engine integrate the same dynamics;
    # over 10 steps they agree to FP32 rounding
    c = W.lj_small()
    a = _run_nve(P, c, 10, True, tiles=True)
    b = _run_nve(P, c, 10, True, tiles=False)
    d = a[0][:, :3] - b[0][:, :3]
    d -= c.L * np.round(d / c.L)
    assert np.abs(d).max() < 1e-4
    np.testing.assert_allclose(a[3], b[3], rtol=1e-5)


def test_tiles_region_overflow_is_reported(P):
    # most particles crowded into one corner: that tile's region holds more
    # than its capacity; the run reports MD_ERR_NBR_OVERFLOW and the context
    # stays usable
    import torch
    c = W.lj_small()
    r = c.r.copy()
    rng = np.random.Generator(np.random.PCG64(9))
    k = 2000
    r[:k, :3] = rng.uniform(0.0, 2.5, size=(k, 3)).astype(np.float32)
    s, nl, rd, st = _setup(P, r, c.L, cap=128)
    _tile_forces(P, s, nl, rd, P.lj_pot(), st)
    assert P.md_status_poll(st) & P.MD_ERR_NBR_OVERFLOW
    # the same library still computes correct results afterwards
    s2, nl2, rd2, st2 = _setup(P, c.r, c.L)
    f, E = _tile_forces(P, s2, nl2, rd2, P.lj_pot(), st2)
    assert P.md_status_poll(st2) == 0
    U, F, _ = O.lj(c.r, c.L)
    assert force_error(f, F) <= 1e-4
