"""GPU parity: cell-list neighbor build, LJ forces and the fused NVE step
(Sec. 3.1-3.3) through the C ABI, against the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import dev, force_error, rows_equal, status_word, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1912_04232_b300 as P
    return P


def _setup(P, r, L, r_cut=2.5, skin=0.3, cap=128, dim=3):
    import torch
    s = P.md_space_periodic(dim, [L] * dim)
    nl = P.NeighborList(s, r.shape[0], r_cut, skin, cap)
    rd = to_dev(r, torch.float32)
    st = status_word()
    return s, nl, rd, st


def _nbr_case(P, r, L, r_list_parts=(2.5, 0.3), cap=128, dim=3):
    import torch
    s, nl, rd, st = _setup(P, r, L, *r_list_parts, cap=cap, dim=dim)
    nl.build(rd, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    cnt_o, nb_o = O.neighbor_list(r, L, float(nl.plan.r_list), dim=dim, cap=cap, fp32_decision=True)
    rows_equal(nl.cnt.cpu().numpy(), nl.nbr.cpu().numpy(), cnt_o, nb_o)
    return nl


def test_neighbor_list_bit_exact_lj4096(P):
    c = W.lj_small()
    nl = _nbr_case(P, c.r, c.L)
    assert nl.stats()[0] == 1


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("ncell", [1, 2, 3, 5])
def test_neighbor_list_bit_exact_tiny_and_ragged(P, dim, ncell):
    # boxes with 1, 2, 3, 5 cells per axis (stencil deduplication), N not a
    # multiple of any block size
    r_list = 1.3
    L = {1: 2.0 * r_list * 1.00003, 2: 2.0 * r_list * 1.001}.get(ncell, ncell * r_list * 1.01)
    rng = np.random.Generator(np.random.PCG64(ncell * 10 + dim))
    N = {1: 37, 2: 61, 3: 131, 5: 517}[ncell]
    r = np.zeros((N, 4), np.float32)
    r[:, :dim] = W.uniform_box_positions(N, L, dim, rng)
    nl = _nbr_case(P, r, L, (1.0, 0.3), cap=N if N < 256 else 256, dim=dim)
    assert list(nl.plan.ncell)[:dim] == [ncell] * dim


@pytest.mark.parametrize("dim", [2, 3])
def test_neighbor_list_dense_stencil_fallback(P, dim):
    # a 3x3(x3) grid whose stencil holds every particle (more candidates than
    # a block stages in shared memory): rows come from the per-warp path
    L = 3 * 1.3 * 1.01
    N = 1100
    rng = np.random.Generator(np.random.PCG64(77 + dim))
    r = np.zeros((N, 4), np.float32)
    r[:, :dim] = W.uniform_box_positions(N, L, dim, rng)
    cap = 256 if dim == 3 else 512
    _nbr_case(P, r, L, (1.0, 0.3), cap=cap, dim=dim)


def test_neighbor_list_bit_exact_lj256k(P):
    c = W.lj_large()
    _nbr_case(P, c.r, c.L, cap=128)


def test_neighbor_overflow_sets_status_and_true_count(P):
    import torch
    c = W.lj_small()
    s, nl, rd, st = _setup(P, c.r, c.L, cap=32)
    nl.build(rd, st)
    torch.cuda.synchronize()
    code = P.md_status_poll(st)
    assert code & P.MD_ERR_NBR_OVERFLOW
    cnt_o, _ = O.neighbor_list(c.r, c.L, float(nl.plan.r_list), cap=1)
    np.testing.assert_array_equal(nl.cnt.cpu().numpy(), cnt_o)
    assert nl.stats()[1] == cnt_o.max()


def test_box_too_small_is_rejected_on_host(P):
    s = P.md_space_periodic(3, [5.5, 5.5, 5.5])
    with pytest.raises(P.MDError) as e:
        P.md_nbr_plan(s, 64, 2.5, 0.3, 64)
    assert e.value.code == P.MD_ERR_BOX_TOO_SMALL


@pytest.mark.parametrize("tpp", [4, 8, 16, 32])
def test_lj_forces_energy_lj4096(P, tpp):
    import torch
    c = W.lj_small()
    s, nl, rd, st = _setup(P, c.r, c.L)
    nl.build(rd, st)
    f = torch.zeros((c.N, 4), dtype=torch.float32, device=dev())
    E = torch.zeros(1, dtype=torch.float64, device=dev())
    P.md_set_pair_tpp(tpp)
    try:
        P.md_energy_forces(s, P.lj_pot(), rd, nl.plan, f, E, st)
        torch.cuda.synchronize()
    finally:
        P.md_set_pair_tpp(4)   # the library default
    assert P.md_status_poll(st) == 0
    U, F, e = O.lj(c.r, c.L)
    fg = f.cpu().numpy()
    assert force_error(fg, F) <= 1e-4
    np.testing.assert_allclose(fg[:, 3], e, rtol=0, atol=2e-5 * np.abs(e).max())
    assert abs(E.item() - U) <= 1e-5 * abs(U)


def test_lj_forces_lj256k(P):
    import torch
    c = W.lj_large()
    s, nl, rd, st = _setup(P, c.r, c.L)
    nl.build(rd, st)
    f = torch.zeros((c.N, 4), dtype=torch.float32, device=dev())
    E = torch.zeros(1, dtype=torch.float64, device=dev())
    P.md_energy_forces(s, P.lj_pot(), rd, nl.plan, f, E, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    U, F, e = O.lj(c.r, c.L)
    assert force_error(f.cpu().numpy(), F) <= 1e-4
    assert abs(E.item() - U) <= 1e-5 * abs(U)


def _run_nve(P, c, nsteps, use_graph, cap=128):
    import torch
    s, nl, rd, st = _setup(P, c.r, c.L, cap=cap)
    vd = to_dev(c.v, torch.float32)
    f = torch.zeros((c.N, 4), dtype=torch.float32, device=dev())
    pot = P.lj_pot()
    nl.build(rd, st)
    P.md_energy_forces(s, pot, rd, nl.plan, f, None, st)
    PE = torch.zeros(nsteps, dtype=torch.float64, device=dev())
    KE = torch.zeros(nsteps, dtype=torch.float64, device=dev())
    P.md_integrate_nve(s, pot, rd, vd, f, 1.0, c.dt, nsteps, nl.plan, PE, KE, use_graph, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    return rd.cpu().numpy(), vd.cpu().numpy(), f.cpu().numpy(), PE.cpu().numpy(), KE.cpu().numpy(), nl


@pytest.mark.parametrize("use_graph", [False, True])
def test_nve_short_trajectory_matches_oracle(P, use_graph):
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


def test_nve_graph_equals_direct_launches_bitwise(P):
    c = W.lj_small()
    a = _run_nve(P, c, 100, False)
    b = _run_nve(P, c, 100, True)
    for x, y in zip(a[:5], b[:5]):
        np.testing.assert_array_equal(x, y)
    assert a[5].stats()[0] == b[5].stats()[0] >= 2


def test_nve_energy_series_tracks_oracle_lj4096(P):
    # 100 steps: the aggregate energies of the FP32 run follow the FP64 run
    c = W.lj_small()
    r, v, f, PE, KE, nl = _run_nve(P, c, c.steps, True)
    _, _, PEo, KEo = O.nve(c.r, c.v, c.L, "lj", dt=c.dt, nsteps=c.steps)
    E, Eo = PE + KE, PEo[1:] + KEo[1:]
    assert np.abs(E - Eo).max() / c.N < 1e-4
    assert nl.stats()[0] >= 2


def test_nve_rebuilds_keep_every_interacting_pair(P):
    # after a run, every pair inside r_cut at the final positions is in the list
    c = W.lj_small()
    r, v, f, PE, KE, nl = _run_nve(P, c, 60, True)
    cnt_o, nb_o = O.neighbor_list(r, c.L, 2.5, cap=128)
    cnt_g, nb_g = nl.cnt.cpu().numpy(), nl.nbr.cpu().numpy()
    for i in range(0, c.N, 7):
        have = set(nb_g[i, : cnt_g[i]].tolist())
        need = set(nb_o[i, : cnt_o[i]].tolist())
        assert need <= have, i


@pytest.mark.parametrize("workload", ["lj4096", "lj256k"])
def test_neighbor_list_rebuilt_in_dynamics_bit_exact(P, workload):
    # rebuilds inside the NVE loop see positions kept inside [0, L), so they
    # take the build's wrapped-position forms (interior cells without the
    # wrap, comparison-based nearest image at the faces); the rows of the
    # last rebuild must equal the oracle's FP32-decision list at the
    # positions of that build
    c = W.lj_small() if workload == "lj4096" else W.lj_large()
    r, v, f, PE, KE, nl = _run_nve(P, c, 60 if workload == "lj4096" else 30, True)
    assert nl.stats()[0] >= 3
    assert min(list(nl.plan.ncell)) >= 5   # interior cells exist
    rref = nl.rref.cpu().numpy()
    cnt_o, nb_o = O.neighbor_list(rref, c.L, float(nl.plan.r_list), cap=128, fp32_decision=True)
    rows_equal(nl.cnt.cpu().numpy(), nl.nbr.cpu().numpy(), cnt_o, nb_o)


@pytest.mark.parametrize("use_graph", [False, True])
@pytest.mark.parametrize("nsteps", [1, 37, 80])
def test_nve_fused_step_equals_separate_kick_drift_bitwise(P, use_graph, nsteps):
    # the fused force + kick-drift kernel alternates two position buffers
    # (odd and even step counts end in different ones) and must reproduce
    # the separate kick-drift kernel bit for bit, rebuilds included
    c = W.lj_small()
    outs = []
    for fuse in (0, 1):
        P.md_set_nve_fusion(fuse)
        try:
            outs.append(_run_nve(P, c, nsteps, use_graph))
        finally:
            P.md_set_nve_fusion(1)
    a, b = outs
    for x, y in zip(a[:5], b[:5]):
        np.testing.assert_array_equal(x, y)
    assert a[5].stats()[0] == b[5].stats()[0]
    if nsteps == 80:
        assert b[5].stats()[0] >= 3
    np.testing.assert_array_equal(a[5].cnt.cpu().numpy(), b[5].cnt.cpu().numpy())
    np.testing.assert_array_equal(a[5].nbr.cpu().numpy(), b[5].nbr.cpu().numpy())


def test_run_to_run_bitwise_determinism(P):
    c = W.lj_small()
    a = _run_nve(P, c, 50, True)
    b = _run_nve(P, c, 50, True)
    for x, y in zip(a[:5], b[:5]):
        np.testing.assert_array_equal(x, y)


def test_launch_count_is_reported(P):
    import torch
    c = W.lj_small()
    n0 = P.md_launch_count()
    _run_nve(P, c, 10, True)
    torch.cuda.synchronize()
    n1 = P.md_launch_count()
    # at least kick-drift + force per step, plus the initial build chain
    assert n1 - n0 >= 2 * 10 + 5
