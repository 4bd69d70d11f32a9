"""Spatial sort of the particles (md_sort_particles): the permutation equals
an independent Z-order reference computed here, the arrays move with it bit
for bit, and physics does not notice: right after the sort every row keeps
its partners in the same order, so the forces are the unsorted ones
relabelled, bit for bit; later rebuilds order a cell's members by their new
indices, so an NVE trajectory agrees with the relabelled unsorted one to the
rounding of reordered sums (Sec. 3.2.2-3.3.1)."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import dev, status_word, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1912_04232_b300 as P
    return P


def _zorder_reference(r, space, plan, dim):
    # cells from the FP32 products the binning takes (positions inside the
    # box, where wrapping is the identity), keys by interleaving the bits of
    # the cell coordinates, ties in ascending old index
    nc = np.array([plan.ncell[k] for k in range(3)])
    sc = np.array([plan.cell_scale[k] for k in range(3)], np.float32)
    linv = np.array([space.Linv[k] for k in range(3)], np.float32)
    x = r[:, :3].astype(np.float32)
    assert np.all(np.floor(x[:, :dim] * linv[:dim]) == 0.0)
    q = np.zeros((r.shape[0], 3), np.int64)
    for a in range(dim):
        q[:, a] = np.clip((x[:, a] * sc[a]).astype(np.int64), 0, nc[a] - 1)
    key = np.zeros(r.shape[0], np.int64)
    for b in range(12):
        for a in range(dim):
            key |= ((q[:, a] >> b) & 1) << (dim * b + a)
    return np.lexsort((np.arange(r.shape[0]), key)).astype(np.int32)


def _shuffled_lj(seed):
    c = W.lj_small(seed)
    p = np.random.default_rng(seed + 7).permutation(c.N)
    return c, np.ascontiguousarray(c.r[p]), np.ascontiguousarray(c.v[p])


def test_sort_permutation_matches_zorder_reference_and_moves_arrays(P):
    import torch
    c, r0, v0 = _shuffled_lj(1)
    s = P.md_space_periodic(3, [c.L] * 3)
    nl = P.NeighborList(s, c.N, 2.5, 0.3, 96)
    r, v = to_dev(r0), to_dev(v0)
    st = status_word()
    perm = nl.sort(r, v, st).cpu().numpy()
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    np.testing.assert_array_equal(perm, _zorder_reference(r0, s, nl.plan, 3))
    np.testing.assert_array_equal(r.cpu().numpy(), r0[perm])
    np.testing.assert_array_equal(v.cpu().numpy(), v0[perm])
    # a sorted system is a fixed point: sorting again is the identity
    perm2 = nl.sort(r, v, st).cpu().numpy()
    np.testing.assert_array_equal(perm2, np.arange(c.N, dtype=np.int32))


def test_forces_after_sort_are_the_relabelled_forces_bitwise(P):
    import torch
    c, r0, v0 = _shuffled_lj(2)
    s = P.md_space_periodic(3, [c.L] * 3)
    st = status_word()
    nl = P.NeighborList(s, c.N, 2.5, 0.3, 96)
    r = to_dev(r0)
    f0 = torch.zeros_like(r)
    nl.build(r, st)
    P.md_energy_forces(s, P.lj_pot(), r, nl.plan, f0, None, st)
    perm = nl.sort(r, None, st)
    f1 = torch.zeros_like(r)
    P.md_energy_forces(s, P.lj_pot(), r, nl.plan, f1, None, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    np.testing.assert_array_equal(f1.cpu().numpy(), f0.cpu().numpy()[perm.cpu().numpy()])


def test_nve_trajectory_after_sort_is_the_relabelled_trajectory(P):
    import torch
    c, r0, v0 = _shuffled_lj(3)
    s = P.md_space_periodic(3, [c.L] * 3)
    runs = []
    for do_sort in (False, True):
        st = status_word()
        nl = P.NeighborList(s, c.N, 2.5, 0.3, 96)
        r, v = to_dev(r0), to_dev(v0)
        f = torch.zeros_like(r)
        perm = np.arange(c.N)
        if do_sort:
            perm = nl.sort(r, v, st).cpu().numpy()
        else:
            nl.build(r, st)
        P.md_energy_forces(s, P.lj_pot(), r, nl.plan, f, None, st)
        PE = torch.zeros(150, dtype=torch.float64, device=dev())
        P.md_integrate_nve(s, P.lj_pot(), r, v, f, 1.0, c.dt, 150, nl.plan, PE, None, True, st)
        torch.cuda.synchronize()
        assert P.md_status_poll(st) == 0
        runs.append((perm, r.cpu().numpy(), v.cpu().numpy(), PE.cpu().numpy(), nl.stats()[0]))
    (_, ra, va, Ea, ba), (perm, rb, vb, Eb, bb) = runs
    # 150 steps of a chaotic system from the same state: the reordered sums
    # after the first rebuild leave differences at the 1e-5 level
    dr = rb[:, :3] - ra[perm, :3]
    dr -= c.L * np.round(dr / c.L)
    assert np.abs(dr).max() < 1e-3
    assert np.abs(vb[:, :3] - va[perm, :3]).max() < 1e-2
    assert abs(ba - bb) <= 1 and ba > 1
    np.testing.assert_allclose(Eb, Ea, rtol=1e-6, atol=0)


def test_sort_2d_soft_disks_carries_the_diameters(P):
    import torch
    pk = W.packing_2d(N=1024, D=1.4, seed=5)
    L = W.f32(W.packing_box(1024, 1.4, 0.9))
    r0 = np.zeros((1024, 4), np.float32)
    r0[:, :2] = (pk.s0 * L).astype(np.float32)
    r0[:, :2] = np.where(r0[:, :2] >= L, 0.0, r0[:, :2])
    r0[:, 3] = pk.diam.astype(np.float32)
    s = P.md_space_periodic(2, [L, L])
    st = status_word()
    nl = P.NeighborList(s, 1024, 1.4, 0.3, 64)
    r = to_dev(r0)
    f0 = torch.zeros_like(r)
    nl.build(r, st)
    P.md_energy_forces(s, P.soft_pot(), r, nl.plan, f0, None, st)
    perm = nl.sort(r, None, st)
    f1 = torch.zeros_like(r)
    P.md_energy_forces(s, P.soft_pot(), r, nl.plan, f1, None, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    p = perm.cpu().numpy()
    np.testing.assert_array_equal(p, _zorder_reference(r0, s, nl.plan, 2))
    np.testing.assert_array_equal(r.cpu().numpy()[:, 3], r0[p, 3])
    np.testing.assert_array_equal(f1.cpu().numpy(), f0.cpu().numpy()[p])


def test_sort_rejects_small_or_misaligned_scratch(P):
    import torch
    c = W.lj_small(0)
    s = P.md_space_periodic(3, [c.L] * 3)
    nl = P.NeighborList(s, c.N, 2.5, 0.3, 96)
    r = to_dev(c.r)
    perm = torch.empty(c.N, dtype=torch.int32, device=dev())
    need = P.md_sort_scratch_bytes(nl.plan)
    assert need > 16 * c.N
    raw = torch.empty(need + 512, dtype=torch.uint8, device=dev())
    off = (-raw.data_ptr()) % 256
    with pytest.raises(P.MDError):
        P.md_sort_particles(s, nl.plan, r, None, perm, raw[off:off + need - 256])
    with pytest.raises(P.MDError):
        P.md_sort_particles(s, nl.plan, r, None, perm, raw[off + 16:off + 16 + need])


@pytest.mark.parametrize("dim,ncell,N", [(3, 1, 37), (3, 2, 61), (2, 2, 45), (2, 5, 301)])
def test_sort_on_tiny_and_ragged_grids(P, dim, ncell, N):
    # grids of 1, 2 and 5 cells per axis (deduplicated stencils), particle
    # counts that fill no block: the permutation is the reference one and
    # the forces right after the sort are the relabelled ones, bit for bit
    import torch
    r_list = 1.3
    L = {1: 2.0 * r_list * 1.00003, 2: 2.0 * r_list * 1.001}.get(ncell, ncell * r_list * 1.01)
    rng = np.random.Generator(np.random.PCG64(100 + 10 * dim + ncell))
    r0 = np.zeros((N, 4), np.float32)
    r0[:, :dim] = W.uniform_box_positions(N, L, dim, rng)
    s = P.md_space_periodic(dim, [L] * dim)
    nl = P.NeighborList(s, N, 1.0, 0.3, N)
    assert list(nl.plan.ncell)[:dim] == [ncell] * dim
    st = status_word()
    r = to_dev(r0)
    f0 = torch.zeros_like(r)
    pot = P.soft_pot()
    r[:, 3] = 1.0                                  # unit disks / spheres
    r0[:, 3] = 1.0
    nl.build(r, st)
    P.md_energy_forces(s, pot, r, nl.plan, f0, None, st)
    perm = nl.sort(r, None, st)
    f1 = torch.zeros_like(r)
    P.md_energy_forces(s, pot, r, nl.plan, f1, None, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    p = perm.cpu().numpy()
    np.testing.assert_array_equal(p, _zorder_reference(r0, s, nl.plan, dim))
    np.testing.assert_array_equal(r.cpu().numpy(), r0[p])
    np.testing.assert_array_equal(f1.cpu().numpy(), f0.cpu().numpy()[p])
