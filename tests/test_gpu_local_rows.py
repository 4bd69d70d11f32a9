"""GPU parity of the block-centred force path (lists with local rows): the
16-bit rows index the shared-memory staging of the region around each block
of 2 x 2 x 2 cells, and the forces, energies per particle and whole NVE
trajectories must be the same bits as with the int32 rows (Sec. 3.2.2-3.3.1)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import dev, force_error, status_word, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1912_04232_b300 as P
    return P


def _forces(P, r, L, pot, r_cut, dim=3, cap=128, local=False, skin=0.3):
    import torch
    s = P.md_space_periodic(dim, [L] * dim)
    nl = P.NeighborList(s, r.shape[0], r_cut, skin, cap, local_rows=local)
    rd = to_dev(r, torch.float32)
    st = status_word()
    nl.build(rd, st)
    f = torch.zeros((r.shape[0], 4), dtype=torch.float32, device=dev())
    E = torch.zeros(1, dtype=torch.float64, device=dev())
    P.md_energy_forces(s, pot, rd, nl.plan, f, E, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    return f.cpu().numpy(), float(E.item()), nl


@pytest.mark.parametrize("workload", ["lj4096", "lj256k"])
def test_local_rows_forces_bitwise_lj(P, workload):
    c = W.lj_small() if workload == "lj4096" else W.lj_large()
    fa, Ea, nla = _forces(P, c.r, c.L, P.lj_pot(), 2.5)
    fb, Eb, nlb = _forces(P, c.r, c.L, P.lj_pot(), 2.5, local=True)
    np.testing.assert_array_equal(fa, fb)
    # totals: FP32 per-thread partial sums over another particle-to-thread map
    assert abs(Ea - Eb) <= 1e-7 * abs(Ea)
    # the int32 rows of a local-row list are those of the plain list
    np.testing.assert_array_equal(nlb.cnt.cpu().numpy(), nla.cnt.cpu().numpy())
    np.testing.assert_array_equal(nlb.nbr.cpu().numpy(), nla.nbr.cpu().numpy())
    if workload == "lj4096":
        U, F, _ = O.lj(c.r, c.L)
        assert force_error(fb, F) <= 1e-4


def test_local_rows_forces_bitwise_soft_2d(P):
    pk = W.packing_2d()
    L = W.f32(W.packing_box(pk.N, pk.D, pk.phi))
    r = np.zeros((pk.N, 4), np.float32)
    r[:, :2] = (pk.s0 * L).astype(np.float32)
    r[:, :2] = np.where(r[:, :2] >= L, 0.0, r[:, :2])
    r[:, 3] = pk.diam.astype(np.float32)
    fa, Ea, _ = _forces(P, r, L, P.soft_pot(), 1.2, dim=2)
    fb, Eb, _ = _forces(P, r, L, P.soft_pot(), 1.2, dim=2, local=True)
    np.testing.assert_array_equal(fa, fb)
    assert abs(Ea - Eb) <= 1e-7 * max(abs(Ea), 1.0)


def test_local_rows_dense_stencils_fall_back_to_int32_rows(P):
    # 3 cells per axis with 2,000 particles: every stencil holds all of them
    # (> 1024 candidates), so every cell takes the int32-row path
    rng = np.random.Generator(np.random.PCG64(7))
    L = W.f32(3 * 2.8 * 1.01)
    N = 2000
    r = np.zeros((N, 4), np.float32)
    r[:, :3] = W.uniform_box_positions(N, L, 3, rng)
    r[:, 3] = 1.0   # unit diameters
    fa, _, _ = _forces(P, r, L, P.soft_pot(), 2.5, cap=512, skin=0.3)
    fb, _, nl = _forces(P, r, L, P.soft_pot(), 2.5, cap=512, skin=0.3, local=True)
    assert list(nl.plan.ncell) == [3, 3, 3]
    np.testing.assert_array_equal(fa, fb)


def test_local_rows_mixed_blocks_fall_back_per_block(P):
    # 8 cells per axis; x-cells 0-5 hold 35 particles each, x-cells 6-7 hold
    # 10: block regions made only of dense cells exceed the 2,048 staged
    # particles and use their int32 rows, the others their local rows, while
    # every stencil stays under the 1,024 candidates the build stages
    rng = np.random.Generator(np.random.PCG64(11))
    nc, rl = 8, 2.8
    L = W.f32(nc * rl * 1.01)
    w = L / nc
    pts = []
    for cz in range(nc):
        for cy in range(nc):
            for cx in range(nc):
                k = 35 if cx < 6 else 10
                u = rng.uniform(0.05, 0.95, size=(k, 3))
                pts.append((np.array([cx, cy, cz]) + u) * w)
    x = np.concatenate(pts)
    x = x[rng.permutation(x.shape[0])]
    r = np.zeros((x.shape[0], 4), np.float32)
    r[:, :3] = x.astype(np.float32)
    r[:, 3] = 1.0
    fa, Ea, _ = _forces(P, r, L, P.soft_pot(), 2.5, cap=256)
    fb, Eb, nl = _forces(P, r, L, P.soft_pot(), 2.5, cap=256, local=True)
    assert list(nl.plan.ncell) == [nc] * 3
    np.testing.assert_array_equal(fa, fb)
    assert abs(Ea - Eb) <= 1e-7 * max(abs(Ea), 1.0)


@pytest.mark.parametrize("use_graph", [False, True])
def test_local_rows_nve_trajectory_bitwise(P, use_graph):
    import torch
    c = W.lj_small()
    out = []
    for local in (False, True):
        s = P.md_space_periodic(3, [c.L] * 3)
        nl = P.NeighborList(s, c.N, 2.5, 0.3, 128, local_rows=local)
        rd, vd = to_dev(c.r, torch.float32), to_dev(c.v, torch.float32)
        f = torch.zeros_like(rd)
        st = status_word()
        pot = P.lj_pot()
        PE = torch.zeros(80, dtype=torch.float64, device=dev())
        KE = torch.zeros_like(PE)
        nl.build(rd, st)
        P.md_energy_forces(s, pot, rd, nl.plan, f, None, st)
        P.md_integrate_nve(s, pot, rd, vd, f, 1.0, c.dt, 80, nl.plan, PE, KE, use_graph, st)
        torch.cuda.synchronize()
        assert P.md_status_poll(st) == 0
        assert nl.stats()[0] >= 3
        out.append((rd.cpu().numpy(), vd.cpu().numpy(), f.cpu().numpy(), PE.cpu().numpy(), KE.cpu().numpy()))
    (ra, va, fa, PEa, KEa), (rb, vb, fb, PEb, KEb) = out
    np.testing.assert_array_equal(ra, rb)
    np.testing.assert_array_equal(va, vb)
    np.testing.assert_array_equal(fa, fb)
    # energies are summed over a different particle-to-thread map (FP32
    # partial sums per thread)
    np.testing.assert_allclose(PEa, PEb, rtol=1e-7)
    np.testing.assert_allclose(KEa, KEb, rtol=1e-7)


def test_local_rows_flag_rules(P):
    s = P.md_space_periodic(3, [20.0] * 3)
    nb = P.md_nbr_plan(s, 1000, 2.5, 0.3, 128)
    base = int(nb.ws_bytes)
    P.md_nbr_set_flags(nb, P.MD_NBR_LOCAL_ROWS)
    assert int(nb.ws_bytes) >= base + 1000 * 128 * 2
    with pytest.raises(P.MDError):
        P.md_nbr_set_flags(nb, P.MD_NBR_LOCAL_ROWS | P.MD_NBR_CANONICAL)
