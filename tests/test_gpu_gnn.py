"""GPU parity of the graph-network potential (Sec. 3.2.4 / 4.1 reading)
against the FP64 autograd oracle: per-atom energies, total energy and
forces on disordered silicon for several widths and step counts (including
vacancies, so the atom count is ragged against the warps of a block);
sampled atoms of the 64,000-atom deployment system against oracle clusters
(exact by locality: E_i needs the atoms within T r_c of i, F_k those within
2 T r_c of k); energy conservation in NVE; a Nose-Hoover run."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import dev, force_error, status_word, to_dev
from oracle import gnn as G

pytestmark = pytest.mark.gpu

RC = 3.77
SKIN = 0.3
CAP = 48


@pytest.fixture(scope="module")
def P():
    import paper_1912_04232_b300 as P
    return P


def _si(n_side, seed=0, jitter=0.15, vacancies=0):
    si = W.sw_silicon(n_side, T_K=0, jitter=jitter, seed=seed)
    r = si.r
    if vacancies:
        keep = np.sort(np.random.Generator(np.random.PCG64(seed + 100)).permutation(r.shape[0])[vacancies:])
        r = np.ascontiguousarray(r[keep])
    return r, si.L


def _gpu(P, r, L, p32, H, T, E_out=True):
    import torch
    s = P.md_space_periodic(3, [L] * 3)
    nl = P.NeighborList(s, r.shape[0], RC, SKIN, CAP)
    rd = to_dev(r, torch.float32)
    st = status_word()
    nl.build(rd, st)
    m = P.GNNModel(to_dev(p32, torch.float32), r.shape[0], CAP, H, T, RC)
    f = torch.zeros((r.shape[0], 4), dtype=torch.float32, device=dev())
    E = torch.zeros(1, dtype=torch.float64, device=dev()) if E_out else None
    P.md_energy_forces(s, m.pot, rd, nl.plan, f, E, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    return f.cpu().numpy(), (E.item() if E_out else None)


@pytest.mark.parametrize("H,T,n_side,vac", [(64, 2, 4, 0), (64, 2, 4, 3), (32, 1, 4, 5), (32, 3, 3, 1),
                                            (64, 4, 3, 0), (64, 2, 6, 7)])
def test_energy_forces_match_oracle(P, H, T, n_side, vac):
    r, L = _si(n_side, seed=H + T, vacancies=vac)
    p32 = W.gnn_params(H, T, seed=T, out_scale=1.0)
    f, E = _gpu(P, r, L, p32, H, T)
    Eo, Eio, Fo = G.energy_forces(r[:, :3].astype(np.float64), float(L), p32.astype(np.float64), H, T, RC)
    scale = np.abs(Eio).max()
    assert np.abs(f[:, 3] - Eio).max() <= 2e-5 * scale
    assert abs(E - Eo) <= 1e-5 * np.abs(Eio).sum()
    assert force_error(f, Fo) <= 1e-4


def _cluster(r, L, k, radius):
    """Atoms within `radius` of atom k as unwrapped coordinates around it
    (index 0 is k)."""
    d = r[:, :3].astype(np.float64) - r[k, :3].astype(np.float64)
    d -= L * np.round(d / L)
    dist = np.sqrt((d ** 2).sum(1))
    idx = np.concatenate([[k], np.nonzero((dist < radius) & (np.arange(r.shape[0]) != k))[0]])
    return idx, d[idx] + 1000.0


def test_deployment_size_sampled_atoms(P):
    # 64,000 atoms, the bench's model (H = 64, T = 2)
    H, T = 64, 2
    r, L = _si(20, seed=11, jitter=0.15)
    p32 = W.gnn_params(H, T, seed=0, out_scale=0.1)
    p64 = p32.astype(np.float64)
    f, E = _gpu(P, r, L, p32, H, T)
    assert np.all(np.isfinite(f))
    rng = np.random.Generator(np.random.PCG64(5))
    for k in rng.choice(r.shape[0], 6, replace=False):
        idx, x = _cluster(r, L, k, 2 * T * RC + 0.5)
        _, Ei, F = G.energy_forces(x, 1.0e6, p64, H, T, RC)
        # E_k needs T r_c around k, F_k 2 T r_c
        assert abs(f[k, 3] - Ei[0]) <= 2e-5 * max(abs(Ei[0]), 1e-3)
        fr = np.linalg.norm(F[0])
        assert np.linalg.norm(f[k, :3] - F[0]) <= 1e-4 * max(fr, 1e-2)
    # translation invariance: the net force vanishes up to FP32 rounding
    assert np.abs(f[:, :3].sum(0)).max() <= 1e-3 * np.abs(f[:, :3]).max() * np.sqrt(r.shape[0])


def test_nve_conserves_energy(P):
    import torch
    H, T = 64, 2
    r, L = _si(4, seed=3, jitter=0.1)
    si = W.sw_silicon(4, T_K=600.0, seed=3)
    p32 = W.gnn_params(H, T, seed=1, out_scale=0.3)
    s = P.md_space_periodic(3, [L] * 3)
    nl = P.NeighborList(s, r.shape[0], RC, SKIN, CAP)
    rd = to_dev(r, torch.float32)
    vd = to_dev(si.v, torch.float32)
    st = status_word()
    nl.build(rd, st)
    m = P.GNNModel(to_dev(p32, torch.float32), r.shape[0], CAP, H, T, RC)
    f = torch.zeros_like(rd)
    n = 400
    PE = torch.zeros(n + 1, dtype=torch.float64, device=dev())
    KE = torch.zeros(n + 1, dtype=torch.float64, device=dev())
    mass = 28.0855 * 103.6427
    P.md_energy_forces(s, m.pot, rd, nl.plan, f, None, st)
    P.md_integrate_nve(s, m.pot, rd, vd, f, mass, 0.5, n, nl.plan, PE, KE, True, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    pe = PE.cpu().numpy()[1:n]
    ke = KE.cpu().numpy()[1:n]
    Et = pe + ke
    # the total drifts by far less than the potential energy exchanges
    assert np.abs(Et - Et[0]).max() <= 2e-3 * ke.mean()
    assert np.ptp(pe) > 5 * np.abs(Et - Et[0]).max()


def test_nose_hoover_run(P):
    import torch
    H, T = 64, 2
    r, L = _si(5, seed=4, jitter=0.1)
    si = W.sw_silicon(5, T_K=800.0, seed=4)
    p32 = W.gnn_params(H, T, seed=2, out_scale=0.3)
    s = P.md_space_periodic(3, [L] * 3)
    nl = P.NeighborList(s, r.shape[0], RC, SKIN, CAP)
    rd = to_dev(r, torch.float32)
    vd = to_dev(si.v, torch.float32)
    st = status_word()
    nl.build(rd, st)
    m = P.GNNModel(to_dev(p32, torch.float32), r.shape[0], CAP, H, T, RC)
    f = torch.zeros_like(rd)
    n, dt, kT = 200, 0.5, 8.617333262e-5 * 800.0
    th = torch.zeros(P.md_nhc_state_doubles(3), dtype=torch.float64, device=dev())
    KE = torch.zeros(n + 1, dtype=torch.float64, device=dev())
    Hx = torch.zeros(n + 1, dtype=torch.float64, device=dev())
    mass = 28.0855 * 103.6427
    P.md_energy_forces(s, m.pot, rd, nl.plan, f, None, st)
    P.md_integrate_nhc(s, m.pot, rd, vd, f, mass, dt, kT, 100.0 * dt, 3, n, nl.plan, th, True, None, KE, Hx, True,
                       st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    h = Hx.cpu().numpy()[1:n]
    ke = KE.cpu().numpy()[1:n]
    assert np.all(np.isfinite(h))
    # the extended energy is conserved to well below the kinetic energy
    assert np.abs(h - h[0]).max() <= 5e-3 * ke.mean()


def test_group_sizes_bitwise_equal(P):
    # atoms per warp change only which warp does the work, not the order of
    # any sum: forces and energies are bit-for-bit the same
    H, T = 64, 2
    r, L = _si(4, seed=21, jitter=0.15, vacancies=5)
    p32 = W.gnn_params(H, T, seed=3, out_scale=1.0)
    ref, Eref = _gpu(P, r, L, p32, H, T)          # default: 4 atoms per warp
    try:
        for G in (1, 2, 8):
            P.md_gnn_set_group(G)
            f, E = _gpu(P, r, L, p32, H, T)
            np.testing.assert_array_equal(f, ref)
            assert E == Eref
    finally:
        P.md_gnn_set_group(4)
    with pytest.raises(P.MDError):
        P.md_gnn_set_group(3)


def _readout_norm(p32, H, T):
    """|w| of the decoder read-out (the block before the final bias c)."""
    return float(np.linalg.norm(p32[-1 - H:-1]))


@pytest.fixture
def tensor_cores(P):
    P.md_gnn_set_tensor_cores(True)
    yield
    P.md_gnn_set_tensor_cores(False)


@pytest.mark.parametrize("T,n_side,vac", [(2, 4, 0), (2, 4, 7), (3, 3, 2), (1, 5, 0)])
def test_tensor_cores_match_oracle(P, tensor_cores, T, n_side, vac):
    # weights BF16-representable (the model the tensor cores hold exactly),
    # activations split into two BF16 parts (about 2^-17 relative), FP32
    # accumulation: the FP32 bar within a factor of a few
    H = 64
    r, L = _si(n_side, seed=30 + T, vacancies=vac)
    p32 = W.gnn_params(H, T, seed=T + 7, out_scale=1.0, bf16=True)
    f, E = _gpu(P, r, L, p32, H, T)
    Eo, Eio, Fo = G.energy_forces(r[:, :3].astype(np.float64), float(L), p32.astype(np.float64), H, T, RC)
    wn = _readout_norm(p32, H, T)
    ee = np.abs(f[:, 3] - Eio).max() / wn
    fe = force_error(f, Fo)
    assert ee <= 2e-5, ee
    assert abs(E - Eo) <= 2e-5 * wn * r.shape[0]
    assert fe <= 5e-4, fe


def test_tensor_cores_deployment_size(P, tensor_cores):
    H, T = 64, 2
    r, L = _si(20, seed=11, jitter=0.15)
    p32 = W.gnn_params(H, T, seed=0, out_scale=0.1, bf16=True)
    f, E = _gpu(P, r, L, p32, H, T)
    P.md_gnn_set_tensor_cores(False)
    f32, E32 = _gpu(P, r, L, p32, H, T)
    assert force_error(f, f32) <= 5e-4
    wn = _readout_norm(p32, H, T)
    assert np.abs(f[:, 3] - f32[:, 3]).max() <= 2e-5 * wn
    assert abs(E - E32) <= 2e-5 * wn * r.shape[0]
    # sampled atoms against the oracle (exact by locality, as above)
    rng = np.random.Generator(np.random.PCG64(6))
    for k in rng.choice(r.shape[0], 3, replace=False):
        idx, x = _cluster(r, L, k, 2 * T * RC + 0.5)
        _, Ei, F = G.energy_forces(x, 1.0e6, p32.astype(np.float64), H, T, RC)
        assert np.linalg.norm(f[k, :3] - F[0]) <= 5e-4 * max(np.linalg.norm(F[0]), 1e-2)


def test_tensor_cores_unrepresentable_weights_stay_close(P, tensor_cores):
    # weights that are not BF16-representable are rounded once when staged:
    # the tensor-core model then differs from the FP32 one by that rounding
    H, T = 64, 2
    r, L = _si(4, seed=40, jitter=0.4)
    p32 = W.gnn_params(H, T, seed=9, out_scale=1.0)
    f, E = _gpu(P, r, L, p32, H, T)
    _, Eio, Fo = G.energy_forces(r[:, :3].astype(np.float64), float(L), p32.astype(np.float64), H, T, RC)
    assert np.abs(f[:, 3] - Eio).max() <= 5e-3 * _readout_norm(p32, H, T)
    assert force_error(f, Fo) <= 5e-2


def test_tensor_cores_nose_hoover_run(P, tensor_cores):
    test_nose_hoover_run(P)


def test_switching_kernels_recaptures_the_md_graph(P):
    # the cached MD graph is keyed by the kernel switches too: the same
    # buffers run with tensor cores after an FP32 run give the tensor-core
    # trajectory, not a replay of the FP32 graph
    import torch
    H, T = 64, 2
    r0, L = _si(4, seed=50, jitter=0.1)
    v0 = W.sw_silicon(4, T_K=600.0, seed=50).v
    p32 = W.gnn_params(H, T, seed=4, out_scale=0.3, bf16=True)
    s = P.md_space_periodic(3, [L] * 3)
    nl = P.NeighborList(s, r0.shape[0], RC, SKIN, CAP)
    m = P.GNNModel(to_dev(p32, torch.float32), r0.shape[0], CAP, H, T, RC)
    rd, vd = to_dev(r0, torch.float32), to_dev(v0, torch.float32)
    f = torch.zeros_like(rd)
    st = status_word()

    def run(tc, r_buf, v_buf):
        P.md_gnn_set_tensor_cores(tc)
        r_buf.copy_(to_dev(r0, torch.float32))
        v_buf.copy_(to_dev(v0, torch.float32))
        nl.build(r_buf, st)
        P.md_energy_forces(s, m.pot, r_buf, nl.plan, f, None, st)
        P.md_integrate_nve(s, m.pot, r_buf, v_buf, f, 28.0855 * 103.6427, 0.5, 20, nl.plan, None, None, True, st)
        torch.cuda.synchronize()
        return r_buf.cpu().numpy().copy()

    try:
        a = run(False, rd, vd)
        b = run(True, rd, vd)
        c = run(True, torch.empty_like(rd), torch.empty_like(vd))
    finally:
        P.md_gnn_set_tensor_cores(False)
    assert P.md_status_poll(st) == 0
    np.testing.assert_array_equal(b, c)
    assert not np.array_equal(a, b)
