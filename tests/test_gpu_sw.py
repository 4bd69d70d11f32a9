"""GPU parity: Stillinger-Weber three-body forces (Sec. 3.3.2) and NVE with
them, through the C ABI, against the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import dev, force_error, status_word, to_dev

pytestmark = pytest.mark.gpu

RC = float(O.SW_SI[2] * O.SW_SI[1])     # a * sigma = 3.77118 A
SKIN = 0.5
MASS = O.SW_MASS_AMU * O.AMU_A2_FS2_EV   # eV fs^2 / A^2


@pytest.fixture(scope="module")
def P():
    import paper_1912_04232_b300 as P
    return P


def _forces(P, r, L, cap=64, lists=False):
    import torch
    s = P.md_space_periodic(3, [L] * 3)
    nl = P.NeighborList(s, r.shape[0], RC, SKIN, cap)
    rd = to_dev(r, torch.float32)
    st = status_word()
    nl.build(rd, st)
    f = torch.zeros((r.shape[0], 4), dtype=torch.float32, device=dev())
    E = torch.zeros(1, dtype=torch.float64, device=dev())
    pot = P.sw_pot(O.SW_SI, N=r.shape[0]) if lists else P.sw_pot(O.SW_SI)
    P.md_energy_forces(s, pot, rd, nl.plan, f, E, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    return f.cpu().numpy(), E.item()


@pytest.mark.parametrize("lists", [False, True])
@pytest.mark.parametrize("n_side,jitter,seed", [(2, 0.2, 7), (4, 0.15, 1), (4, 0.35, 2), (3, 0.25, 3), (20, 0.2, 4)])
def test_sw_forces_energy_match_oracle(P, n_side, jitter, seed, lists):
    # lists: the two-kernel form (partners inside a*sigma stored first)
    si = W.sw_silicon(n_side, T_K=0, jitter=jitter, seed=seed)
    f, E = _forces(P, si.r, si.L, lists=lists)
    U, F, e = O.sw(si.r, si.L)
    assert force_error(f, F) <= 1e-4
    np.testing.assert_allclose(f[:, 3], e, rtol=0, atol=2e-5 * np.abs(e).max())
    assert abs(E - U) <= 1e-5 * abs(U)


def test_sw_partner_lists_give_the_same_terms(P):
    # the same triplets with the same FP32 vectors: the two forms differ
    # only by the order in which each atom's terms are summed
    si = W.sw_silicon(6, T_K=0, jitter=0.3, seed=5)
    f0, E0 = _forces(P, si.r, si.L, lists=False)
    f1, E1 = _forces(P, si.r, si.L, lists=True)
    scale = np.abs(f0[:, :3]).max()
    assert np.abs(f1[:, :3] - f0[:, :3]).max() <= 2e-6 * scale
    np.testing.assert_allclose(f1[:, 3], f0[:, 3], rtol=0, atol=2e-6 * np.abs(f0[:, 3]).max())
    assert abs(E1 - E0) <= 1e-6 * abs(E0)


def test_sw_diamond_cohesive_energy(P):
    si = W.sw_silicon(4, T_K=0)
    f, E = _forces(P, si.r, si.L)
    assert abs(E / si.N - (-4.3366)) < 2e-4
    assert np.abs(f[:, :3]).max() < 1e-3


@pytest.mark.parametrize("lists", [False, True])
def test_sw_nve_short_trajectory_matches_oracle(P, lists):
    import torch
    si = W.sw_silicon(4, T_K=1500, jitter=0.1, seed=7)
    s = P.md_space_periodic(3, [si.L] * 3)
    nl = P.NeighborList(s, si.N, RC, SKIN, 64)
    rd = to_dev(si.r, torch.float32)
    vd = to_dev(si.v, torch.float32)
    f = torch.zeros((si.N, 4), dtype=torch.float32, device=dev())
    st = status_word()
    pot = P.sw_pot(O.SW_SI, N=si.N) if lists else P.sw_pot(O.SW_SI)
    nl.build(rd, st)
    P.md_energy_forces(s, pot, rd, nl.plan, f, None, st)
    n, dt = 20, 1.0
    PE = torch.zeros(n, dtype=torch.float64, device=dev())
    KE = torch.zeros(n, dtype=torch.float64, device=dev())
    P.md_integrate_nve(s, pot, rd, vd, f, MASS, dt, n, nl.plan, PE, KE, True, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    ro, vo, PEo, KEo = O.nve(si.r, si.v, si.L, "sw", mass=MASS, dt=dt, nsteps=n)
    d = rd.cpu().numpy()[:, :3] - ro
    d -= si.L * np.round(d / si.L)
    assert np.abs(d).max() < 1e-4
    np.testing.assert_allclose(PE.cpu().numpy(), PEo[1:], rtol=1e-5)
    np.testing.assert_allclose(KE.cpu().numpy(), KEo[1:], rtol=1e-4)


def _langevin(P, si, n, gamma, kT, seed, step0=0, lists=False):
    import torch
    s = P.md_space_periodic(3, [si.L] * 3)
    nl = P.NeighborList(s, si.N, RC, SKIN, 64)
    rd = to_dev(si.r, torch.float32)
    vd = to_dev(si.v, torch.float32)
    f = torch.zeros((si.N, 4), dtype=torch.float32, device=dev())
    st = status_word()
    pot = P.sw_pot(O.SW_SI, N=si.N) if lists else P.sw_pot(O.SW_SI)
    nl.build(rd, st)
    P.md_energy_forces(s, pot, rd, nl.plan, f, None, st)
    PE = torch.zeros(n, dtype=torch.float64, device=dev())
    KE = torch.zeros(n, dtype=torch.float64, device=dev())
    P.md_integrate_langevin(s, pot, rd, vd, f, MASS, 1.0, gamma, kT, seed, step0, n, nl.plan, PE, KE, True, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    return rd.cpu().numpy(), vd.cpu().numpy(), PE.cpu().numpy(), KE.cpu().numpy()


@pytest.mark.parametrize("lists", [False, True])
def test_langevin_trajectory_matches_oracle_noise_bit_for_bit(P, lists):
    # same Philox counters on both sides: the FP32 run follows the FP64 run
    si = W.sw_silicon(4, T_K=1200, jitter=0.1, seed=11)
    kT = W.KB_EV * 1200.0
    n = 20
    r, v, PE, KE = _langevin(P, si, n, 0.01, kT, seed=1234567, step0=40, lists=lists)
    ro, vo, PEo, KEo = O.langevin(si.r, si.v, si.L, "sw", mass=MASS, dt=1.0, gamma=0.01, kT=kT, seed=1234567,
                                  step0=40, nsteps=n)
    d = r[:, :3] - ro
    d -= si.L * np.round(d / si.L)
    assert np.abs(d).max() < 1e-4
    assert np.abs(v[:, :3] - vo).max() < 1e-4
    np.testing.assert_allclose(PE, PEo, rtol=1e-5)
    np.testing.assert_allclose(KE, KEo, rtol=1e-4)


def test_langevin_thermalises_to_target_temperature(P):
    si = W.sw_silicon(4, T_K=0, jitter=0.05, seed=12)
    T = 900.0
    kT = W.KB_EV * T
    r, v, PE, KE = _langevin(P, si, 3000, 0.02, kT, seed=99)
    T_kin = 2.0 * KE[1000:].mean() / (3 * si.N * W.KB_EV)
    assert abs(T_kin - T) < 0.05 * T


@pytest.mark.parametrize("lists", [False, True])
def test_sw_more_partners_than_slots_is_reported(P, lists):
    # 40 atoms packed within 1.3 A of one point: each has about 39 partners
    # inside a*sigma, more than the 32 an atom keeps (one-kernel form and
    # partner lists alike); the list itself (cap 128) does not overflow
    import torch
    si = W.sw_silicon(3, T_K=0, jitter=0.0, seed=0)
    r = si.r.copy()
    rng = np.random.default_rng(5)
    d = rng.normal(size=(40, 3))
    d *= (1.3 * rng.uniform(0.2, 1.0, size=(40, 1)) ** (1 / 3)) / np.linalg.norm(d, axis=1, keepdims=True)
    r[:40, :3] = (np.float32(si.L / 2) + d).astype(np.float32)
    s = P.md_space_periodic(3, [si.L] * 3)
    nl = P.NeighborList(s, si.N, RC, 0.3, 128)
    rd = to_dev(r, torch.float32)
    st = status_word()
    nl.build(rd, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    f = torch.zeros((si.N, 4), dtype=torch.float32, device=dev())
    pot = P.sw_pot(O.SW_SI, N=si.N) if lists else P.sw_pot(O.SW_SI)
    P.md_energy_forces(s, pot, rd, nl.plan, f, None, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) & P.MD_ERR_NBR_OVERFLOW
