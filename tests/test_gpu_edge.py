"""Degenerate inputs on the GPU path (Sec. 3.2-3.3): a single particle, an
isolated dimer against its closed form, a dilute gas whose particles have
no partners, and a zero-step integration, each through the C ABI."""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import dev, status_word, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1912_04232_b300 as P
    return P


def _system(P, r, L, cap=32):
    s = P.md_space_periodic(3, [L] * 3)
    nl = P.NeighborList(s, r.shape[0], 2.5, 0.3, cap)
    return s, nl


def test_single_particle_has_no_partners_and_flies_freely(P):
    import torch
    L = 10.0
    r0 = np.array([[1.0, 2.0, 3.0, 0.0]], np.float32)
    v0 = np.array([[0.7, -0.4, 0.25, 0.0]], np.float32)
    s, nl = _system(P, r0, L)
    r, v = to_dev(r0), to_dev(v0)
    f = torch.ones_like(r)
    E = torch.zeros(1, dtype=torch.float64, device=dev())
    st = status_word()
    nl.build(r, st)
    P.md_energy_forces(s, P.lj_pot(), r, nl.plan, f, E, st)
    torch.cuda.synchronize()
    assert nl.cnt.cpu().numpy()[0] == 0
    assert np.all(f.cpu().numpy() == 0.0) and E.item() == 0.0
    PE = torch.zeros(200, dtype=torch.float64, device=dev())
    P.md_integrate_nve(s, P.lj_pot(), r, v, f, 1.0, 0.005, 200, nl.plan, PE, None, True, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    x = r.cpu().numpy()[0, :3].astype(np.float64)
    want = np.mod(r0[0, :3] + 200 * 0.005 * v0[0, :3].astype(np.float64), L)
    np.testing.assert_allclose(x, want, rtol=0, atol=5e-5)
    np.testing.assert_array_equal(v.cpu().numpy(), v0)
    assert np.all(PE.cpu().numpy() == 0.0)


def test_isolated_dimer_matches_closed_form(P):
    import torch
    L, d = 12.0, 1.3
    r0 = np.array([[5.0, 5.0, 5.0, 0.0], [5.0 + d, 5.0, 5.0, 0.0]], np.float32)
    s, nl = _system(P, r0, L)
    r = to_dev(r0)
    f = torch.zeros_like(r)
    E = torch.zeros(1, dtype=torch.float64, device=dev())
    st = status_word()
    nl.build(r, st)
    P.md_energy_forces(s, P.lj_pot(), r, nl.plan, f, E, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    # u(r) = 4 (r^-12 - r^-6) - u_c, F on particle 0 along -x: u'(r)
    dd = float(np.float32(5.0 + d) - np.float32(5.0))
    uc = 4.0 * (2.5 ** -12 - 2.5 ** -6)
    u = 4.0 * (dd ** -12 - dd ** -6) - uc
    du = 4.0 * (-12 * dd ** -13 + 6 * dd ** -7)
    fo = f.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(E.item(), u, rtol=1e-6)
    np.testing.assert_allclose(fo[0, 0], du, rtol=1e-5)
    np.testing.assert_allclose(fo[1, 0], -du, rtol=1e-5)
    assert np.all(fo[:, 1:3] == 0.0)
    np.testing.assert_allclose(fo[:, 3], [u / 2, u / 2], rtol=1e-6)


def test_dilute_gas_has_no_partners(P):
    import torch
    # 27 particles on a cubic grid of spacing 3.2 > r_list = 2.8
    g = np.arange(3) * 3.2 + 0.5
    pts = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    r0 = np.zeros((27, 4), np.float32)
    r0[:, :3] = pts
    s, nl = _system(P, r0, 9.6)
    r = to_dev(r0)
    f = torch.ones_like(r)
    st = status_word()
    nl.build(r, st)
    P.md_energy_forces(s, P.lj_pot(), r, nl.plan, f, None, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    assert np.all(nl.cnt.cpu().numpy() == 0)
    assert np.all(f.cpu().numpy() == 0.0)
    cnt_o, _ = O.neighbor_list(r0, 9.6, float(np.float32(2.5) + np.float32(0.3)), dim=3)
    assert np.all(cnt_o == 0)


def test_zero_steps_leave_the_state_untouched(P):
    import torch
    rng = np.random.default_rng(4)
    r0 = np.zeros((64, 4), np.float32)
    r0[:, :3] = rng.uniform(0, 8.0, (64, 3))
    v0 = np.zeros_like(r0)
    v0[:, :3] = rng.normal(0, 1, (64, 3))
    s, nl = _system(P, r0, 8.0, cap=64)
    r, v = to_dev(r0), to_dev(v0)
    f = torch.zeros_like(r)
    st = status_word()
    nl.build(r, st)
    P.md_integrate_nve(s, P.lj_pot(), r, v, f, 1.0, 0.005, 0, nl.plan, None, None, True, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    np.testing.assert_array_equal(r.cpu().numpy(), r0)
    np.testing.assert_array_equal(v.cpu().numpy(), v0)
