"""GPU parity of Nose-Hoover chain NVT (Sec. 3.3.1; Martyna, Klein,
Tuckerman 1992) against the FP64 oracle: LJ trajectories, energy series
and the conserved extended energy, the chain state, graph = host launches,
continuation across calls, and Stillinger-Weber silicon at 1000 K."""
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


def _nhc_gpu(P, r, v, L, pot, rc, skin, mass, dt, kT, tau, M, nsteps, use_graph=True, chunks=None, cap=128):
    import torch
    s = P.md_space_periodic(3, [L] * 3)
    nl = P.NeighborList(s, r.shape[0], rc, skin, cap)
    rd, vd = to_dev(r, torch.float32), to_dev(v, torch.float32)
    f = torch.zeros_like(rd)
    th = torch.zeros(P.md_nhc_state_doubles(M), dtype=torch.float64, device=dev())
    st = status_word()
    nl.build(rd, st)
    P.md_energy_forces(s, pot, rd, nl.plan, f, None, st)
    PE, KE, H = [], [], []
    reset = True
    for c in (chunks or [nsteps]):
        pe = torch.zeros(c, dtype=torch.float64, device=dev())
        ke, h = torch.zeros_like(pe), torch.zeros_like(pe)
        P.md_integrate_nhc(s, pot, rd, vd, f, mass, dt, kT, tau, M, c, nl.plan, th, reset, pe, ke, h, use_graph, st)
        reset = False
        PE.append(pe)
        KE.append(ke)
        H.append(h)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    cat = lambda xs: torch.cat(xs).cpu().numpy()
    return rd.cpu().numpy(), vd.cpu().numpy(), cat(PE), cat(KE), cat(H), th.cpu().numpy(), nl


def _lj(seed=0):
    return W.lj_small(seed)


@pytest.mark.parametrize("use_graph", [False, True])
def test_nhc_lj_matches_oracle(P, use_graph):
    c = _lj()
    n, kT, tau, M = 60, 1.5, 0.25, 3
    x, v, PE, KE, H, th, nl = _nhc_gpu(P, c.r, c.v, c.L, P.lj_pot(), 2.5, 0.3, 1.0, c.dt, kT, tau, M, n,
                                       use_graph=use_graph)
    xo, vo, PEo, KEo, Ho, (xio, wo) = O.nhc(c.r, c.v, c.L, "lj", dt=c.dt, kT=kT, tau=tau, M=M, nsteps=n)
    d = x[:, :3] - xo
    d -= c.L * np.round(d / c.L)
    assert np.abs(d).max() < 5e-4
    assert np.abs(v[:, :3] - vo).max() < 5e-3
    np.testing.assert_allclose(PE, PEo[1:], rtol=5e-5)
    np.testing.assert_allclose(KE, KEo[1:], rtol=5e-5)
    np.testing.assert_allclose(H, Ho[1:], rtol=5e-5)
    np.testing.assert_allclose(th[:M], xio, rtol=1e-3, atol=1e-7)
    np.testing.assert_allclose(th[M:2 * M], wo, rtol=1e-3, atol=1e-6)
    assert nl.stats()[0] >= 2


def test_nhc_graph_equals_host_launches_bitwise(P):
    c = _lj(1)
    a = _nhc_gpu(P, c.r, c.v, c.L, P.lj_pot(), 2.5, 0.3, 1.0, c.dt, 1.2, 0.3, 4, 70, use_graph=False)
    b = _nhc_gpu(P, c.r, c.v, c.L, P.lj_pot(), 2.5, 0.3, 1.0, c.dt, 1.2, 0.3, 4, 70, use_graph=True)
    for x, y in zip(a[:6], b[:6]):
        np.testing.assert_array_equal(x, y)


def test_nhc_continuation_is_bitwise(P):
    c = _lj(2)
    a = _nhc_gpu(P, c.r, c.v, c.L, P.lj_pot(), 2.5, 0.3, 1.0, c.dt, 1.2, 0.3, 3, 60)
    b = _nhc_gpu(P, c.r, c.v, c.L, P.lj_pot(), 2.5, 0.3, 1.0, c.dt, 1.2, 0.3, 3, 60, chunks=[25, 1, 34])
    for x, y in zip(a[:6], b[:6]):
        np.testing.assert_array_equal(x, y)


def test_nhc_heavy_thermostat_is_nve(P):
    # tau -> infinity: the chain stays at rest and the step is velocity Verlet
    import torch
    c = _lj(3)
    n = 40
    x, v, PE, KE, H, th, _ = _nhc_gpu(P, c.r, c.v, c.L, P.lj_pot(), 2.5, 0.3, 1.0, c.dt, 1.0, 1e9, 3, n)
    xo, vo, PEo, KEo = O.nve(c.r, c.v, c.L, "lj", dt=c.dt, nsteps=n)
    np.testing.assert_allclose(PE, PEo[1:], rtol=5e-5)
    np.testing.assert_allclose(KE, KEo[1:], rtol=5e-5)


@pytest.mark.parametrize("lists", [False, True])
def test_nhc_sw_silicon_1000K(P, lists):
    # the paper's NVT deployment setting (SW silicon, 1000 K, dt = 1 fs), in
    # the one-kernel form and on partner lists
    si = W.sw_silicon(4, T_K=1000.0, jitter=0.05, seed=5)
    mass = O.SW_MASS_AMU * O.AMU_A2_FS2_EV
    kT = W.KB_EV * 1000.0
    rc = float(O.SW_SI[2] * O.SW_SI[1])
    n, tau, M = 50, 100.0, 3
    pot = P.sw_pot(O.SW_SI, N=si.N) if lists else P.sw_pot(O.SW_SI)
    x, v, PE, KE, H, th, _ = _nhc_gpu(P, si.r, si.v, si.L, pot, rc, 0.5, mass, 1.0, kT, tau, M, n, cap=64)
    xo, vo, PEo, KEo, Ho, (xio, wo) = O.nhc(si.r, si.v, si.L, "sw", mass=mass, dt=1.0, kT=kT, tau=tau, M=M,
                                           nsteps=n)
    np.testing.assert_allclose(PE, PEo[1:], rtol=1e-5)
    np.testing.assert_allclose(KE, KEo[1:], rtol=2e-4)
    np.testing.assert_allclose(H, Ho[1:], rtol=1e-5)


def test_nhc_rejects_bad_arguments(P):
    import torch
    c = _lj()
    s = P.md_space_periodic(3, [c.L] * 3)
    nl = P.NeighborList(s, c.N, 2.5, 0.3, 128)
    z = torch.zeros((c.N, 4), dtype=torch.float32, device=dev())
    th = torch.zeros(64, dtype=torch.float64, device=dev())
    with pytest.raises(P.MDError):
        P.md_integrate_nhc(s, P.lj_pot(), z, z.clone(), z.clone(), 1.0, 0.005, 1.0, 0.5, 9, 1, nl.plan, th)
    with pytest.raises(P.MDError):
        P.md_integrate_nhc(s, P.lj_pot(), z, z.clone(), z.clone(), 1.0, 0.005, -1.0, 0.5, 3, 1, nl.plan, th)


def test_nhc_samples_the_canonical_kinetic_energy(P):
    # a long NVT run of the N = 4,096 LJ fluid at kT = 1.5 from its T = 1
    # start (tau = 50 dt): over the second half the mean temperature is the
    # target, and the kinetic energy fluctuates as in the canonical ensemble,
    # Var(K) / <K>^2 = 2 / g with g = 3N (a rescaling thermostat would give
    # no fluctuation, a weakly coupled one too little); H' stays conserved
    c = _lj(2)
    n, kT, tau, M = 6000, 1.5, 0.25, 3
    x, v, PE, KE, H, th, nl = _nhc_gpu(P, c.r, c.v, c.L, P.lj_pot(), 2.5, 0.3, 1.0, c.dt, kT, tau, M, n)
    g = 3 * c.N
    K = KE[n // 2:]
    assert abs(2.0 * K.mean() / (g * kT) - 1.0) < 0.02
    rel = K.std() / K.mean()
    assert 0.7 * np.sqrt(2.0 / g) < rel < 1.4 * np.sqrt(2.0 / g), (rel, np.sqrt(2.0 / g))
    assert np.abs(H - H[0]).max() / c.N < 5e-3
