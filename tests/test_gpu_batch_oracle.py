"""GPU parity against the FP64 oracle for the batched-replica workload (the
paper's vmap over independent systems, Sec. 4.2) and for 3-D soft spheres
(Sec. 3.3.2): forces and energies of single 3-D soft-sphere systems, and a
sample of replicas taken from one batched launch -- the smallest LJ and
soft-sphere boxes (deduplicated stencils), a mid-size and the largest of
each kind -- compared element by element with the oracle, forces right
after the build and 20-step velocity-Verlet trajectories."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import dev, force_error, status_word, to_dev

pytestmark = pytest.mark.gpu

CAP = 128


@pytest.fixture(scope="module")
def P():
    import paper_1912_04232_b300 as P
    return P


def _soft_system(N, rho, seed, relax=0):
    rng = np.random.Generator(np.random.PCG64(seed))
    L = W.f32((N / rho) ** (1.0 / 3.0))
    r = np.zeros((N, 4), np.float32)
    r[:, :3] = W.uniform_box_positions(N, L, 3, rng)
    r[:, 3] = np.where(np.arange(N) < N // 2, 1.0, 1.4)
    return r, L


@pytest.mark.parametrize("tpp", [4, 8])
def test_soft_spheres_3d_forces_energies(P, tpp):
    # 50/50 diameters 1.0 / 1.4 in the w column, number density 0.8
    import torch
    r, L = _soft_system(3000, 0.8, 21)
    s = P.md_space_periodic(3, [L] * 3)
    nl = P.NeighborList(s, r.shape[0], 1.4, 0.3, CAP)
    rd = to_dev(r, torch.float32)
    st = status_word()
    f = torch.zeros_like(rd)
    E = torch.zeros(1, dtype=torch.float64, device=dev())
    nl.build(rd, st)
    P.md_set_pair_tpp(tpp)
    try:
        P.md_energy_forces(s, P.soft_pot(1.0, 2.0), rd, nl.plan, f, E, st)
        torch.cuda.synchronize()
    finally:
        P.md_set_pair_tpp(4)
    assert P.md_status_poll(st) == 0
    U, F, e = O.soft(r, r[:, 3].astype(np.float64), L, dim=3)
    fg = f.cpu().numpy()
    assert force_error(fg, F) <= 1e-4
    np.testing.assert_allclose(fg[:, 3], e, rtol=0, atol=2e-5 * np.abs(e).max())
    assert abs(E.item() - U) <= 1e-5 * abs(U)


def test_soft_spheres_3d_nve_vs_oracle(P):
    # 20 velocity-Verlet steps from a relaxed start (50 gradient-descent
    # steps), dt 0.01: positions, velocities and energies against FP64
    import torch
    r, L = _soft_system(2000, 0.8, 22)
    s = P.md_space_periodic(3, [L] * 3)
    nl = P.NeighborList(s, r.shape[0], 1.4, 0.3, CAP)
    rd = to_dev(r, torch.float32)
    st = status_word()
    f = torch.zeros_like(rd)
    nl.build(rd, st)
    P.md_minimize(s, P.soft_pot(), 0, 0.05, 50, rd, f, nl.plan, None, st)
    x = rd.cpu().numpy()
    x[:, :3] = np.mod(x[:, :3], np.float32(L)).astype(np.float32)
    x[:, :3][x[:, :3] >= np.float32(L)] = 0.0
    v = W.thermal_velocities(r.shape[0], 3, 1.0, 1.0, np.random.Generator(np.random.PCG64(5)))
    v4 = np.zeros((r.shape[0], 4), np.float32)
    v4[:, :3] = v
    rd = to_dev(x, torch.float32)
    vd = to_dev(v4, torch.float32)
    nl.build(rd, st)
    P.md_energy_forces(s, P.soft_pot(), rd, nl.plan, f, None, st)
    n = 20
    PE = torch.zeros(n, dtype=torch.float64, device=dev())
    KE = torch.zeros_like(PE)
    P.md_integrate_nve(s, P.soft_pot(), rd, vd, f, 1.0, 0.01, n, nl.plan, PE, KE, True, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    ro, vo, PEo, KEo = O.nve(x, v4, L, "soft", dt=0.01, nsteps=n, diam=x[:, 3].astype(np.float64))
    d = rd.cpu().numpy()[:, :3] - ro
    d -= L * np.round(d / L)
    assert np.abs(d).max() < 2e-4
    assert np.abs(vd.cpu().numpy()[:, :3] - vo).max() < 2e-3
    np.testing.assert_allclose(PE.cpu().numpy(), PEo[1:], rtol=2e-4, atol=1e-6 * r.shape[0])
    np.testing.assert_allclose(KE.cpu().numpy(), KEo[1:], rtol=2e-5)


def _desc(P, spec):
    d = P.md_replica_desc()
    d.N, d.L = spec.N, spec.L
    if spec.kind == "lj":
        pot = P.lj_pot()
        d.kind, d.eps, d.sigma, d.r_cut, d.e_shift = P.MD_LJ, pot.eps, pot.sigma, pot.r_cut, pot.e_shift
    else:
        d.kind, d.eps, d.alpha, d.r_cut = P.MD_SOFT_SPHERE, 1.0, 2.0, 1.4
    d.skin, d.dt, d.mass = 0.3, spec.dt, 1.0
    return d


def _initial(P, spec):
    """Starting state; soft-sphere replicas relaxed by 50 GD steps (library)."""
    import torch
    r, v = W.replica_initial(spec)
    if spec.kind == "soft":
        s = P.md_space_periodic(3, [spec.L] * 3)
        nl = P.NeighborList(s, spec.N, 1.4, 0.3, CAP)
        rd = to_dev(r, torch.float32)
        f = torch.zeros_like(rd)
        st = status_word()
        nl.build(rd, st)
        P.md_minimize(s, P.soft_pot(), 0, 0.05, 50, rd, f, nl.plan, None, st)
        x = rd.cpu().numpy()
        x[:, :3] = np.mod(x[:, :3], np.float32(spec.L)).astype(np.float32)
        x[:, :3][x[:, :3] >= np.float32(spec.L)] = 0.0
        r = x
    return r, v


def _oracle_forces(spec, r):
    if spec.kind == "lj":
        return O.lj(r, spec.L)
    return O.soft(r, r[:, 3].astype(np.float64), spec.L, dim=3)


def _sample(specs):
    """Smallest, a mid-size and the largest replica of each kind."""
    out = []
    for kind in ("lj", "soft"):
        idx = [k for k, sp in enumerate(specs) if sp.kind == kind]
        idx.sort(key=lambda k: specs[k].N)
        out += [idx[0], idx[len(idx) // 2], idx[-1]]
    return out


def test_batched_replicas_match_oracle(P):
    # the 512-replica plan (N log-uniform in [64, 8192], density in
    # [0.7, 0.95], half LJ, half soft spheres), advanced in one launch
    import torch
    specs = W.replica_plan(R=512, n_max=8192, seed=0)
    states = [_initial(P, sp) for sp in specs]
    sample = _sample(specs)
    # the smallest replicas have fewer than three cells per axis: their
    # stencils are deduplicated
    for k in sample[:1] + sample[3:4]:
        rl = 2.8 if specs[k].kind == "lj" else 1.7
        assert int(specs[k].L / rl) < 3
    b = P.Batch([_desc(P, sp) for sp in specs], cap=CAP)
    r = to_dev(np.concatenate([s[0] for s in states]), torch.float32)
    v = to_dev(np.concatenate([s[1] for s in states]), torch.float32)
    f = torch.zeros_like(r)
    st = status_word()
    n = 20
    PE = torch.zeros((len(specs), n), dtype=torch.float64, device=dev())
    KE = torch.zeros_like(PE)
    P.md_batch_build(b.plan, r, st)
    P.md_batch_forces(b.plan, r, f, st)
    torch.cuda.synchronize()
    f0 = f.cpu().numpy()
    P.md_batch_run_nve(b.plan, r, v, f, n, PE, KE, True, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    rg, vg, PEg, KEg = r.cpu().numpy(), v.cpu().numpy(), PE.cpu().numpy(), KE.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum([sp.N for sp in specs])])
    for k in sample:
        sp, (r0, v0) = specs[k], states[k]
        a, z = offs[k], offs[k + 1]
        # forces of the batched build against the oracle's
        U, F, e = _oracle_forces(sp, r0)
        assert force_error(f0[a:z], F) <= 1e-4, (k, sp.kind, sp.N)
        np.testing.assert_allclose(f0[a:z, 3], e, rtol=0, atol=2e-5 * max(np.abs(e).max(), 1e-12))
        # 20 velocity-Verlet steps of the batched launch against FP64
        kw = {} if sp.kind == "lj" else {"diam": r0[:, 3].astype(np.float64)}
        ro, vo, PEo, KEo = O.nve(r0, v0, sp.L, sp.kind, dt=sp.dt, nsteps=n, **kw)
        d = rg[a:z, :3] - ro
        d -= sp.L * np.round(d / sp.L)
        assert np.abs(d).max() < 2e-4, (k, sp.kind, sp.N)
        assert np.abs(vg[a:z, :3] - vo).max() < 2e-3, (k, sp.kind, sp.N)
        np.testing.assert_allclose(PEg[k], PEo[1:], rtol=2e-4, atol=1e-6 * sp.N)
        np.testing.assert_allclose(KEg[k], KEo[1:], rtol=2e-5, atol=1e-6 * sp.N)
