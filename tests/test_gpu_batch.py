"""GPU: batched replicas (the paper's vmap over independent systems,
Sec. 4.2) -- hundreds of uneven LJ and soft-sphere systems advanced in one
graph launch -- against the same replicas advanced one launch each (bit for
bit), plus energy conservation and the autotuner."""
import json
import os

import numpy as np
import pytest

import workloads as W
from gpu_helpers import dev, status_word, to_dev

pytestmark = pytest.mark.gpu

CAP = 128


@pytest.fixture(scope="module")
def P():
    import paper_1912_04232_b300 as P
    return P


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


def _pot(P, spec):
    return P.lj_pot() if spec.kind == "lj" else P.soft_pot(1.0, 2.0)


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
        # fold back into the box (GD works in unwrapped coordinates)
        x = rd.cpu().numpy()
        x[:, :3] = np.mod(x[:, :3], np.float32(spec.L)).astype(np.float32)
        x[:, :3][x[:, :3] >= np.float32(spec.L)] = 0.0
        r = x
    return r, v


def _single(P, spec, r, v, nsteps):
    import torch
    s = P.md_space_periodic(3, [spec.L] * 3)
    rc = 2.5 if spec.kind == "lj" else 1.4
    nl = P.NeighborList(s, spec.N, rc, 0.3, CAP)
    rd, vd = to_dev(r, torch.float32), to_dev(v, torch.float32)
    f = torch.zeros_like(rd)
    st = status_word()
    pot = _pot(P, spec)
    nl.build(rd, st)
    P.md_energy_forces(s, pot, rd, nl.plan, f, None, st)
    P.md_integrate_nve(s, pot, rd, vd, f, 1.0, spec.dt, nsteps, nl.plan, None, None, True, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    return rd.cpu().numpy(), vd.cpu().numpy()


def _batched(P, specs, states, nsteps, tune=None):
    import torch
    b = P.Batch([_desc(P, sp) for sp in specs], cap=CAP)
    r = to_dev(np.concatenate([s[0] for s in states]), torch.float32)
    v = to_dev(np.concatenate([s[1] for s in states]), torch.float32)
    f = torch.zeros_like(r)
    st = status_word()
    PE = torch.zeros((len(specs), nsteps), dtype=torch.float64, device=dev())
    KE = torch.zeros_like(PE)
    if tune is not None:
        scratch = torch.empty((2 * b.plan.N, 4), dtype=torch.float32, device=dev())
        P.md_batch_autotune(b.plan, r, v, f, scratch, 20, tune)
    P.md_batch_build(b.plan, r, st)
    P.md_batch_forces(b.plan, r, f, st)
    P.md_batch_run_nve(b.plan, r, v, f, nsteps, PE, KE, True, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    return b, r.cpu().numpy(), v.cpu().numpy(), PE.cpu().numpy(), KE.cpu().numpy()


def _specs(R, seed):
    return W.replica_plan(R=R, n_max=2048, seed=seed)


def test_batch_equals_one_launch_per_replica_bitwise(P):
    specs = _specs(8, 3)
    states = [_initial(P, sp) for sp in specs]
    n = 120
    b, r, v, PE, KE = _batched(P, specs, states, n)
    # same lanes per particle as the batch plan's default, whatever an
    # earlier test left set
    P.md_set_pair_tpp(4)
    off = 0
    for sp, stt in zip(specs, states):
        rs, vs = _single(P, sp, stt[0], stt[1], n)
        np.testing.assert_array_equal(r[off:off + sp.N], rs)
        np.testing.assert_array_equal(v[off:off + sp.N, :3], vs[:, :3])
        off += sp.N
    assert min(P.md_batch_stats(b.plan)) >= 1


def _single_drift(P, spec, r, v, dt, nsteps):
    import torch
    s = P.md_space_periodic(3, [spec.L] * 3)
    rc = 2.5 if spec.kind == "lj" else 1.4
    nl = P.NeighborList(s, spec.N, rc, 0.3, CAP)
    rd, vd = to_dev(r, torch.float32), to_dev(v, torch.float32)
    f = torch.zeros_like(rd)
    st = status_word()
    pot = _pot(P, spec)
    nl.build(rd, st)
    P.md_energy_forces(s, pot, rd, nl.plan, f, None, st)
    pe = torch.zeros(nsteps, dtype=torch.float64, device=dev())
    ke = torch.zeros_like(pe)
    P.md_integrate_nve(s, pot, rd, vd, f, 1.0, dt, nsteps, nl.plan, pe, ke, True, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    E = (pe + ke).cpu().numpy()
    return np.abs(E - E[0]).max() / spec.N


def test_batch_512_replicas_500_steps(P):
    specs = W.replica_plan(R=512, n_max=8192, seed=0)
    states = [_initial(P, sp) for sp in specs]
    n = 500
    b, r, v, PE, KE = _batched(P, specs, states, n)
    N = np.array([sp.N for sp in specs])
    assert b.plan.N == N.sum() and N.min() >= 64 and N.max() <= 8192
    E = PE + KE
    assert np.all(np.isfinite(E))
    drift = np.abs(E - E[:, :1]).max(axis=1) / N
    soft = np.array([sp.kind == "soft" for sp in specs])
    assert drift[soft].max() < 1e-3
    # the largest LJ drift (dense replicas released from a lattice) is
    # integration error: it shrinks as dt does -- between first order (pairs
    # crossing the cutoff, where the force is discontinuous) and second
    # order (velocity Verlet); a force error would not shrink
    k = int(np.argmax(np.where(soft, -1, drift)))
    sp = specs[k]
    d1 = _single_drift(P, sp, states[k][0], states[k][1], sp.dt, n)
    d2 = _single_drift(P, sp, states[k][0], states[k][1], sp.dt / 2, 2 * n)
    assert abs(d1 - drift[k]) <= 1e-6 * max(1.0, d1)
    assert 2.2 <= d1 / d2 <= 5.5, (d1, d2)
    # a sample of replicas advanced alone agree bit for bit
    offs = np.concatenate([[0], np.cumsum(N)])
    for k in (0, 101, 300, 511):
        rs, vs = _single(P, specs[k], states[k][0], states[k][1], n)
        np.testing.assert_array_equal(r[offs[k]:offs[k + 1]], rs)


def test_autotuner_picks_and_caches(P, tmp_path):
    specs = _specs(16, 7)
    states = [_initial(P, sp) for sp in specs]
    path = str(tmp_path / "tune.json")
    b, r, v, PE, KE = _batched(P, specs, states, 50, tune=path)
    assert b.plan.tpp in (4, 8, 16)
    cached = json.load(open(path))
    assert list(cached.values()) == [b.plan.tpp]
    # the cached choice is read back without timing
    b2 = P.Batch([_desc(P, sp) for sp in specs], cap=CAP)
    import torch
    x = torch.zeros((b2.plan.N, 4), dtype=torch.float32, device=dev())
    scratch = torch.empty((2 * b2.plan.N, 4), dtype=torch.float32, device=dev())
    t = P.md_batch_autotune(b2.plan, x, x.clone(), x.clone(), scratch, 20, path)
    assert t == b.plan.tpp
