"""Pins for the Behler-Parrinello oracle: closed-form descriptors for two
and three atoms, invariances, and finite differences of the descriptors,
the energy (forces) and the loss (weight gradients).  CPU only."""
import math

import numpy as np
import pytest
import torch

import oracle.bp as B


def _graph(r, L):
    return B.triplets(*B.pairs_within(r, L), r.shape[0])


def test_fc_cutoff_function():
    r = torch.tensor([0.0, B.R_C / 2, B.R_C, B.R_C + 0.1], dtype=torch.float64)
    np.testing.assert_allclose(B.fc(r).numpy(), [1.0, 0.5, 0.0, 0.0], atol=1e-15)


def test_two_atom_radial_closed_form():
    L = 30.0
    d = 2.4
    r = np.array([[10.0, 10.0, 10.0], [10.0 + d, 10.0, 10.0]])
    G = B.descriptors(torch.tensor(r), L, *_graph(r, L)).numpy()
    fcd = 0.5 * (math.cos(math.pi * d / B.R_C) + 1)
    for m, Rm in enumerate(B.R_M):
        assert abs(G[0, m] - math.exp(-B.ETA_R * (d - Rm) ** 2) * fcd) < 1e-15
    np.testing.assert_allclose(G[0], G[1], atol=1e-15)
    assert np.all(G[:, 8:] == 0.0)


def test_three_atom_angular_closed_form():
    L = 30.0
    r1, r2, th = 2.3, 2.9, math.radians(104.0)
    c = np.array([10.0, 10.0, 10.0])
    r = np.stack([c, c + [r1, 0, 0], c + [r2 * math.cos(th), r2 * math.sin(th), 0]])
    G = B.descriptors(torch.tensor(r), L, *_graph(r, L)).numpy()
    f1 = 0.5 * (math.cos(math.pi * r1 / B.R_C) + 1)
    f2 = 0.5 * (math.cos(math.pi * r2 / B.R_C) + 1)
    col = 8
    for z in B.ZETAS:
        for lam in B.LAMS:
            want = 2 ** (1 - z) * (1 + lam * math.cos(th)) ** z * math.exp(-B.ETA_A * (r1 ** 2 + r2 ** 2)) * f1 * f2
            assert abs(G[0, col] - want) < 1e-14 * max(1.0, want)
            col += 1


def _cluster(n=12, seed=0):
    rng = np.random.default_rng(seed)
    pts = [np.zeros(3)]
    while len(pts) < n:
        p = pts[rng.integers(len(pts))] + rng.normal(size=3) * 1.6
        if min(np.linalg.norm(p - q) for q in pts) > 2.0:
            pts.append(p)
    return np.array(pts) + 20.0


def test_descriptor_invariances():
    L = 60.0
    r = _cluster()
    G = B.descriptors(torch.tensor(r), L, *_graph(r, L)).numpy()
    A = np.linalg.qr(np.random.default_rng(1).normal(size=(3, 3)))[0]
    c = r.mean(0)
    r2 = (r - c) @ A.T + c + np.array([1.3, -0.7, 2.2])
    G2 = B.descriptors(torch.tensor(r2), L, *_graph(r2, L)).numpy()
    np.testing.assert_allclose(G2, G, atol=1e-12)
    perm = np.random.default_rng(2).permutation(len(r))
    G3 = B.descriptors(torch.tensor(r[perm]), L, *_graph(r[perm], L)).numpy()
    np.testing.assert_allclose(G3, G[perm], atol=1e-12)


def _si_snapshot(seed=3):
    import workloads as W
    si = W.sw_silicon(2, T_K=0, jitter=0.25, seed=seed)
    return si.r[:, :3].astype(np.float64), si.L


def test_descriptor_and_energy_finite_differences():
    r, L = _si_snapshot()
    graph = _graph(r, L)
    p = B.init_params(0)
    mu, sd = torch.zeros(16, dtype=torch.float64), torch.ones(16, dtype=torch.float64)
    E, F, Ei, G = B.energy_forces(r, L, p, mu, sd, graph)
    h = 1e-6
    for (a, k) in [(0, 0), (5, 1), (17, 2), (40, 0)]:
        rp, rm = r.copy(), r.copy()
        rp[a, k] += h
        rm[a, k] -= h
        Gp = B.descriptors(torch.tensor(rp), L, *graph)
        Gm = B.descriptors(torch.tensor(rm), L, *graph)
        rt = torch.tensor(r, requires_grad=True)
        Gt = B.descriptors(rt, L, *graph)
        jac = torch.autograd.grad(Gt[:, 3].sum() + Gt[:, 12].sum(), rt)[0][a, k].item()
        fd = ((Gp[:, 3].sum() + Gp[:, 12].sum()) - (Gm[:, 3].sum() + Gm[:, 12].sum())).item() / (2 * h)
        assert abs(jac - fd) < 1e-7 * max(1.0, abs(fd))
        Ep = B.energy_forces(rp, L, p, mu, sd, graph)[0]
        Em = B.energy_forces(rm, L, p, mu, sd, graph)[0]
        assert abs(-(Ep - Em) / (2 * h) - F[a, k]) < 1e-7 * max(1.0, abs(F[a, k]))


def test_loss_weight_gradient_finite_differences():
    r, L = _si_snapshot(4)
    p = B.init_params(1)
    mu, sd = torch.zeros(16, dtype=torch.float64), torch.ones(16, dtype=torch.float64)
    E, F, _, _ = B.energy_forces(r, L, p, mu, sd)
    batch = [(r + 0.01, L, E + 0.3, F * 0.7)]
    loss, grads = B.loss_and_grads(batch, p, mu, sd, w_F=1.0)
    h = 1e-6
    for name, idx in [("W1", (3, 5)), ("W2", (10, 20)), ("w3", (7,)), ("b1", (2,)), ("b3", ())]:
        q = {k: v.clone() for k, v in p.items()}
        q[name][idx] += h
        lp, _ = B.loss_and_grads(batch, q, mu, sd)
        q[name][idx] -= 2 * h
        lm, _ = B.loss_and_grads(batch, q, mu, sd)
        fd = (lp - lm) / (2 * h)
        assert abs(grads[name][idx].item() - fd) < 1e-6 * max(1e-3, abs(fd)), (name, grads[name][idx].item(), fd)
