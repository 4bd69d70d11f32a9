"""Behler-Parrinello learned potential -- FP64 oracle (TEST INFRASTRUCTURE).

Plain PyTorch CPU float64 ops; forces and training gradients by autograd,
as the paper obtains forces from an energy model (Sec. 4.1: forces are the
negative gradient of the network energy; Sec. 3.2.4: symmetry-function
featurizers feeding a Behler-Parrinello network).  The paper names the
architecture and cites Behler (2011) for the descriptors without printing
them; this module fixes the reading:

  cutoff     f_c(r) = (cos(pi r / R_c) + 1) / 2 for r < R_c, else 0; R_c = 3.77 A
  radial     G_m   = sum_j exp(-eta_r (r_ij - R_m)^2) f_c(r_ij),
             R_m = 2.0 + 0.25 (m - 1) A (m = 1..8), eta_r = 8 A^-2
  angular    G_zl  = 2^(1 - zeta) sum_{j<k} (1 + lam cos theta_jik)^zeta
                     exp(-eta_a (r_ij^2 + r_ik^2)) f_c(r_ij) f_c(r_ik),
             zeta in {1, 2, 4, 16}, lam in {+1, -1} (8 terms), eta_a = 0.05 A^-2
  network    x = (G - mu) / sd;  E_i = w3 . silu(W2 silu(W1 x + b1) + b2) + b3
             (16 -> 64 -> 64 -> 1), E = sum_i E_i, F = -dE/dr
  loss       mean_s ((E_s - E_ref_s) / N)^2 + w_F mean_{s,i,c} (F - F_ref)^2

Parity unpinned: none (pins in tests/test_oracle_bp.py).
"""
from __future__ import annotations

import math

import numpy as np
import torch

R_C = 3.77
ETA_R = 8.0
R_M = [2.0 + 0.25 * m for m in range(8)]
ETA_A = 0.05
ZETAS = [1.0, 2.0, 4.0, 16.0]
LAMS = [1.0, -1.0]
N_DESC = 16
HIDDEN = 64

F64 = torch.float64


def fc(r):
    return torch.where(r < R_C, 0.5 * (torch.cos(math.pi * r / R_C) + 1.0), torch.zeros_like(r))


def pairs_within(r_np, L, rc=R_C):
    """Ordered pairs (i, j), i != j, with minimum-image distance < rc
    (brute force in FP64; fine for the sizes the oracle runs)."""
    x = np.asarray(r_np, np.float64)[:, :3]
    d = x[:, None, :] - x[None, :, :]
    d -= L * np.round(d / L)
    dist = np.sqrt((d ** 2).sum(-1))
    np.fill_diagonal(dist, np.inf)
    i, j = np.nonzero(dist < rc)
    return i, j


def triplets(i, j, N):
    """For each centre i, all ordered index pairs (a, b) of its pair list
    with j_a < j_b (each angular triplet once)."""
    order = np.lexsort((j, i))
    i, j = i[order], j[order]
    start = np.searchsorted(i, np.arange(N + 1))
    ta, tb = [], []
    for c in range(N):
        s, e = start[c], start[c + 1]
        for a in range(s, e):
            for b in range(a + 1, e):
                ta.append(a)
                tb.append(b)
    return i, j, np.asarray(ta, np.int64), np.asarray(tb, np.int64)


def descriptors(r, L, i, j, ta, tb):
    """G [N, 16] for positions r (torch [N, 3], requires_grad allowed).
    Displacements d_ij = r_j - r_i with the image shift fixed from the
    current positions (piecewise constant)."""
    N = r.shape[0]
    with torch.no_grad():
        shift = -L * torch.round((r[j] - r[i]) / L)
    d = r[j] - r[i] + shift
    rij = torch.sqrt((d * d).sum(-1))
    f = fc(rij)
    it = torch.as_tensor(i)
    cols = []
    for Rm in R_M:
        cols.append(torch.zeros(N, dtype=r.dtype).index_add(0, it, torch.exp(-ETA_R * (rij - Rm) ** 2) * f))
    ta_t = torch.as_tensor(ta, dtype=torch.long)
    tb_t = torch.as_tensor(tb, dtype=torch.long)
    u, w = d[ta_t], d[tb_t]
    ru, rw = rij[ta_t], rij[tb_t]
    cos = (u * w).sum(-1) / (ru * rw)
    base = torch.exp(-ETA_A * (ru * ru + rw * rw)) * f[ta_t] * f[tb_t]
    ci = it[ta_t]
    for z in ZETAS:
        for lam in LAMS:
            term = 2.0 ** (1.0 - z) * (1.0 + lam * cos) ** z * base
            cols.append(torch.zeros(N, dtype=r.dtype).index_add(0, ci, term))
    return torch.stack(cols, 1)


def silu(x):
    return x * torch.sigmoid(x)


def init_params(seed=0, hidden=HIDDEN):
    g = torch.Generator().manual_seed(seed)
    W1 = torch.randn(hidden, N_DESC, generator=g, dtype=F64) / math.sqrt(N_DESC)
    b1 = torch.zeros(hidden, dtype=F64)
    W2 = torch.randn(hidden, hidden, generator=g, dtype=F64) / math.sqrt(hidden)
    b2 = torch.zeros(hidden, dtype=F64)
    w3 = torch.randn(hidden, generator=g, dtype=F64) / math.sqrt(hidden)
    b3 = torch.zeros((), dtype=F64)
    return {"W1": W1, "b1": b1, "W2": W2, "b2": b2, "w3": w3, "b3": b3}


def mlp(x, p):
    h1 = silu(x @ p["W1"].T + p["b1"])
    h2 = silu(h1 @ p["W2"].T + p["b2"])
    return h2 @ p["w3"] + p["b3"]


def energy(r, L, graph, p, mu, sd):
    """Per-atom energies and total (graph = (i, j, ta, tb))."""
    G = descriptors(r, L, *graph)
    Ei = mlp((G - mu) / sd, p)
    return Ei, Ei.sum()


def energy_forces(r_np, L, p, mu, sd, graph=None):
    """(E, F [N,3], E_i [N], G [N,16]) in FP64."""
    r = torch.tensor(np.asarray(r_np, np.float64)[:, :3], requires_grad=True)
    if graph is None:
        graph = triplets(*pairs_within(r_np, L), r.shape[0])
    G = descriptors(r, L, *graph)
    Ei = mlp((G - mu) / sd, p)
    E = Ei.sum()
    (g,) = torch.autograd.grad(E, r)
    return E.item(), (-g).detach().numpy(), Ei.detach().numpy(), G.detach().numpy()


def loss_and_grads(batch, p, mu, sd, w_F=1.0):
    """Energy + force loss over a batch of snapshots [(r, L, E_ref, F_ref)]
    and its gradient with respect to every parameter (double backward
    through the force term by autograd)."""
    params = {k: v.clone().requires_grad_(True) for k, v in p.items()}
    lossE = 0.0
    lossF = 0.0
    nF = 0
    for (r_np, L, E_ref, F_ref) in batch:
        r = torch.tensor(np.asarray(r_np, np.float64)[:, :3], requires_grad=True)
        N = r.shape[0]
        graph = triplets(*pairs_within(r_np, L), N)
        G = descriptors(r, L, *graph)
        E = mlp((G - mu) / sd, params).sum()
        (g,) = torch.autograd.grad(E, r, create_graph=True)
        F = -g
        lossE = lossE + ((E - float(E_ref)) / N) ** 2
        lossF = lossF + ((F - torch.as_tensor(np.asarray(F_ref, np.float64)[:, :3])) ** 2).sum()
        nF += 3 * N
    loss = lossE / len(batch) + w_F * lossF / nF
    grads = torch.autograd.grad(loss, list(params.values()))
    return loss.item(), {k: gr.detach() for k, gr in zip(params.keys(), grads)}
