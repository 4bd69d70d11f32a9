"""Graph-network potential -- FP64 oracle (TEST INFRASTRUCTURE).

Plain PyTorch CPU float64 ops; forces by autograd, since the paper defines
forces as the negative gradient of the network energy (Sec. 4.1).  The
paper names the model only: a graph network built from GraphNet blocks
(Battaglia et al. 2018), the standard network used for glasses by Bapst et
al. (2020) (Sec. 3.2.4), which is not invariant to rotations (Sec. 4.1
trains it with random rotations and flips).  This module fixes the reading
(encode - process - decode, hidden width H, T message-passing steps):

  graph      directed edges (i <- j) for the ordered pairs with minimum-
             image distance r_ij < r_c (i receives, j sends)
  cutoff     s(r) = (cos(pi r / r_c) + 1) / 2 for r < r_c, else 0
  encode     e0_ij = silu(W_enc x_ij + b_enc),  x_ij = (R_j - R_i) / r_c
             v0_i  = u                         (one species)
  process    for t = 1..T (own weights per step):
             e_ij = silu(A_e e_ij + A_r v_i + A_s v_j + a)
             m_i  = sum_j s(r_ij) e_ij
             v_i  = silu(B_v v_i + B_m m_i + b)
  decode     E_i = w . silu(D v_i + d) + c,    E = sum_i E_i,  F = -dE/dR

The cutoff weight on the messages makes E and F continuous as pairs cross
r_c.  Flat parameter layout (shared with the device library's header):

  W_enc [H][3], b_enc [H], u [H],
  T x { A [H][3H] (columns: A_e | A_r | A_s), a [H], B [H][2H] (B_v | B_m), b [H] },
  D [H][H], d [H], w [H], c
  count = 5H + T (5H^2 + 2H) + H^2 + 2H + 1

Parity unpinned: none (pins in tests/test_oracle_gnn.py).
"""
from __future__ import annotations

import math

import numpy as np
import torch

F64 = torch.float64


def param_count(H, T):
    return 5 * H + T * (5 * H * H + 2 * H) + H * H + 2 * H + 1


def unpack(p, H, T):
    """Views of the flat parameter vector (torch, any dtype)."""
    o = 0

    def take(n, shape):
        nonlocal o
        v = p[o:o + n].reshape(shape)
        o += n
        return v

    out = {"W_enc": take(3 * H, (H, 3)), "b_enc": take(H, (H,)), "u": take(H, (H,)), "layers": []}
    for _ in range(T):
        A = take(3 * H * H, (H, 3 * H))
        a = take(H, (H,))
        B = take(2 * H * H, (H, 2 * H))
        b = take(H, (H,))
        out["layers"].append({"A_e": A[:, :H], "A_r": A[:, H:2 * H], "A_s": A[:, 2 * H:], "a": a,
                              "B_v": B[:, :H], "B_m": B[:, H:], "b": b})
    out["D"] = take(H * H, (H, H))
    out["d"] = take(H, (H,))
    out["w"] = take(H, (H,))
    out["c"] = take(1, (1,))
    assert o == p.shape[0]
    return out


def cutoff(r, rc):
    return torch.where(r < rc, 0.5 * (torch.cos(math.pi * r / rc) + 1.0), torch.zeros_like(r))


def silu(x):
    return x * torch.sigmoid(x)


def edges_within(R_np, L, rc):
    """Directed edges (i <- j), i != j, minimum-image distance < rc; brute
    force in FP64 (the sizes the oracle runs)."""
    x = np.asarray(R_np, np.float64)[:, :3]
    d = x[None, :, :] - x[:, None, :]          # d[i, j] = R_j - R_i
    d -= L * np.round(d / L)
    dist = np.sqrt((d ** 2).sum(-1))
    np.fill_diagonal(dist, np.inf)
    i, j = np.nonzero(dist < rc)
    return i, j


def energy(R, L, params, H, T, rc, edges):
    """E (scalar) and E_i [N] for positions R (torch [N, 3], FP64)."""
    P = unpack(params, H, T)
    i, j = (torch.as_tensor(k, dtype=torch.long) for k in edges)
    N = R.shape[0]
    d = R[j] - R[i]
    d = d - L * torch.round(d.detach() / L)
    r = torch.sqrt((d * d).sum(-1))
    s = cutoff(r, rc)
    e = silu((d / rc) @ P["W_enc"].T + P["b_enc"])
    v = P["u"].expand(N, H)
    for ly in P["layers"]:
        e = silu(e @ ly["A_e"].T + v[i] @ ly["A_r"].T + v[j] @ ly["A_s"].T + ly["a"])
        m = torch.zeros(N, H, dtype=R.dtype).index_add(0, i, s[:, None] * e)
        v = silu(v @ ly["B_v"].T + m @ ly["B_m"].T + ly["b"])
    Ei = silu(v @ P["D"].T + P["d"]) @ P["w"] + P["c"]
    return Ei.sum(), Ei


def energy_forces(R_np, L, params, H, T, rc, edges=None):
    """(E, E_i [N], F [N, 3]) in FP64 numpy; params a flat array."""
    R = torch.tensor(np.asarray(R_np, np.float64)[:, :3], dtype=F64, requires_grad=True)
    p = torch.as_tensor(np.asarray(params, np.float64), dtype=F64)
    if edges is None:
        edges = edges_within(R_np, L, rc)
    E, Ei = energy(R, L, p, H, T, rc, edges)
    (g,) = torch.autograd.grad(E, R)
    return float(E.detach()), Ei.detach().numpy(), -g.numpy()


def loss(batch, params, H, T, rc, w_F=1.0, create_graph=False):
    """Energy + force loss over snapshots [(R, L, E_ref, F_ref)] (the fit of
    Sec. 4.1, as for the BP network):
        mean_s ((E_s - E_ref,s) / n)^2 + w_F mean_{s,i,c} (F - F_ref)^2
    params: a torch FP64 vector (may require grad)."""
    lossE = 0.0
    lossF = 0.0
    nF = 0
    for (R_np, L, E_ref, F_ref) in batch:
        R = torch.tensor(np.asarray(R_np, np.float64)[:, :3], dtype=F64, requires_grad=True)
        n = R.shape[0]
        E, _ = energy(R, L, params, H, T, rc, edges_within(R_np, L, rc))
        (g,) = torch.autograd.grad(E, R, create_graph=create_graph)
        F = -g
        lossE = lossE + ((E - float(E_ref)) / n) ** 2
        lossF = lossF + ((F - torch.as_tensor(np.asarray(F_ref, np.float64)[:, :3])) ** 2).sum()
        nF += 3 * n
    return lossE / len(batch) + w_F * lossF / nF


def loss_and_grads(batch, params, H, T, rc, w_F=1.0):
    """(loss, d loss / d params as a flat FP64 array): the force term's
    gradient is a double backward (autograd through autograd)."""
    p = torch.tensor(np.asarray(params, np.float64), dtype=F64, requires_grad=True)
    L_ = loss(batch, p, H, T, rc, w_F, create_graph=True)
    (g,) = torch.autograd.grad(L_, p)
    return float(L_.detach()), g.numpy()
