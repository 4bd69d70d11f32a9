"""FIRE through a soft-disk packing and dE_final/dD -- FP64 oracle (TEST
INFRASTRUCTURE).

Plain PyTorch CPU float64 ops with autograd.  The packing is the one of
Sec. 4.2 / App. A: 2-D disks, the first nA of diameter D and the rest of
diameter dB, in a square box whose edge L(D) = sqrt((N/2) pi (D^2 + dB^2) /
(4 phi)) keeps the packing fraction at phi; r_0 = L(D) s_0, unwrapped
coordinates (minimum image with image integers taken as constants), the
soft-sphere energy u = (eps/alpha)(1 - r/sigma)^alpha for r < sigma_ij =
(D_i + D_j)/2.  The minimiser is FIRE (Bitzek et al., PRL 97, 170201
(2006); Sec. 3.3.1) from rest, one step in the published order:

  v += dt/2 F;  r += dt v;  F = F(r);  v += dt/2 F;  P = F . v
  v = (1 - alpha) v + alpha |v| F / |F|          (no F term when |F| = 0)
  P > 0:  npos += 1;  npos > n_min: dt = min(dt f_inc, dt_max), alpha *= f_alpha
  P <= 0: v = 0;  dt *= f_dec;  alpha = alpha_start;  npos = 0

E = U(r_T).  dt, alpha and the P > 0 decisions are plain numbers (the map
is piecewise smooth; its derivative is taken with the decisions of the
trajectory held fixed), so autograd differentiates E through every state,
force, norm and mixing step, the box L(D) and the diameters.

Parity unpinned: none (pins in tests/test_oracle_fire_adjoint.py).
"""
from __future__ import annotations

import math

import numpy as np
import torch

F64 = torch.float64
FIRE_DEFAULTS = dict(dt_start=0.1, dt_max=0.4, f_inc=1.1, f_dec=0.5, alpha_start=0.1, f_alpha=0.99, n_min=5)


def _forces_energy(r, diam, L, eps, alpha):
    """Soft-disk forces [N, 2] and energy, all pairs (the sizes the oracle
    runs); image integers are constants."""
    d = r[:, None, :] - r[None, :, :]
    d = d - L * torch.round(d.detach() / L)
    N = r.shape[0]
    eye = torch.eye(N, dtype=torch.bool)
    r2 = (d * d).sum(-1)
    rr = torch.sqrt(torch.where(eye, torch.ones_like(r2), r2))
    sig = 0.5 * (diam[:, None] + diam[None, :])
    inside = (rr < sig) & ~eye
    x = torch.where(inside, 1.0 - rr / sig, torch.zeros_like(rr))
    U = 0.5 * torch.where(inside, (eps / alpha) * x ** alpha, torch.zeros_like(rr)).sum()
    # F_i = sum_j (eps / sigma) x^(alpha - 1) d_ij / r
    mag = torch.where(inside, (eps / sig) * x ** (alpha - 1.0) / rr, torch.zeros_like(rr))
    F = (mag[:, :, None] * d).sum(1)
    return F, U


def fire_packing(s0, D, nA, dB=1.0, phi=0.9, eps=1.0, alpha=2.0, T=300, fire=None, grad=True):
    """(E_final, dE/dD, history): history[s] = (dt, alpha, froze) of step s."""
    fp = dict(FIRE_DEFAULTS, **(fire or {}))
    s0 = torch.as_tensor(np.asarray(s0, np.float64)[:, :2], dtype=F64)
    N = s0.shape[0]
    Dt = torch.tensor(float(D), dtype=F64, requires_grad=grad)
    L = torch.sqrt((N // 2) * math.pi * (Dt ** 2 + dB ** 2) / (4.0 * phi))
    diam = torch.cat([Dt.expand(nA), torch.full((N - nA,), float(dB), dtype=F64)])
    r = L * s0
    v = torch.zeros_like(r)
    F, _ = _forces_energy(r, diam, L, eps, alpha)
    dt, a, npos = fp["dt_start"], fp["alpha_start"], 0
    hist = []
    for _ in range(T):
        v = v + 0.5 * dt * F
        r = r + dt * v
        F, _ = _forces_energy(r, diam, L, eps, alpha)
        v = v + 0.5 * dt * F
        P = float((F * v).sum().detach())
        vn = torch.sqrt((v * v).sum())
        fn = torch.sqrt((F * F).sum())
        step = (dt, a, P <= 0.0)
        if float(fn.detach()) > 0.0:
            v = (1.0 - a) * v + a * vn * F / fn
        else:
            v = (1.0 - a) * v
        if P > 0.0:
            npos += 1
            if npos > fp["n_min"]:
                dt = min(dt * fp["f_inc"], fp["dt_max"])
                a = a * fp["f_alpha"]
        else:
            v = torch.zeros_like(v)
            dt = dt * fp["f_dec"]
            a = fp["alpha_start"]
            npos = 0
        hist.append(step)
    _, U = _forces_energy(r, diam, L, eps, alpha)
    g = float(torch.autograd.grad(U, Dt)[0]) if grad else None
    return float(U.detach()), g, hist
