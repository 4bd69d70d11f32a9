"""The minimised energy of a bidisperse disk packing as a differentiable
function of the small/large diameter ratio (Sec. 4.2, App. A): a
torch.autograd.Function over the library's hand-written adjoints.

The paper differentiates ``minimize_energy(diameter, key)`` with ``grad``.
Here the forward pass is one call of ``md_minimize_adjoint`` (gradient
descent) or ``md_minimize_fire_adjoint`` (FIRE), which runs the minimisation
and its reverse sweep with sqrt(T) checkpoints on the GPU and returns both
E_final and dE_final/dD; backward multiplies the stored derivative by the
incoming gradient.  The derivative includes every way D enters: the
diameters, the box L(D) that keeps the packing fraction fixed, and the
start r_0 = L(D) s_0.  Only argument marshalling happens in Python.
"""
from __future__ import annotations

import math

from . import jmd as J


class _Plans:
    """Lists, workspaces and buffers per (N, D, T, K, minimiser, device),
    kept so that repeated calls reuse the adjoint's captured graph."""

    def __init__(self):
        self.cache = {}

    def get(self, N, D, phi, T, K, fire, device):
        import torch
        key = (N, float(D), float(phi), T, K, fire, str(device))
        if key in self.cache:
            return self.cache[key]
        # the box L(D) at packing fraction phi comes from the library
        space, _ = J.md_packing_space(N, N // 2, D, 1.0, phi)
        nl = J.NeighborList(space, N, max(D, 1.0), 0.3, 64, device=device, canonical=True)
        nbytes = (J.md_fire_adjoint_workspace_size if fire else J.md_adjoint_workspace_size)(N, T, K)
        raw = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        ws = raw[(-raw.data_ptr()) % 256:]
        bufs = [torch.zeros((N, 4), dtype=torch.float32, device=device) for _ in range(3)]
        s0 = torch.zeros((N, 4), dtype=torch.float32, device=device)
        out = torch.zeros(2, dtype=torch.float64, device=device)
        st = torch.zeros(1, dtype=torch.int32, device=device)
        entry = dict(space=space, nl=nl, raw=raw, ws=ws, bufs=bufs, s0=s0, out=out, st=st, phi=phi)
        if len(self.cache) >= 64:
            self.cache.pop(next(iter(self.cache)))
        self.cache[key] = entry
        return entry


_PLANS = _Plans()


def _import_torch():
    import torch
    return torch


class MinimizedPackingEnergy(_import_torch().autograd.Function):
    """E_final(D) of the packing started from fractional positions s0
    (float32 [N, 2] on the device, half of diameter D first), minimised for
    T steps; forward returns a float64 scalar tensor."""

    @staticmethod
    def forward(ctx, D, s0, T, K, phi, eta, fire):
        N = int(s0.shape[0])
        d = float(D.detach().item())
        P = _PLANS.get(N, d, phi, T, K, fire, s0.device)
        P["s0"][:, :2].copy_(s0[:, :2])
        r, v, f = P["bufs"]
        if fire:
            J.md_minimize_fire_adjoint(P["space"], J.soft_pot(), J.fire_params(), P["nl"].plan, P["s0"], N // 2, d,
                                       1.0, P["phi"], T, K, r, v, f, P["ws"], P["out"], P["st"])
        else:
            J.md_minimize_adjoint(P["space"], J.soft_pot(), P["nl"].plan, P["s0"], N // 2, d, 1.0, P["phi"], eta, T, K,
                                  r, f, P["ws"], P["out"], P["st"])
        code = J.md_status_poll(P["st"])
        if code != 0:
            raise J.MDError(code, "MinimizedPackingEnergy")
        out = P["out"].clone()
        ctx.save_for_backward(out[1:2])
        return out[0].to(D.dtype)

    @staticmethod
    def backward(ctx, grad_E):
        (dEdD,) = ctx.saved_tensors
        return (grad_E * dEdD[0]).to(grad_E.dtype), None, None, None, None, None, None


def packing_energy(D, s0, T: int, K: int | None = None, phi: float = 0.9, eta: float = 0.05,
                   minimizer: str = "gd"):
    """Differentiable minimised energy of the bidisperse packing.

    D: scalar tensor (on the device; requires_grad for dE/dD), the diameter of
    the first N/2 disks (the others have diameter 1).  s0: [N, 2] fractional
    start positions in [0, 1).  T minimisation steps (gradient descent with
    step eta, or FIRE with Bitzek's parameters), K checkpoint interval
    (default ceil(sqrt(T))).  Calls with the same N, D, T, K and minimiser
    reuse their lists and the adjoint's captured graph."""
    if minimizer not in ("gd", "fire"):
        raise ValueError("minimizer must be 'gd' or 'fire'")
    K = K or int(math.ceil(math.sqrt(T)))
    return MinimizedPackingEnergy.apply(D, s0, int(T), int(K), float(phi), float(eta), minimizer == "fire")
