"""dE_final/dD through torch.autograd (Sec. 4.2: ``grad(minimize_energy)``):
the autograd.Function over the hand-written adjoints returns the energy and,
on backward, the derivative the FP64 reverse-mode oracles give, for gradient
descent and for FIRE, and it composes with other torch operations."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import dev
from oracle import fire_adjoint as FA

pytestmark = pytest.mark.gpu


def _s0(p):
    import torch
    return torch.from_numpy(p.s0.astype(np.float32)).to(dev())


def test_autograd_gradient_descent_matches_fp64_reverse_mode():
    import torch
    from paper_1912_04232_b300.autodiff import packing_energy
    D0, T = 1.3, 60
    p = W.packing_2d(N=128, D=D0, seed=11)
    D = torch.tensor(D0, dtype=torch.float64, device=dev(), requires_grad=True)
    E = packing_energy(D, _s0(p), T)
    E.backward()
    Eo, go, _ = O.gd_adjoint(p.s0, D0, T=T)
    assert abs(E.item() - Eo) <= 1e-4 * abs(Eo) + 1e-7
    assert abs(D.grad.item() - go) <= 2e-3 * abs(go) + 1e-6, (D.grad.item(), go)


def test_autograd_fire_matches_fp64_reverse_mode():
    import torch
    from paper_1912_04232_b300.autodiff import packing_energy
    D0, N, T = 1.2, 64, 120
    p = W.packing_2d(N=N, D=D0, seed=1)
    D = torch.tensor(D0, dtype=torch.float64, device=dev(), requires_grad=True)
    E = packing_energy(D, _s0(p), T, minimizer="fire")
    E.backward()
    Eo, go, _ = FA.fire_packing(p.s0, D0, N // 2, T=T)
    assert abs(E.item() - Eo) <= 1e-4 * abs(Eo) + 1e-7
    assert abs(D.grad.item() - go) <= 2e-3 * abs(go) + 1e-6, (D.grad.item(), go)


def test_autograd_chain_rule_and_repeat_calls():
    # y = E^2 + 3 E: dy/dD = (2 E + 3) dE/dD; a second call with the same
    # arguments (replaying the adjoint's captured graph) gives the same bits
    import torch
    from paper_1912_04232_b300.autodiff import packing_energy
    p = W.packing_2d(N=128, D=1.25, seed=6)
    s0 = _s0(p)
    D = torch.tensor(1.25, dtype=torch.float64, device=dev(), requires_grad=True)
    E = packing_energy(D, s0, 80)
    (g,) = torch.autograd.grad(E, D)
    D2 = torch.tensor(1.25, dtype=torch.float64, device=dev(), requires_grad=True)
    E2 = packing_energy(D2, s0, 80)
    y = E2 * E2 + 3.0 * E2
    y.backward()
    assert E2.item() == E.item()
    np.testing.assert_allclose(D2.grad.item(), (2.0 * E.item() + 3.0) * g.item(), rtol=1e-12)
