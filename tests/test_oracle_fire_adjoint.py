"""Pins of the FIRE-through-packing oracle (Sec. 4.2 / App. A with the FIRE
minimiser of Sec. 3.3.1): its forward trajectory against the separate C
FIRE oracle on the same packing, and dE_final/dD against central finite
differences of the final energy (steps small enough that every P > 0
decision of the trajectory stays the same)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import fire_adjoint as FA


@pytest.mark.parametrize("N,D,T,seed", [(32, 1.3, 60, 0), (64, 1.2, 120, 1)])
def test_forward_matches_c_fire(N, D, T, seed):
    p = W.packing_2d(N=N, D=D, seed=seed)
    E, _, hist = FA.fire_packing(p.s0, D, N // 2, T=T, grad=False)
    L = O.packing_box(N, D, 0.9)
    r = np.zeros((N, 3))
    r[:, :2] = p.s0 * L
    diam = np.where(np.arange(N) < N // 2, D, 1.0)
    _, _, Ec, dts, st = O.fire(r, L, "soft", nsteps=T, dim=2, diam=diam, eps=1.0, alpha=2.0)
    assert abs(E - Ec[T]) <= 1e-9 * max(1.0, abs(E))
    np.testing.assert_allclose([h[0] for h in hist[1:]], dts[:-1], rtol=1e-12)


@pytest.mark.parametrize("N,D,T,seed", [(32, 1.3, 60, 0), (48, 1.4, 100, 2)])
def test_gradient_matches_finite_differences(N, D, T, seed):
    p = W.packing_2d(N=N, D=D, seed=seed)
    E, g, hist = FA.fire_packing(p.s0, D, N // 2, T=T)
    h = 1e-6
    Ep, _, hp = FA.fire_packing(p.s0, D + h, N // 2, T=T, grad=False)
    Em, _, hm = FA.fire_packing(p.s0, D - h, N // 2, T=T, grad=False)
    assert [x[2] for x in hp] == [x[2] for x in hist] == [x[2] for x in hm]
    fd = (Ep - Em) / (2 * h)
    assert abs(fd - g) <= 1e-5 * max(1.0, abs(g)), (fd, g)
    assert any(x[2] for x in hist)      # the trajectory has resets (P <= 0)
