"""Host-side packing geometry (App. A): the library's box L(D) at fixed
packing fraction and its derivative, and the adjoints' check that the space
they are given is that box (no GPU needed: both are host logic)."""
import math

import pytest

import workloads as W


@pytest.fixture(scope="module")
def P():
    import paper_1912_04232_b300 as P
    return P


@pytest.mark.parametrize("N,D,phi", [(128, 1.4, 0.9), (1024, 1.0, 0.9), (256, 0.7, 0.85)])
def test_packing_space_box_and_derivative(P, N, D, phi):
    s, lp = P.md_packing_space(N, N // 2, D, 1.0, phi)
    L = W.packing_box(N, D, phi)           # the input generator's box
    assert s.dim == 2 and abs(s.L64[0] - L) <= 1e-12 * L and s.L64[1] == s.L64[0]
    assert s.L[0] == W.f32(L)
    # dL/dD against a central difference of the library's own box
    h = 1e-6 * D
    Lm = P.md_packing_space(N, N // 2, D - h, 1.0, phi)[0].L64[0]
    Lq = P.md_packing_space(N, N // 2, D + h, 1.0, phi)[0].L64[0]
    assert abs(lp - (Lq - Lm) / (2 * h)) <= 1e-7 * abs(lp)
    # fixed packing fraction: disk area / L^2 = phi
    area = (N // 2) * math.pi * (D * D + 1.0) / 4.0
    assert abs(area / s.L64[0] ** 2 - phi) <= 1e-12


def test_packing_space_rejects_bad_arguments(P):
    for args in ((0, 0, 1.0, 1.0, 0.9), (10, 11, 1.0, 1.0, 0.9), (10, 5, -1.0, 1.0, 0.9), (10, 5, 1.0, 1.0, 0.0)):
        with pytest.raises(P.MDError):
            P.md_packing_space(*args)


def test_adjoint_rejects_a_box_other_than_the_packing(P):
    # host validation runs before any device work: a space that is not L(D)
    N, D, phi = 128, 1.4, 0.9
    L = W.f32(W.packing_box(N, D, phi))
    wrong = P.md_space_periodic(2, [L * 1.01, L * 1.01])
    nb = P.md_nbr_plan(wrong, N, D, 0.3, 64)
    lib = P.lib()
    import ctypes as C
    code = lib.md_minimize_adjoint(C.byref(wrong), C.byref(P.soft_pot()), C.byref(nb), None, N // 2, D, 1.0, phi,
                                   0.05, 10, 4, None, None, None, None, None, None)
    assert code == P.MD_ERR_INVALID
    code = lib.md_minimize_fire_adjoint(C.byref(wrong), C.byref(P.soft_pot()), C.byref(P.fire_params()), C.byref(nb),
                                        None, N // 2, D, 1.0, phi, 10, 4, None, None, None, None, None, None, None)
    assert code == P.MD_ERR_INVALID
