"""Failure detection without a GPU fault: device-side conditions are
reported through the status word, and the context stays usable."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import dev, status_word, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1912_04232_b300 as P
    return P


def test_nonfinite_position_is_reported(P):
    import torch
    c = W.lj_small()
    r = c.r.copy()
    r[17, 0] = np.nan
    s = P.md_space_periodic(3, [c.L] * 3)
    nl = P.NeighborList(s, c.N, 2.5, 0.3, 128)
    rd = to_dev(r, torch.float32)
    st = status_word()
    nl.build(rd, st)
    f = torch.zeros_like(rd)
    E = torch.zeros(1, dtype=torch.float64, device=dev())
    P.md_energy_forces(s, P.lj_pot(), rd, nl.plan, f, E, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) & P.MD_ERR_NONFINITE
    # the context is still usable
    st.zero_()
    rd = to_dev(c.r, torch.float32)
    nl.build(rd, st)
    P.md_energy_forces(s, P.lj_pot(), rd, nl.plan, f, E, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0 and np.isfinite(E.item())


def test_nonfinite_velocity_reaches_the_energy_reduction(P):
    import torch
    c = W.lj_small()
    v = c.v.copy()
    v[5, 1] = np.inf
    s = P.md_space_periodic(3, [c.L] * 3)
    nl = P.NeighborList(s, c.N, 2.5, 0.3, 128)
    rd, vd = to_dev(c.r, torch.float32), to_dev(v, torch.float32)
    st = status_word()
    nl.build(rd, st)
    f = torch.zeros_like(rd)
    P.md_energy_forces(s, P.lj_pot(), rd, nl.plan, f, None, st)
    KE = torch.zeros(1, dtype=torch.float64, device=dev())
    P.md_integrate_nve(s, P.lj_pot(), rd, vd, f, 1.0, 0.005, 1, nl.plan, None, KE, True, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) & P.MD_ERR_NONFINITE


def test_bounded_wait_times_out_and_returns(P):
    import torch
    flag = torch.zeros(1, dtype=torch.int32, device=dev())   # nothing ever sets it
    st = status_word()
    P.md_bounded_wait(flag, 2000, st)                        # ~2000 polls, well under a second
    torch.cuda.synchronize()
    assert P.md_status_poll(st) & P.MD_ERR_TIMEOUT
    # a set flag ends the wait at once, no timeout
    flag.fill_(1)
    st.zero_()
    P.md_bounded_wait(flag, 2000, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0


def test_overflowed_list_is_flagged_and_regrown(P):
    # an undersized cap raises NBR_OVERFLOW; the host grows cap to the
    # reported maximum and rebuilds, and then the run is clean
    import torch
    c = W.lj_small()
    s = P.md_space_periodic(3, [c.L] * 3)
    rd = to_dev(c.r, torch.float32)
    st = status_word()
    nl = P.NeighborList(s, c.N, 2.5, 0.3, 40)
    nl.build(rd, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) & P.MD_ERR_NBR_OVERFLOW
    need = nl.stats()[1]
    cap = ((int(need * 1.25) + 31) // 32) * 32
    st.zero_()
    nl = P.NeighborList(s, c.N, 2.5, 0.3, cap)
    nl.build(rd, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0 and nl.stats()[1] == need


def test_corrupted_row_entry_is_reported_with_bounds_checks(P):
    # with the bounds-checked pair kernels (md_set_pair_options bit 1) a row
    # entry outside [0, N) is skipped and reported as MD_ERR_BOUNDS; nothing
    # reads outside the positions, the context stays usable, and every other
    # particle's force keeps its bits
    import torch
    c = W.lj_small()
    s = P.md_space_periodic(3, [c.L] * 3)
    nl = P.NeighborList(s, c.N, 2.5, 0.3, 128)
    r = to_dev(c.r)
    st = status_word()
    nl.build(r, st)
    f0 = torch.zeros_like(r)
    P.md_energy_forces(s, P.lj_pot(), r, nl.plan, f0, None, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    nl.nbr[5, 2] = c.N + 1000
    nl.nbr[9, 0] = -3
    f1 = torch.zeros_like(r)
    try:
        P.md_set_pair_options(3)
        P.md_energy_forces(s, P.lj_pot(), r, nl.plan, f1, None, st)
        torch.cuda.synchronize()
    finally:
        P.md_set_pair_options(1)
    assert P.md_status_poll(st) == P.MD_ERR_BOUNDS
    a, b = f1.cpu().numpy(), f0.cpu().numpy()
    keep = np.ones(c.N, bool)
    keep[[5, 9]] = False
    np.testing.assert_array_equal(a[keep], b[keep])
    assert np.all(np.isfinite(a[[5, 9]]))
    # the context still works: a fresh list and the default kernels
    st2 = status_word()
    nl.build(r, st2)
    P.md_energy_forces(s, P.lj_pot(), r, nl.plan, f1, None, st2)
    torch.cuda.synchronize()
    assert P.md_status_poll(st2) == 0
    np.testing.assert_array_equal(f1.cpu().numpy(), b)
