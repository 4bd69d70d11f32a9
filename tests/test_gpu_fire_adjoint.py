"""GPU parity of the FIRE adjoint (Sec. 3.3.1 minimiser through the Sec. 4.2
/ App. A packing): E_final and dE_final/dD by the hand-written reverse mode
with checkpoint replay, against the FP64 autograd oracle; identical for
every checkpoint interval; the forward equal to md_minimize_fire."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import dev, status_word, to_dev
from oracle import fire_adjoint as FA

pytestmark = pytest.mark.gpu

SKIN = 0.3


@pytest.fixture(scope="module")
def P():
    import paper_1912_04232_b300 as P
    return P


def _run(P, p, D, T, K, phi=0.9):
    import torch
    N = p.N
    L64 = O.packing_box(N, D, phi)
    L = W.f32(L64)
    s = P.md_space_periodic(2, [L, L])
    nl = P.NeighborList(s, N, max(D, 1.0), SKIN, 64, canonical=True)
    s0 = np.zeros((N, 4), np.float32)
    s0[:, :2] = p.s0
    s0d = to_dev(s0, torch.float32)
    r = torch.zeros((N, 4), dtype=torch.float32, device=dev())
    v = torch.zeros_like(r)
    f = torch.zeros_like(r)
    ws = torch.empty(P.md_fire_adjoint_workspace_size(N, T, K) + 256, dtype=torch.uint8, device=dev())
    off = (-ws.data_ptr()) % 256
    wsv = ws[off:]
    out = torch.zeros(2, dtype=torch.float64, device=dev())
    st = status_word()
    P.md_minimize_fire_adjoint(s, P.soft_pot(), P.fire_params(), nl.plan, s0d, N // 2, D, 1.0, phi, T, K, r, v, f,
                               wsv, out, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    return out.cpu().numpy(), r.cpu().numpy(), (s, nl, s0d, L)


@pytest.mark.parametrize("N,D,T,seed", [(32, 1.3, 60, 0), (64, 1.2, 120, 1), (48, 1.4, 100, 2)])
def test_fire_adjoint_matches_fp64_autograd(P, N, D, T, seed):
    p = W.packing_2d(N=N, D=D, seed=seed)
    K = int(math.ceil(math.sqrt(T)))
    (E, g), r, _ = _run(P, p, D, T, K)
    Eo, go, hist = FA.fire_packing(p.s0, D, N // 2, T=T)
    assert any(h[2] for h in hist)
    assert abs(E - Eo) <= 1e-4 * abs(Eo) + 1e-7, (E, Eo)
    assert abs(g - go) <= 2e-3 * abs(go) + 1e-6, (g, go)


def test_fire_adjoint_app_a_packing_within_oracle_sensitivity(P):
    # App. A's packing (128 disks, 300 FIRE steps): dE/dD of a trajectory
    # this long is ill-conditioned at the size of FP32 rounding (the
    # oracle's own value moves by O(1) when s_0 moves by 3e-8), so the GPU
    # value is bounded by the oracle's spread over such perturbations
    p = W.packing_2d(N=128, D=1.4, seed=0)
    T = 300
    (E, g), _, _ = _run(P, p, 1.4, T, 18)
    rng = np.random.Generator(np.random.PCG64(11))
    Es, gs = [], []
    for k in range(6):
        s0 = p.s0 + (rng.uniform(-3e-8, 3e-8, p.s0.shape) if k else 0.0)
        Eo, go, _ = FA.fire_packing(s0, 1.4, 64, T=T)
        Es.append(Eo)
        gs.append(go)
    spread = max(gs) - min(gs)
    assert min(gs) - 0.5 * spread <= g <= max(gs) + 0.5 * spread, (g, gs)
    assert min(Es) - 1e-4 * abs(Es[0]) <= E <= max(Es) + 1e-4 * abs(Es[0])


def test_fire_adjoint_identical_for_every_checkpoint_interval(P):
    p = W.packing_2d(N=64, D=1.25, seed=5)
    T = 60
    res = [_run(P, p, 1.25, T, K)[0] for K in (1, 7, T)]
    for x in res[1:]:
        assert x[0] == res[0][0] and x[1] == res[0][1]


def test_fire_adjoint_forward_equals_minimize_fire(P):
    import torch
    p = W.packing_2d(N=64, D=1.3, seed=6)
    T = 80
    (E, g), rT, (s, nl, s0d, L) = _run(P, p, 1.3, T, 9)
    r = torch.zeros((p.N, 4), dtype=torch.float32, device=dev())
    r[:, :2] = s0d[:, :2] * L
    r[:, 3] = torch.where(torch.arange(p.N, device=dev()) < p.N // 2, 1.3, 1.0)
    v = torch.zeros_like(r)
    f = torch.zeros_like(r)
    st = status_word()
    state = torch.zeros(P.md_fire_state_bytes() + 256, dtype=torch.uint8, device=dev())
    off = (-state.data_ptr()) % 256
    Es = torch.zeros(T + 1, dtype=torch.float64, device=dev())
    nl.build(r, st)
    P.md_minimize_fire(s, P.soft_pot(), P.fire_params(), T, r, v, f, nl.plan, state[off:], True, Es, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    np.testing.assert_array_equal(r.cpu().numpy(), rT)
    assert Es.cpu().numpy()[T] == E


def test_fire_adjoint_graph_replay_and_host_launches_agree_bitwise(P):
    # with loop graphs on, a call is captured once per argument set and
    # replayed; the capture, its replay and plain host launches give the
    # same bits
    import torch
    N, D, T, K = 128, 1.4, 300, 18
    p = W.packing_2d(N=N, D=D, phi=0.9, seed=3)
    L64 = O.packing_box(N, D, 0.9)
    L = W.f32(L64)
    s = P.md_space_periodic(2, [L, L])
    nl = P.NeighborList(s, N, D, SKIN, 64, canonical=True)
    s0 = np.zeros((N, 4), np.float32)
    s0[:, :2] = p.s0
    s0d = to_dev(s0, torch.float32)
    r, v, f = (torch.zeros((N, 4), dtype=torch.float32, device=dev()) for _ in range(3))
    ws = torch.empty(P.md_fire_adjoint_workspace_size(N, T, K) + 256, dtype=torch.uint8, device=dev())
    wsv = ws[(-ws.data_ptr()) % 256:]
    out = torch.zeros(2, dtype=torch.float64, device=dev())
    st = status_word()
    res = []
    try:
        for graphs in (True, True, False):
            P.md_set_loop_graphs(graphs)
            P.md_minimize_fire_adjoint(s, P.soft_pot(), P.fire_params(), nl.plan, s0d, N // 2, D, 1.0, 0.9, T, K,
                                       r, v, f, wsv, out, st)
            torch.cuda.synchronize()
            assert P.md_status_poll(st) == 0
            res.append([x.cpu().numpy().copy() for x in (out, r, v, f)])
    finally:
        P.md_set_loop_graphs(True)
    for other in res[1:]:
        for a, b in zip(res[0], other):
            np.testing.assert_array_equal(a, b)


def test_graph_cache_eviction_keeps_results(P):
    # a sweep over more argument sets than the adjoint keeps graphs for (32):
    # the oldest captured graphs are evicted on the way, and every call still
    # returns what plain host launches return for the same arguments
    import torch
    N, T, K = 32, 12, 4
    p = W.packing_2d(N=N, D=1.2, phi=0.9, seed=4)
    s0 = np.zeros((N, 4), np.float32)
    s0[:, :2] = p.s0
    s0d = to_dev(s0, torch.float32)
    r, v, f = (torch.zeros((N, 4), dtype=torch.float32, device=dev()) for _ in range(3))
    ws = torch.empty(P.md_fire_adjoint_workspace_size(N, T, K) + 256, dtype=torch.uint8, device=dev())
    wsv = ws[(-ws.data_ptr()) % 256:]
    out = torch.zeros(2, dtype=torch.float64, device=dev())
    st = status_word()
    Ds = [1.05 + 0.01 * k for k in range(36)]

    def call(D):
        L64 = O.packing_box(N, D, 0.9)
        L = W.f32(L64)
        s = P.md_space_periodic(2, [L, L])
        nl = P.NeighborList(s, N, D, SKIN, 32, canonical=True)
        P.md_minimize_fire_adjoint(s, P.soft_pot(), P.fire_params(), nl.plan, s0d, N // 2, D, 1.0, 0.9, T, K,
                                   r, v, f, wsv, out, st)
        torch.cuda.synchronize()
        assert P.md_status_poll(st) == 0
        return out.cpu().numpy().copy()

    graphs = [call(D) for D in Ds]
    try:
        P.md_set_loop_graphs(False)
        host = [call(D) for D in (Ds[0], Ds[17], Ds[-1])]
    finally:
        P.md_set_loop_graphs(True)
    for g, h in zip((graphs[0], graphs[17], graphs[-1]), host):
        np.testing.assert_array_equal(g, h)
