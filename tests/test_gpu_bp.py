"""GPU parity: the learned potential (Sec. 3.2.4, 4.1) -- symmetry-function
descriptors, per-atom network, forces, descriptor JVP and the energy+force
training gradient (double backward) -- through the C ABI, against the FP64
autograd oracle."""
import numpy as np
import pytest

import oracle.bp as B
import workloads as W
from gpu_helpers import dev, force_error, status_word, to_dev

pytestmark = pytest.mark.gpu

SKIN = 0.3


@pytest.fixture(scope="module")
def P():
    import paper_1912_04232_b300 as P
    return P


def pack(p):
    return np.concatenate([p["W1"].numpy().ravel(), p["b1"].numpy(), p["W2"].numpy().ravel(), p["b2"].numpy(),
                           p["w3"].numpy(), np.atleast_1d(p["b3"].numpy())]).astype(np.float32)


def f32_params(p):
    """The oracle's parameters rounded to FP32 (what the GPU sees)."""
    import torch
    return {k: torch.as_tensor(v.numpy().astype(np.float32).astype(np.float64)) for k, v in p.items()}


def _col_err(a, ref):
    """Largest error per descriptor column relative to that column's scale
    (floored at 1e-3 of the largest column scale, for near-empty columns)."""
    scale = np.abs(ref).max(axis=0)
    scale = np.maximum(scale, 1e-3 * scale.max())
    return float((np.abs(a - ref) / scale).max())


def _norm(G):
    mu = G.mean(0).astype(np.float32)
    sd = (G.std(0) + 0.05).astype(np.float32)
    return mu, sd


def _snapshot(n_side=2, seed=0, jitter=0.25):
    si = W.sw_silicon(n_side, T_K=0, jitter=jitter, seed=seed)
    return si.r, si.L


def _list(P, r, L, cap=48):
    import torch
    s = P.md_space_periodic(3, [L] * 3)
    nl = P.NeighborList(s, r.shape[0], B.R_C, SKIN, cap)
    rd = to_dev(r, torch.float32)
    st = status_word()
    nl.build(rd, st)
    return s, nl, rd, st


def _oracle_G(r, L):
    import torch
    x = np.asarray(r, np.float64)[:, :3]
    return B.descriptors(torch.tensor(x), L, *B.triplets(*B.pairs_within(x, L), len(x))).numpy()


@pytest.mark.parametrize("n_side,seed", [(2, 0), (4, 1)])
def test_descriptors_match_oracle(P, n_side, seed):
    import torch
    r, L = _snapshot(n_side, seed)
    s, nl, rd, st = _list(P, r, L)
    G = torch.zeros((r.shape[0], 16), dtype=torch.float32, device=dev())
    P.md_bp_descriptors(s, rd, nl.plan, 0, G, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    Go = _oracle_G(r, L)
    assert _col_err(G.cpu().numpy(), Go) <= 2e-5


def _model(P, r, L, seed=0):
    import torch
    p = B.init_params(seed)
    G = _oracle_G(r, L)
    mu, sd = _norm(G)
    params = to_dev(pack(p), torch.float32)
    norm = to_dev(np.concatenate([mu, sd]), torch.float32)
    return p, mu, sd, params, norm


@pytest.mark.parametrize("lists", [False, True])
@pytest.mark.parametrize("n_side,seed", [(2, 2), (4, 3)])
def test_network_energy_and_forces_match_oracle(P, n_side, seed, lists):
    # lists: the descriptor kernel stores the partner lists the force gather reads
    import torch
    r, L = _snapshot(n_side, seed)
    s, nl, rd, st = _list(P, r, L)
    p, mu, sd, params, norm = _model(P, r, L, seed)
    m = P.BPModel(params, norm, r.shape[0], lists=lists)
    f = torch.zeros((r.shape[0], 4), dtype=torch.float32, device=dev())
    E = torch.zeros(1, dtype=torch.float64, device=dev())
    P.md_energy_forces(s, m.pot, rd, nl.plan, f, E, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    t64 = lambda a: __import__("torch").as_tensor(a.astype(np.float64))
    Eo, Fo, Eio, _ = B.energy_forces(r, L, f32_params(p), t64(mu), t64(sd))
    assert force_error(f.cpu().numpy(), Fo) <= 1e-4
    np.testing.assert_allclose(m.Ei.cpu().numpy(), Eio, rtol=0, atol=1e-5 * np.abs(Eio).max())
    assert abs(E.item() - Eo) <= 1e-5 * abs(Eo)


def test_partner_lists_give_the_same_forces(P):
    # the same triplets with the same FP32 vectors in both forms; only the
    # order of each atom's sums differs
    import torch
    r, L = _snapshot(5, 9, jitter=0.3)
    s, nl, rd, st = _list(P, r, L)
    p, mu, sd, params, norm = _model(P, r, L, 9)
    out = []
    for lists in (False, True):
        m = P.BPModel(params, norm, r.shape[0], lists=lists)
        f = torch.zeros((r.shape[0], 4), dtype=torch.float32, device=dev())
        E = torch.zeros(1, dtype=torch.float64, device=dev())
        P.md_energy_forces(s, m.pot, rd, nl.plan, f, E, st)
        torch.cuda.synchronize()
        assert P.md_status_poll(st) == 0
        out.append((f.cpu().numpy(), E.item()))
    (f0, E0), (f1, E1) = out
    assert np.abs(f1[:, :3] - f0[:, :3]).max() <= 2e-6 * np.abs(f0[:, :3]).max()
    assert E1 == E0   # the energies come from the network, before the force gather


def test_descriptor_jvp_matches_oracle(P):
    import torch
    r, L = _snapshot(2, 4)
    s, nl, rd, st = _list(P, r, L)
    rng = np.random.default_rng(0)
    dF = np.zeros((r.shape[0], 4), np.float32)
    dF[:, :3] = rng.normal(size=(r.shape[0], 3))
    V = torch.zeros((r.shape[0], 16), dtype=torch.float32, device=dev())
    P.md_bp_jvp(s, rd, nl.plan, 0, to_dev(dF), V, st)
    torch.cuda.synchronize()
    x = torch.tensor(np.asarray(r, np.float64)[:, :3])
    graph = B.triplets(*B.pairs_within(x.numpy(), L), len(x))
    _, Vo = torch.autograd.functional.jvp(lambda y: B.descriptors(y, L, *graph), x,
                                          torch.tensor(dF[:, :3].astype(np.float64)))
    Vo = Vo.numpy()
    assert _col_err(V.cpu().numpy(), Vo) <= 1e-4


def _training_case(P, wF=0.7):
    """Two 64-atom silicon snapshots through the GPU forward pass, loss and
    descriptor JVP; returns the training kernels' inputs and the FP64
    oracle's loss and gradient (double backward)."""
    import torch
    S, n_side = 2, 2
    snaps = [_snapshot(n_side, 10 + k) for k in range(S)]
    L = snaps[0][1]
    n = snaps[0][0].shape[0]
    p, mu, sd, params, norm = _model(P, snaps[0][0], L, seed=5)
    # references: the SW energies/forces of each snapshot (oracle)
    import oracle as O
    refs = [O.sw(r, L) for r, _ in snaps]
    rs = np.concatenate([r for r, _ in snaps]).astype(np.float32)
    N = S * n
    # one neighbor list per snapshot, local indices, concatenated rows
    s = P.md_space_periodic(3, [L] * 3)
    plan = P.md_nbr_plan(s, n, B.R_C, SKIN, 48)
    nbr = torch.zeros((N, 48), dtype=torch.int32, device=dev())
    cnt = torch.zeros(N, dtype=torch.int32, device=dev())
    rref = torch.zeros((N, 4), dtype=torch.float32, device=dev())
    ws = torch.empty(int(plan.ws_bytes) + 256, dtype=torch.uint8, device=dev())
    wsv = ws[(-ws.data_ptr()) % 256:][: int(plan.ws_bytes)]
    rd = to_dev(rs, torch.float32)
    st = status_word()
    for k in range(S):
        sl = slice(k * n, (k + 1) * n)
        P.md_nbr_bind(plan, nbr[sl], cnt[sl], rref[sl], wsv)
        P.md_neighbor_list_build(s, rd[sl], plan, st)
    comb = P.md_nbr.from_buffer_copy(plan)
    comb.N = N
    comb.nbr, comb.cnt, comb.rref = nbr.data_ptr(), cnt.data_ptr(), rref.data_ptr()
    G = torch.zeros((N, 16), dtype=torch.float32, device=dev())
    Ei = torch.zeros(N, dtype=torch.float32, device=dev())
    dEdG = torch.zeros((N, 16), dtype=torch.float32, device=dev())
    F = torch.zeros((N, 4), dtype=torch.float32, device=dev())
    Fref = np.zeros((N, 4), np.float32)
    Fref[:, :3] = np.concatenate([rf[1] for rf in refs])
    Eref = np.array([rf[0] for rf in refs])
    cE = torch.zeros(N, dtype=torch.float32, device=dev())
    dF = torch.zeros((N, 4), dtype=torch.float32, device=dev())
    loss = torch.zeros(2 * S, dtype=torch.float64, device=dev())
    V = torch.zeros((N, 16), dtype=torch.float32, device=dev())
    P.md_bp_descriptors(s, rd, comb, n, G, st)
    P.md_bp_mlp_infer(params, norm, G, N, Ei, dEdG)
    P.md_bp_forces(s, rd, comb, n, dEdG, Ei, F, None, st)
    P.md_bp_loss_prep(Ei, F, to_dev(Fref), to_dev(Eref), S, n, wF, cE, dF, loss)
    P.md_bp_jvp(s, rd, comb, n, dF, V, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    t64 = lambda a: torch.as_tensor(np.asarray(a, np.float64))
    batch = [(r, L, rf[0], rf[1]) for (r, _), rf in zip(snaps, refs)]
    lo, go = B.loss_and_grads(batch, f32_params(p), t64(mu), t64(sd), w_F=wF)
    g_o = np.concatenate([go[k].numpy().ravel() for k in ("W1", "b1", "W2", "b2", "w3")] +
                         [np.atleast_1d(go["b3"].numpy())])
    return dict(params=params, norm=norm, G=G, V=V, cE=cE, N=N, loss=loss, lo=lo, g_o=g_o)


# parameter blocks of the packed vector: W1, b1, W2, b2, w3, b3
BLOCKS = [(0, 1024), (1024, 1088), (1088, 5184), (5184, 5248), (5248, 5312), (5312, 5313)]


def _grad_errors(g, ref):
    """Relative error of the whole gradient and of each parameter block
    (each against its own norm), and the cosine with the reference."""
    rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    blocks = [np.linalg.norm(g[a:b] - ref[a:b]) / np.linalg.norm(ref[a:b]) for a, b in BLOCKS]
    cos = g @ ref / (np.linalg.norm(g) * np.linalg.norm(ref))
    return rel, max(blocks), cos


def test_training_gradient_matches_oracle_double_backward(P):
    import torch
    c = _training_case(P)
    scratch = torch.empty(P.md_bp_train_scratch_size(c["N"]), dtype=torch.uint8, device=dev())
    grad = torch.zeros(P.BP_NPARAMS, dtype=torch.float32, device=dev())
    P.md_bp_mlp_train(c["params"], c["norm"], c["G"], c["V"], c["cE"], 1.0, c["N"], scratch, grad)
    torch.cuda.synchronize()
    assert abs(c["loss"].sum().item() - c["lo"]) <= 1e-4 * c["lo"]
    rel, _, cos = _grad_errors(grad.cpu().numpy().astype(np.float64), c["g_o"])
    assert rel <= 1e-3 and cos >= 0.99999, (rel, cos)


def test_tensor_core_training_gradient_matches_oracle(P):
    # tcgen05 BF16 MMAs with FP32 accumulation: the weights, inputs and
    # per-atom factors rounded to 8 significant bits; every parameter block
    # within 2e-2 of its norm, cosine >= 0.999
    import torch
    c = _training_case(P)
    scratch = torch.empty(P.md_bp_train_scratch_size(c["N"]), dtype=torch.uint8, device=dev())
    grad = torch.zeros(P.BP_NPARAMS, dtype=torch.float32, device=dev())
    st = status_word()
    P.md_bp_mlp_train_tc(c["params"], c["norm"], c["G"], c["V"], c["cE"], 1.0, c["N"], scratch, grad, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    rel, worst_block, cos = _grad_errors(grad.cpu().numpy().astype(np.float64), c["g_o"])
    assert rel <= 2e-2 and worst_block <= 2e-2 and cos >= 0.999, (rel, worst_block, cos)


@pytest.mark.parametrize("N", [1037, 40000])
def test_tensor_core_training_gradient_matches_fp32_kernel(P, N):
    # many tiles (40,000 atoms: up to three per CTA, accumulated in tensor
    # memory) and a ragged last tile, against the FP32 kernel on the same
    # inputs; two calls give the same bits (fixed-order sum over CTAs)
    import torch
    rng = np.random.default_rng(N)
    p = B.init_params(3)
    G = rng.normal(size=(N, 16)).astype(np.float32) * 0.5 + 1.0
    mu, sd = _norm(G)
    V = (rng.normal(size=(N, 16)) * 0.05).astype(np.float32)
    cE = (rng.normal(size=N) * 1e-3).astype(np.float32)
    params = to_dev(pack(p), torch.float32)
    norm = to_dev(np.concatenate([mu, sd]), torch.float32)
    Gd, Vd, cEd = to_dev(G, torch.float32), to_dev(V, torch.float32), to_dev(cE, torch.float32)
    scratch = torch.empty(P.md_bp_train_scratch_size(N), dtype=torch.uint8, device=dev())
    g32 = torch.zeros(P.BP_NPARAMS, dtype=torch.float32, device=dev())
    gtc = torch.zeros_like(g32)
    gtc2 = torch.zeros_like(g32)
    st = status_word()
    P.md_bp_mlp_train(params, norm, Gd, Vd, cEd, 0.8, N, scratch, g32)
    P.md_bp_mlp_train_tc(params, norm, Gd, Vd, cEd, 0.8, N, scratch, gtc, st)
    P.md_bp_mlp_train_tc(params, norm, Gd, Vd, cEd, 0.8, N, scratch, gtc2, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    ref = g32.cpu().numpy().astype(np.float64)
    rel, worst_block, cos = _grad_errors(gtc.cpu().numpy().astype(np.float64), ref)
    assert rel <= 2e-2 and worst_block <= 2e-2 and cos >= 0.999, (rel, worst_block, cos)
    assert torch.equal(gtc, gtc2)


@pytest.mark.parametrize("N", [1037, 64000])
def test_tensor_core_network_matches_fp32_network(P, N):
    # tcgen05 BF16 MMAs (FP32 accumulate) vs the FP32 CUDA-core network on
    # the same inputs; BF16 rounds inputs, weights and hidden activations to
    # 8 significant bits, so agreement is to about 1e-2 of each output's scale
    import torch
    rng = np.random.default_rng(N)
    p = B.init_params(7)
    G = rng.normal(size=(N, 16)).astype(np.float32) * 0.5 + 1.0
    mu, sd = _norm(G)
    params = to_dev(pack(p), torch.float32)
    norm = to_dev(np.concatenate([mu, sd]), torch.float32)
    Gd = to_dev(G, torch.float32)
    E32 = torch.zeros(N, dtype=torch.float32, device=dev())
    D32 = torch.zeros((N, 16), dtype=torch.float32, device=dev())
    Etc = torch.zeros(N, dtype=torch.float32, device=dev())
    Dtc = torch.zeros((N, 16), dtype=torch.float32, device=dev())
    st = status_word()
    P.md_bp_mlp_infer(params, norm, Gd, N, E32, D32)
    P.md_bp_mlp_infer_tc(params, norm, Gd, N, Etc, Dtc, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    e32, etc = E32.cpu().numpy(), Etc.cpu().numpy()
    d32, dtc = D32.cpu().numpy(), Dtc.cpu().numpy()
    assert np.abs(etc - e32).max() <= 2e-2 * np.abs(e32).max()
    assert _col_err(dtc, d32) <= 3e-2
    # and it is really computing: correlation with the FP32 result
    assert np.corrcoef(etc, e32)[0, 1] > 0.999


@pytest.mark.parametrize("n_side,lists", [(2, True), (5, False), (5, True), (20, True)])
def test_fused_descriptor_network_kernel_equals_separate_kernels(P, n_side, lists):
    # on the tensor cores an evaluation computes the descriptors inside the
    # network kernel; its per-atom energies and input gradients must be the
    # separate kernels' bit for bit (64 atoms: one partial tile; 1,000 atoms:
    # 7 full tiles and a ragged one; 64,000 atoms: 500 tiles)
    # (kernel against kernel: the inputs' normalisation comes from the GPU
    # descriptors, no oracle is needed)
    import torch
    r, L = _snapshot(n_side, 21, jitter=0.3)
    N = r.shape[0]
    s, nl, rd, st = _list(P, r, L)
    G0 = torch.zeros((N, 16), dtype=torch.float32, device=dev())
    P.md_bp_descriptors(s, rd, nl.plan, 0, G0, st)
    mu, sd = _norm(G0.cpu().numpy().astype(np.float64))
    params = to_dev(pack(B.init_params(21)), torch.float32)
    norm = to_dev(np.concatenate([mu, sd]), torch.float32)
    m = P.BPModel(params, norm, N, lists=lists)
    f = torch.zeros((N, 4), dtype=torch.float32, device=dev())
    P.md_bp_set_tensor_cores(True)
    try:
        P.md_energy_forces(s, m.pot, rd, nl.plan, f, None, st)
    finally:
        P.md_bp_set_tensor_cores(False)
    G = torch.zeros((N, 16), dtype=torch.float32, device=dev())
    Ei = torch.zeros(N, dtype=torch.float32, device=dev())
    D = torch.zeros((N, 16), dtype=torch.float32, device=dev())
    P.md_bp_descriptors(s, rd, nl.plan, 0, G, st)
    P.md_bp_mlp_infer_tc(params, norm, G, N, Ei, D, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    assert torch.equal(m.Ei, Ei)
    assert torch.equal(m.dEdG, D)


def test_tensor_core_forces_match_oracle(P):
    import torch
    r, L = _snapshot(4, 8)
    s, nl, rd, st = _list(P, r, L)
    p, mu, sd, params, norm = _model(P, r, L, 8)
    m = P.BPModel(params, norm, r.shape[0])
    f = torch.zeros((r.shape[0], 4), dtype=torch.float32, device=dev())
    E = torch.zeros(1, dtype=torch.float64, device=dev())
    P.md_bp_set_tensor_cores(True)
    try:
        P.md_energy_forces(s, m.pot, rd, nl.plan, f, E, st)
        torch.cuda.synchronize()
    finally:
        P.md_bp_set_tensor_cores(False)
    assert P.md_status_poll(st) == 0
    t64 = lambda a: torch.as_tensor(a.astype(np.float64))
    Eo, Fo, Eio, _ = B.energy_forces(r, L, f32_params(p), t64(mu), t64(sd))
    assert force_error(f.cpu().numpy(), Fo) <= 3e-2
    # the total is a cancelling sum of per-atom terms: compare it on their scale
    np.testing.assert_allclose(m.Ei.cpu().numpy(), Eio, rtol=0, atol=2e-2 * np.abs(Eio).max())
    assert abs(E.item() - Eo) <= 1e-2 * np.abs(Eio).sum()


def test_fused_evaluation_on_concatenated_systems_equals_each_alone(P):
    # equal-size snapshots concatenated (rows local to each, md_bp_model
    # sys_n) through md_energy_forces on the tensor cores: every atom's
    # energy, input gradient and force must be the ones of its snapshot
    # evaluated alone, bit for bit
    import types
    import torch
    import paper_1912_04232_b300.learned as LP
    S = 3
    snaps = [W.sw_silicon(3, T_K=0, jitter=0.3, seed=31 + k) for k in range(S)]
    n, L = snaps[0].N, snaps[0].L
    ds = types.SimpleNamespace(r=to_dev(np.stack([s.r for s in snaps]), torch.float32), n=n, L=L)
    LP.build_lists(ds)
    nb = LP.batch_list_view(ds, 0, S)
    space = P.md_space_periodic(3, [L] * 3)
    st = status_word()
    G0 = torch.zeros((S * n, 16), dtype=torch.float32, device=dev())
    P.md_bp_descriptors(space, ds.r.reshape(S * n, 4), nb, n, G0, st)
    mu, sd = _norm(G0.cpu().numpy().astype(np.float64))
    params = to_dev(pack(B.init_params(31)), torch.float32)
    norm = to_dev(np.concatenate([mu, sd]), torch.float32)
    P.md_bp_set_tensor_cores(True)
    try:
        m = P.BPModel(params, norm, S * n, sys_n=n)
        f = torch.zeros((S * n, 4), dtype=torch.float32, device=dev())
        P.md_energy_forces(space, m.pot, ds.r.reshape(S * n, 4), nb, f, None, st)
        alone = []
        for k in range(S):
            s1, nl1, rd1, st1 = _list(P, snaps[k].r, L)
            m1 = P.BPModel(params, norm, n)
            f1 = torch.zeros((n, 4), dtype=torch.float32, device=dev())
            P.md_energy_forces(s1, m1.pot, rd1, nl1.plan, f1, None, st1)
            torch.cuda.synchronize()
            assert P.md_status_poll(st1) == 0
            alone.append((m1.Ei.clone(), m1.dEdG.clone(), f1.clone()))
    finally:
        P.md_bp_set_tensor_cores(False)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    for k, (Ei, D, f1) in enumerate(alone):
        sl = slice(k * n, (k + 1) * n)
        assert torch.equal(m.Ei[sl], Ei)
        assert torch.equal(m.dEdG[sl], D)
        assert torch.equal(f[sl], f1)


@pytest.mark.parametrize("lists", [False, True])
def test_more_partners_than_slots_is_reported(P, lists):
    # 60 atoms within 1.4 A of one point: more than the 48 partners inside
    # R_c an atom keeps; the list (cap 128) does not overflow
    import torch
    si = W.sw_silicon(3, T_K=0, jitter=0.0, seed=0)
    r = si.r.copy()
    rng = np.random.default_rng(6)
    d = rng.normal(size=(60, 3))
    d *= (1.4 * rng.uniform(0.2, 1.0, size=(60, 1)) ** (1 / 3)) / np.linalg.norm(d, axis=1, keepdims=True)
    r[:60, :3] = (np.float32(si.L / 2) + d).astype(np.float32)
    s, nl, rd, st = _list(P, r, si.L, cap=128)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    params = to_dev(pack(B.init_params(3)), torch.float32)
    norm = to_dev(np.concatenate([np.zeros(16), np.ones(16)]).astype(np.float32), torch.float32)
    m = P.BPModel(params, norm, si.N, lists=lists)
    f = torch.zeros((si.N, 4), dtype=torch.float32, device=dev())
    P.md_energy_forces(s, m.pot, rd, nl.plan, f, None, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) & P.MD_ERR_NBR_OVERFLOW
