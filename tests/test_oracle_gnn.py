"""Pins of the graph-network oracle (Sec. 3.2.4 / 4.1 reading): weights
chosen so the network reduces to models with closed forms (an embedding of
the smooth coordination number; a second step that reads the sender's or
the receiver's node state; an encoder read through one message), forces
against central finite differences, translation and permutation invariance,
zero net force and continuity as a pair crosses the cutoff.  The flat
parameter offsets are computed here, independently of the oracle's
unpacking."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import gnn as G

RC = 3.77


def _silu(x):
    return x / (1.0 + np.exp(-x))


def _dsilu(x):
    s = 1.0 / (1.0 + np.exp(-x))
    return s * (1.0 + x * (1.0 - s))


def _s(r):
    x = np.pi * np.minimum(r, RC) / RC
    return np.where(r < RC, 0.5 * (np.cos(x) + 1.0), 0.0)


def _ds(r):
    x = np.pi * np.minimum(r, RC) / RC
    return np.where(r < RC, -0.5 * np.pi / RC * np.sin(x), 0.0)


class Flat:
    """Flat parameter vector with named blocks at explicitly computed
    offsets: W_enc, b_enc, u, then per step A (H x 3H), a, B (H x 2H), b,
    then D, d, w, c."""

    def __init__(self, H, T):
        self.H, self.T = H, T
        self.p = np.zeros(5 * H + T * (5 * H * H + 2 * H) + H * H + 2 * H + 1)

    def _layer(self, t):
        return 5 * self.H + t * (5 * self.H ** 2 + 2 * self.H)

    def set(self, name, val, t=0):
        H = self.H
        o = {"W_enc": (0, (H, 3)), "b_enc": (3 * H, (H,)), "u": (4 * H, (H,)),
             "A": (self._layer(t), (H, 3 * H)), "a": (self._layer(t) + 3 * H * H, (H,)),
             "B": (self._layer(t) + 3 * H * H + H, (H, 2 * H)), "b": (self._layer(t) + 5 * H * H + H, (H,)),
             "D": (self._layer(self.T), (H, H)), "d": (self._layer(self.T) + H * H, (H,)),
             "w": (self._layer(self.T) + H * H + H, (H,)), "c": (self._layer(self.T) + H * H + 2 * H, (1,))}[name]
        n = int(np.prod(o[1]))
        self.p[o[0]:o[0] + n] = np.asarray(val, np.float64).reshape(-1)


def _config(N, L, seed, min_sep=1.2):
    rng = np.random.Generator(np.random.PCG64(seed))
    R = []
    while len(R) < N:
        x = rng.uniform(0, L, 3)
        if all(np.linalg.norm((x - y) - L * np.round((x - y) / L)) > min_sep for y in R):
            R.append(x)
    return np.array(R)


def _pairs(R, L):
    """All ordered pairs i != j: distances and R_j - R_i (minimum image)."""
    d = R[None, :, :] - R[:, None, :]
    d -= L * np.round(d / L)
    r = np.sqrt((d ** 2).sum(-1))
    np.fill_diagonal(r, np.inf)
    return d, r


def _coordination_params(H, T, rng):
    f = Flat(H, T)
    alpha, gamma, b1 = rng.normal(0, 1, H), rng.normal(0, 1, H), rng.normal(0, 0.3, H)
    f.set("b_enc", rng.normal(0, 1, H))
    f.set("u", rng.normal(0, 1, H))
    f.set("a", alpha, 0)
    B = np.zeros((H, 2 * H))
    B[:, H:] = np.diag(gamma)
    f.set("B", B, 0)
    f.set("b", b1, 0)
    return f, _silu(alpha), gamma, b1


def test_coordination_number_model():
    # one step, every weight but the biases and diagonal read-outs zero:
    # E = sum_i f(n_i), n_i = sum_j s(r_ij), a smooth coordination number
    H, L = 4, 9.0
    rng = np.random.Generator(np.random.PCG64(1))
    f, c1, gamma, b1 = _coordination_params(H, 1, rng)
    delta, d0, w = rng.normal(0, 1, H), rng.normal(0, 0.3, H), rng.normal(0, 1, H)
    f.set("D", np.diag(delta))
    f.set("d", d0)
    f.set("w", w)
    f.set("c", [0.37])
    R = _config(40, L, 2)
    d, r = _pairs(R, L)
    n = _s(r).sum(1)
    z1 = gamma * c1 * n[:, None] + b1
    z2 = delta * _silu(z1) + d0
    Ei = _silu(z2) @ w + 0.37
    fp = (_dsilu(z2) * delta * _dsilu(z1) * gamma * c1) @ w          # f'(n_i)
    # dE/dR_k = sum_j (f'(n_k) + f'(n_j)) s'(r_kj) (R_k - R_j) / r_kj
    u = -d / r[:, :, None]
    dE = ((fp[:, None] + fp[None, :]) * _ds(r))[:, :, None] * u
    F = -dE.sum(1)
    E, Ei_o, F_o = G.energy_forces(R, L, f.p, H, 1, RC)
    np.testing.assert_allclose(Ei_o, Ei, rtol=0, atol=1e-12)
    assert abs(E - Ei.sum()) < 1e-10
    np.testing.assert_allclose(F_o, F, rtol=0, atol=1e-11)


@pytest.mark.parametrize("side", ["sender", "receiver"])
def test_second_step_reads_sender_or_receiver(side):
    # step 1 gives v_i = g(n_i); step 2 with A_s (or A_r) diagonal and all
    # else zero: m_i = sum_j s_ij silu(k g(n_j))   (sender)
    #            m_i = n_i silu(k g(n_i))          (receiver)
    H, L = 4, 9.0
    rng = np.random.Generator(np.random.PCG64(3))
    f, c1, gamma, b1 = _coordination_params(H, 2, rng)
    kappa, w = rng.normal(0, 1, H), rng.normal(0, 1, H)
    A = np.zeros((H, 3 * H))
    A[:, (2 * H if side == "sender" else H):][:, :H] = np.diag(kappa)
    f.set("A", A, 1)
    B = np.zeros((H, 2 * H))
    B[:, H:] = np.eye(H)
    f.set("B", B, 1)
    f.set("D", np.eye(H))
    f.set("w", w)
    R = _config(40, L, 4)
    d, r = _pairs(R, L)
    s = _s(r)
    n = s.sum(1)
    g = _silu(gamma * c1 * n[:, None] + b1)
    q = _silu(kappa * g)
    m = s @ q if side == "sender" else n[:, None] * q
    Ei = _silu(_silu(m)) @ w
    E, Ei_o, _ = G.energy_forces(R, L, f.p, H, 2, RC)
    np.testing.assert_allclose(Ei_o, Ei, rtol=0, atol=1e-12)


def test_encoder_direction_through_one_message():
    # one step with A_e = I, all else zero: m_i = sum_j s_ij silu(silu(W x_ij + b)),
    # x_ij = (R_j - R_i) / r_c  (the sign of x is seen by the read-out)
    H, L = 4, 9.0
    rng = np.random.Generator(np.random.PCG64(5))
    f = Flat(H, 1)
    Wenc, benc, w = rng.normal(0, 1, (H, 3)), rng.normal(0, 1, H), rng.normal(0, 1, H)
    f.set("W_enc", Wenc)
    f.set("b_enc", benc)
    A = np.zeros((H, 3 * H))
    A[:, :H] = np.eye(H)
    f.set("A", A, 0)
    B = np.zeros((H, 2 * H))
    B[:, H:] = np.eye(H)
    f.set("B", B, 0)
    f.set("D", np.eye(H))
    f.set("w", w)
    R = _config(30, L, 6)
    d, r = _pairs(R, L)
    e = _silu(_silu(d / RC @ Wenc.T + benc))                      # [N, N, H]
    m = (_s(r)[:, :, None] * e).sum(1)
    Ei = _silu(_silu(m)) @ w
    _, Ei_o, _ = G.energy_forces(R, L, f.p, H, 1, RC)
    np.testing.assert_allclose(Ei_o, Ei, rtol=0, atol=1e-12)


def _random_case(seed=7, N=30, L=8.0, H=8, T=2):
    p = W.gnn_params(H, T, seed=seed, out_scale=1.0).astype(np.float64)
    return _config(N, L, seed), L, p, H, T


def test_forces_match_finite_differences():
    R, L, p, H, T = _random_case()
    E, _, F = G.energy_forces(R, L, p, H, T, RC)
    edges = G.edges_within(R, L, RC)
    h = 1e-6
    for k in range(0, R.shape[0], 4):
        for c in range(3):
            Rp, Rm = R.copy(), R.copy()
            Rp[k, c] += h
            Rm[k, c] -= h
            fd = -(G.energy_forces(Rp, L, p, H, T, RC, edges)[0] - G.energy_forces(Rm, L, p, H, T, RC, edges)[0]) / (2 * h)
            assert abs(fd - F[k, c]) < 1e-6 * max(1.0, abs(F[k, c]))


def test_invariances_and_zero_net_force():
    R, L, p, H, T = _random_case(seed=8)
    E, Ei, F = G.energy_forces(R, L, p, H, T, RC)
    assert np.abs(F.sum(0)).max() < 1e-10
    shift = np.array([1.3, -2.9, 4.4])
    E2, Ei2, F2 = G.energy_forces(np.mod(R + shift, L), L, p, H, T, RC)
    assert abs(E2 - E) < 1e-10
    np.testing.assert_allclose(F2, F, rtol=0, atol=1e-10)
    perm = np.random.Generator(np.random.PCG64(0)).permutation(R.shape[0])
    E3, Ei3, F3 = G.energy_forces(R[perm], L, p, H, T, RC)
    assert abs(E3 - E) < 1e-10
    np.testing.assert_allclose(F3, F[perm], rtol=0, atol=1e-10)


def test_continuous_as_a_pair_crosses_the_cutoff():
    H, T = 8, 2
    p = W.gnn_params(H, T, seed=9, out_scale=1.0).astype(np.float64)
    L = 20.0
    lone = G.energy_forces(np.array([[5.0, 5.0, 5.0]]), L, p, H, T, RC)[0]
    for eps in (1e-3, 1e-4):
        inside = np.array([[5.0, 5.0, 5.0], [5.0 + RC * (1 - eps), 5.0, 5.0]])
        outside = np.array([[5.0, 5.0, 5.0], [5.0 + RC * (1 + eps), 5.0, 5.0]])
        Ein, _, Fin = G.energy_forces(inside, L, p, H, T, RC)
        Eout, _, Fout = G.energy_forces(outside, L, p, H, T, RC)
        assert abs(Eout - 2 * lone) < 1e-14
        assert np.all(Fout == 0.0)
        # s(r) ~ (pi eps / 2)^2 near the cutoff and s' ~ eps
        assert abs(Ein - Eout) < 10 * (math.pi * eps / 2) ** 2
        assert np.abs(Fin).max() < 10 * eps


def test_loss_gradient_matches_finite_differences():
    # the force-matching term needs second derivatives: check the double
    # backward against central differences of the loss itself
    H, T, L = 8, 2, 8.0
    p = W.gnn_params(H, T, seed=12, out_scale=1.0).astype(np.float64)
    batch = []
    for s in range(2):
        R = _config(20, L, 30 + s)
        rng = np.random.Generator(np.random.PCG64(40 + s))
        batch.append((R, L, rng.normal(0.0, 1.0), rng.normal(0.0, 0.1, size=(20, 3))))
    loss0, g = G.loss_and_grads(batch, p, H, T, RC, w_F=0.7)
    import torch
    f = lambda q: float(G.loss(batch, torch.tensor(q), H, T, RC, 0.7))
    h = 1e-6
    idx = list(range(0, 3 * H, 5)) + list(range(5 * H, 5 * H + 3 * H * H, 97)) + [len(p) - 2 - H, len(p) - 1]
    for k in idx:
        qp, qm = p.copy(), p.copy()
        qp[k] += h
        qm[k] -= h
        fd = (f(qp) - f(qm)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])), (k, fd, g[k])
