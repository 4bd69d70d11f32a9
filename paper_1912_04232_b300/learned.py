"""Learned potential workflow (Sec. 4.1): data from the plain Stillinger-
Weber simulator, training of the Behler-Parrinello network and of the graph
network with the energy + force loss, evaluation, and deployment in MD.

Every arithmetic step runs in libjmd kernels (Langevin/NVE integrators, SW
and learned forces, descriptors, network forward / double backward, loss
bookkeeping, Adam, statistics).  This module only sequences those calls and
owns the device buffers (torch tensors as storage).

Units: eV, Angstrom, fs; masses in eV fs^2 / A^2 (amu x 103.6427).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import jmd as J

SW_SI = (2.1683, 2.0951, 1.80, 21.0, 1.20, 7.049556277, 0.6022245584, 4.0, 0.0, -1.0 / 3.0)
SW_RC = SW_SI[2] * SW_SI[1]
MASS_SI = 28.0855 * 103.6427
KB = 8.617333262e-5
BP_RC = 3.77
SKIN = 0.3
CAP = 48
N_PARAMS = 5313


def _t():
    import torch
    return torch


@dataclass
class Dataset:
    r: "object"        # [S, n, 4] float32 (device)
    F: "object"        # [S, n, 4] float32 SW forces
    E: "object"        # [S] float64 SW energies
    T: np.ndarray      # temperature of each snapshot
    L: float
    n: int
    nbr: "object" = None   # [S*n, CAP] int32, rows local to each snapshot
    cnt: "object" = None   # [S*n] int32
    plan: "object" = None  # md_nbr for one snapshot (box, cap)
    ws: "object" = None


def generate_sw_dataset(temps, n_snap, stride=20, equil=2000, n_side=4, a=5.431, gamma=0.01, dt=1.0, seed=0,
                        device="cuda"):
    """SW silicon (8 n_side^3 atoms, diamond start) under BAOAB Langevin at
    each temperature; a snapshot (positions, SW forces and energy) every
    `stride` steps after `equil` steps."""
    torch = _t()
    import workloads as W
    S = len(temps) * n_snap
    si0 = W.sw_silicon(n_side, a=a, T_K=0.0)
    n, L = si0.N, si0.L
    space = J.md_space_periodic(3, [L] * 3)
    pot = J.sw_pot(SW_SI, N=n, device=device)
    R = torch.zeros((S, n, 4), dtype=torch.float32, device=device)
    F = torch.zeros((S, n, 4), dtype=torch.float32, device=device)
    E = torch.zeros(S, dtype=torch.float64, device=device)
    Ts = np.zeros(S)
    st = torch.zeros(1, dtype=torch.int32, device=device)
    k = 0
    for ti, T in enumerate(temps):
        si = W.sw_silicon(n_side, a=a, T_K=T, seed=seed * 1000 + ti)
        nl = J.NeighborList(space, n, SW_RC, 0.5, 64, device=device)
        r = torch.from_numpy(si.r).to(device)
        v = torch.from_numpy(si.v).to(device)
        f = torch.zeros_like(r)
        pe = torch.zeros(max(stride, equil), dtype=torch.float64, device=device)
        nl.build(r, st)
        J.md_energy_forces(space, pot, r, nl.plan, f, None, st)
        kT = KB * T
        step = 0
        J.md_integrate_langevin(space, pot, r, v, f, MASS_SI, dt, gamma, kT, seed * 7919 + ti, step, equil,
                                nl.plan, pe, None, True, st)
        step += equil
        for s in range(n_snap):
            J.md_integrate_langevin(space, pot, r, v, f, MASS_SI, dt, gamma, kT, seed * 7919 + ti, step, stride,
                                    nl.plan, pe, None, True, st)
            step += stride
            R[k].copy_(r)
            F[k].copy_(f)
            E[k:k + 1].copy_(pe[stride - 1:stride])
            Ts[k] = T
            k += 1
    code = J.md_status_poll(st)
    if code:
        raise J.MDError(code, "generate_sw_dataset")
    # store in a seeded random order so contiguous index ranges mix temperatures
    perm = np.random.default_rng(seed).permutation(S)
    pt = torch.as_tensor(perm, device=device)
    return Dataset(r=R[pt].contiguous(), F=F[pt].contiguous(), E=E[pt].contiguous(), T=Ts[perm], L=L, n=n)


def augment_cubic(ds: Dataset, idx_lo, idx_hi, copies, seed=0, keep=None):
    """Snapshots [idx_lo, idx_hi) under `copies` random symmetry operations
    each of the periodic cubic box (axis permutations and reflections, the
    periodic form of the random rotations and flips the paper trains its
    graph network with: that network is not rotation invariant), followed
    by the snapshots `keep` = (lo, hi) unchanged (held out).  Energies are
    unchanged, positions mapped and wrapped into [0, L), forces mapped."""
    torch = _t()
    rng = np.random.default_rng(seed)
    L = float(ds.L)
    R, F, E, T = [], [], [], []
    for s in range(idx_lo, idx_hi):
        for _ in range(copies):
            perm = torch.as_tensor(rng.permutation(3), device=ds.r.device)
            sign = torch.as_tensor(rng.choice([-1.0, 1.0], 3), dtype=torch.float32, device=ds.r.device)
            r = ds.r[s].clone()
            x = ds.r[s][:, perm] * sign
            x = torch.remainder(x, L)
            r[:, :3] = torch.where(x >= L, x - L, x)
            f = ds.F[s].clone()
            f[:, :3] = ds.F[s][:, perm] * sign
            R.append(r)
            F.append(f)
            E.append(ds.E[s:s + 1])
            T.append(ds.T[s])
    if keep is not None:
        for s in range(*keep):
            R.append(ds.r[s])
            F.append(ds.F[s])
            E.append(ds.E[s:s + 1])
            T.append(ds.T[s])
    return Dataset(r=torch.stack(R).contiguous(), F=torch.stack(F).contiguous(), E=torch.cat(E).contiguous(),
                   T=np.asarray(T), L=ds.L, n=ds.n)


def build_lists(ds: Dataset, device="cuda"):
    """One neighbor list (r_list = 3.77 + 0.3 A) per snapshot, rows local to
    the snapshot, concatenated."""
    torch = _t()
    S, n = ds.r.shape[0], ds.n
    space = J.md_space_periodic(3, [ds.L] * 3)
    plan = J.md_nbr_plan(space, n, BP_RC, SKIN, CAP)
    nbr = torch.zeros((S * n, CAP), dtype=torch.int32, device=device)
    cnt = torch.zeros(S * n, dtype=torch.int32, device=device)
    rref = torch.zeros((S * n, 4), dtype=torch.float32, device=device)
    ws = torch.empty(int(plan.ws_bytes) + 256, dtype=torch.uint8, device=device)
    wsv = ws[(-ws.data_ptr()) % 256:][: int(plan.ws_bytes)]
    st = torch.zeros(1, dtype=torch.int32, device=device)
    rflat = ds.r.reshape(S * n, 4)
    for k in range(S):
        sl = slice(k * n, (k + 1) * n)
        J.md_nbr_bind(plan, nbr[sl], cnt[sl], rref[sl], wsv)
        J.md_neighbor_list_build(space, rflat[sl], plan, st)
    code = J.md_status_poll(st)
    if code:
        raise J.MDError(code, "build_lists")
    ds.nbr, ds.cnt, ds.plan, ds.ws = nbr, cnt, plan, (ws, wsv)
    return ds


def _batch_list(ds: Dataset, s0: int, S: int):
    """md_nbr view of snapshots [s0, s0 + S) as one concatenated system."""
    nb = J.md_nbr.from_buffer_copy(ds.plan)
    n = ds.n
    nb.N = S * n
    nb.nbr = ds.nbr[s0 * n:(s0 + S) * n].data_ptr()
    nb.cnt = ds.cnt[s0 * n:(s0 + S) * n].data_ptr()
    nb.ws = ds.ws[1].data_ptr()
    return nb


def batch_list_view(ds: Dataset, s0: int, S: int):
    """md_nbr view of snapshots [s0, s0 + S) as one concatenated system
    (rows local to each snapshot) with a workspace planned for the S n
    atoms, so that md_energy_forces can run on it (the force kernels'
    reductions live there)."""
    torch = _t()
    n = ds.n
    key = ("view_ws", S)
    cache = getattr(ds, "_view_ws", None)
    if cache is None:
        cache = {}
        ds._view_ws = cache
    if key not in cache:
        space = J.md_space_periodic(3, [ds.L] * 3)
        big = J.md_nbr_plan(space, S * n, BP_RC, SKIN, CAP)
        ws = torch.zeros(int(big.ws_bytes) + 256, dtype=torch.uint8, device=ds.nbr.device)   # control words start at 0
        cache[key] = (big, ws, ws[(-ws.data_ptr()) % 256:][: int(big.ws_bytes)])
    big, _, wsv = cache[key]
    nb = J.md_nbr.from_buffer_copy(big)
    nb.nbr = ds.nbr[s0 * n:(s0 + S) * n].data_ptr()
    nb.cnt = ds.cnt[s0 * n:(s0 + S) * n].data_ptr()
    nb.ws = wsv.data_ptr()
    return nb


class Trainer:
    """Adam on the FP32 packed parameters; batches of contiguous snapshots.
    tensor_cores: the network's forward pass and training gradient on the
    tcgen05 kernels (BF16 operands, FP32 accumulation; the default), else
    the FP32 CUDA-core kernels."""

    def __init__(self, ds: Dataset, batch=16, lr=1e-3, wF=1.0, seed=0, device="cuda", params=None,
                 init_bias=True, tensor_cores=True):
        torch = _t()
        self.ds, self.B, self.lr, self.wF = ds, batch, lr, wF
        self.tc = bool(tensor_cores)
        n = ds.n
        N = batch * n
        g = torch.Generator().manual_seed(seed)
        if params is None:
            p = torch.zeros(N_PARAMS, dtype=torch.float32)
            p[0:1024] = torch.randn(1024, generator=g) / 4.0
            p[1088:5184] = torch.randn(4096, generator=g) / 8.0
            p[5248:5312] = torch.randn(64, generator=g) / 8.0
            params = p.to(device)
        self.params = params
        self.m = torch.zeros_like(params)
        self.v = torch.zeros_like(params)
        self.grad = torch.zeros_like(params)
        self.space = J.md_space_periodic(3, [ds.L] * 3)
        self.G = torch.zeros((N, 16), dtype=torch.float32, device=device)
        self.Ei = torch.zeros(N, dtype=torch.float32, device=device)
        self.dEdG = torch.zeros((N, 16), dtype=torch.float32, device=device)
        self.Fp = torch.zeros((N, 4), dtype=torch.float32, device=device)
        self.cE = torch.zeros(N, dtype=torch.float32, device=device)
        self.dF = torch.zeros((N, 4), dtype=torch.float32, device=device)
        self.V = torch.zeros((N, 16), dtype=torch.float32, device=device)
        self.loss = torch.zeros(2 * batch, dtype=torch.float64, device=device)
        self.scratch = torch.empty(J.md_bp_train_scratch_size(N), dtype=torch.uint8, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        self.step_count = 0
        self.norm = self._normalisation(device)
        if init_bias:
            # output bias: mean energy per atom of the data (kernel statistics)
            stats = torch.zeros(2, dtype=torch.float32, device=device)
            e32 = (ds.E / ds.n).float().contiguous()
            J.md_column_stats(e32, ds.E.shape[0], 1, stats)
            self.params[5312:5313].copy_(stats[0:1])

    def _normalisation(self, device):
        """Descriptor mean / std over (up to) 64 snapshots."""
        torch = _t()
        ds = self.ds
        S = min(64, ds.r.shape[0])
        N = S * ds.n
        G = torch.zeros((N, 16), dtype=torch.float32, device=device)
        nb = _batch_list(ds, 0, S)
        J.md_bp_descriptors(self.space, ds.r[:S].reshape(N, 4), nb, ds.n, G, self.status)
        norm = torch.zeros(32, dtype=torch.float32, device=device)
        J.md_column_stats(G, N, 16, norm)
        norm[16:] += 1e-3   # floor the spread of nearly constant descriptors
        return norm

    def forward(self, s0, S):
        ds, n = self.ds, self.ds.n
        N = S * n
        nb = _batch_list(ds, s0, S)
        r = ds.r[s0:s0 + S].reshape(N, 4)
        J.md_bp_descriptors(self.space, r, nb, n, self.G[:N], self.status)
        if self.tc:
            J.md_bp_mlp_infer_tc(self.params, self.norm, self.G[:N], N, self.Ei[:N], self.dEdG[:N], self.status)
        else:
            J.md_bp_mlp_infer(self.params, self.norm, self.G[:N], N, self.Ei[:N], self.dEdG[:N])
        J.md_bp_forces(self.space, r, nb, n, self.dEdG[:N], self.Ei[:N], self.Fp[:N], None, self.status)
        J.md_bp_loss_prep(self.Ei[:N], self.Fp[:N], ds.F[s0:s0 + S].reshape(N, 4), ds.E[s0:s0 + S], S, n, self.wF,
                          self.cE[:N], self.dF[:N], self.loss[:2 * S])
        return nb, r, N

    def step(self, s0):
        n = self.ds.n
        nb, r, N = self.forward(s0, self.B)
        J.md_bp_jvp(self.space, r, nb, n, self.dF[:N], self.V[:N], self.status)
        if self.tc:
            J.md_bp_mlp_train_tc(self.params, self.norm, self.G[:N], self.V[:N], self.cE[:N], 1.0, N, self.scratch,
                                 self.grad, self.status)
        else:
            J.md_bp_mlp_train(self.params, self.norm, self.G[:N], self.V[:N], self.cE[:N], 1.0, N, self.scratch,
                              self.grad)
        self.step_count += 1
        J.md_adam_step(self.params, self.grad, self.m, self.v, N_PARAMS, self.lr, 0.9, 0.999, 1e-8,
                       self.step_count)

    def train(self, idx_lo, idx_hi, epochs, seed=0, lr_end=None):
        """Epochs over contiguous batches of snapshots [idx_lo, idx_hi),
        batch order shuffled each epoch; cosine learning-rate decay."""
        rng = np.random.default_rng(seed)
        starts = np.arange(idx_lo, idx_hi - self.B + 1, self.B)
        total = epochs * len(starts)
        lr0 = self.lr
        k = 0
        for _ in range(epochs):
            for s0 in rng.permutation(starts):
                if lr_end is not None:
                    self.lr = lr_end + 0.5 * (lr0 - lr_end) * (1 + math.cos(math.pi * k / max(1, total)))
                self.step(int(s0))
                k += 1
        self.lr = lr0

    def evaluate(self, idx_lo, idx_hi):
        """(energy RMSE per atom [eV/atom], force RMSE [eV/A]) over snapshots
        [idx_lo, idx_hi), from the loss kernel's per-snapshot terms."""
        e2 = f2 = 0.0
        cnt = 0
        wF = self.wF
        self.wF = 1.0
        for s0 in range(idx_lo, idx_hi, self.B):
            S = min(self.B, idx_hi - s0)
            self.forward(s0, S)
            l = self.loss[:2 * S].cpu().numpy()
            e2 += l[0::2].sum() * S
            f2 += l[1::2].sum() * S
            cnt += S
        self.wF = wF
        code = J.md_status_poll(self.status)
        if code:
            raise J.MDError(code, "evaluate")
        return math.sqrt(e2 / cnt), math.sqrt(f2 / cnt)


class GNNTrainer(Trainer):
    """The graph-network potential (Sec. 4.1: the GNN fitted to energies and
    forces with Adam) on the same data: forward by md_energy_forces on the
    concatenated batch (rows local to each snapshot), loss terms by the
    loss kernel, the parameter gradient by md_gnn_train_grad (forward with
    the force-error tangent, reverse through values and tangents), Adam.
    Epochs, learning-rate decay and evaluation are the BP trainer's."""

    def __init__(self, ds: Dataset, batch=16, lr=1e-3, wF=1.0, seed=0, device="cuda", params=None, H=64, T=2,
                 init_bias=True):
        torch = _t()
        import workloads as W
        self.ds, self.B, self.lr, self.wF = ds, batch, lr, wF
        self.H, self.T = H, T
        n = ds.n
        N = batch * n
        if params is None:
            params = torch.from_numpy(W.gnn_params(H, T, seed=seed, out_scale=0.1)).to(device)
        self.params = params
        self.n_params = J.md_gnn_param_count(H, T)
        self.m = torch.zeros_like(params)
        self.v = torch.zeros_like(params)
        self.grad = torch.zeros_like(params)
        self.space = J.md_space_periodic(3, [ds.L] * 3)
        self.model = J.GNNModel(params, N, CAP, H, T, BP_RC, device=device, sys_n=n)
        self.Ei = torch.zeros(N, dtype=torch.float32, device=device)
        self.Fp = torch.zeros((N, 4), dtype=torch.float32, device=device)
        self.cE = torch.zeros(N, dtype=torch.float32, device=device)
        self.dF = torch.zeros((N, 4), dtype=torch.float32, device=device)
        self.loss = torch.zeros(2 * batch, dtype=torch.float64, device=device)
        nbytes = J.md_gnn_train_scratch_bytes(N, CAP, H, T)
        self._scratch = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        self.scratch = self._scratch[(-self._scratch.data_ptr()) % 256:][:nbytes]
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        self.step_count = 0
        if init_bias:
            # read-out bias c (the last parameter): mean energy per atom of the data
            stats = torch.zeros(2, dtype=torch.float32, device=device)
            e32 = (ds.E / ds.n).float().contiguous()
            J.md_column_stats(e32, ds.E.shape[0], 1, stats)
            self.params[self.n_params - 1:self.n_params].copy_(stats[0:1])

    def forward(self, s0, S):
        ds, n = self.ds, self.ds.n
        N = S * n
        nb = batch_list_view(ds, s0, S)
        r = ds.r[s0:s0 + S].reshape(N, 4)
        J.md_energy_forces(self.space, self.model.pot, r, nb, self.Fp[:N], None, self.status)
        self.Ei[:N].copy_(self.Fp[:N, 3])
        J.md_bp_loss_prep(self.Ei[:N], self.Fp[:N], ds.F[s0:s0 + S].reshape(N, 4), ds.E[s0:s0 + S], S, n, self.wF,
                          self.cE[:N], self.dF[:N], self.loss[:2 * S])
        return nb, r, N

    def step(self, s0):
        nb, r, N = self.forward(s0, self.B)
        J.md_gnn_train_grad(self.space, r, nb, self.model, self.cE[:N], self.dF[:N], self.scratch, self.grad,
                            self.status)
        self.step_count += 1
        J.md_adam_step(self.params, self.grad, self.m, self.v, self.n_params, self.lr, 0.9, 0.999, 1e-8,
                       self.step_count)


def force_rmse_sw2body(ds: Dataset, idx_lo, idx_hi, device="cuda"):
    """RMSE of the SW two-body forces alone (lambda = 0) against full SW,
    through the loss kernel (force term only)."""
    torch = _t()
    p = list(SW_SI)
    p[3] = 0.0
    pot = J.sw_pot(p)
    n = ds.n
    space = J.md_space_periodic(3, [ds.L] * 3)
    nl = J.NeighborList(space, n, SW_RC, 0.3, 64, device=device)
    st = torch.zeros(1, dtype=torch.int32, device=device)
    f = torch.zeros((n, 4), dtype=torch.float32, device=device)
    zeros = torch.zeros(n, dtype=torch.float32, device=device)
    cE = torch.zeros(n, dtype=torch.float32, device=device)
    dF = torch.zeros((n, 4), dtype=torch.float32, device=device)
    loss = torch.zeros(2, dtype=torch.float64, device=device)
    f2 = 0.0
    for k in range(idx_lo, idx_hi):
        nl.build(ds.r[k], st)
        J.md_energy_forces(space, pot, ds.r[k], nl.plan, f, None, st)
        J.md_bp_loss_prep(zeros, f, ds.F[k], ds.E[k:k + 1], 1, n, 1.0, cE, dF, loss)
        f2 += loss[1].item()
    return math.sqrt(f2 / (idx_hi - idx_lo))


def deploy_compare(params, norm, n_side=20, T=1000.0, steps=200, warmup=20, dt=1.0, seed=0, device="cuda"):
    """NVE of an n_side^3-cell diamond (8 n_side^3 atoms) at temperature T
    with plain SW and with the learned potential (tensor-core network and
    FP32 network).  Returns particle-steps/s of each and the learned force
    RMSE against SW on the starting and final configurations."""
    torch = _t()
    import workloads as W
    si = W.sw_silicon(n_side, T_K=T, seed=seed)
    N, L = si.N, si.L
    space = J.md_space_periodic(3, [L] * 3)
    st = torch.zeros(1, dtype=torch.int32, device=device)
    out = {"N": N, "T_K": T, "steps": steps, "dt_fs": dt}
    model = J.BPModel(params, norm, N, device=device)
    sw = J.sw_pot(SW_SI, N=N, device=device)
    n = N
    zeros = torch.zeros(n, dtype=torch.float32, device=device)
    cE = torch.zeros(n, dtype=torch.float32, device=device)
    dF = torch.zeros((n, 4), dtype=torch.float32, device=device)
    loss = torch.zeros(2, dtype=torch.float64, device=device)
    Edummy = torch.zeros(1, dtype=torch.float64, device=device)

    def rmse(r, nl):
        fs = torch.zeros((n, 4), dtype=torch.float32, device=device)
        fb = torch.zeros((n, 4), dtype=torch.float32, device=device)
        J.md_energy_forces(space, sw, r, nl.plan, fs, None, st)
        J.md_energy_forces(space, model.pot, r, nl.plan, fb, None, st)
        J.md_bp_loss_prep(zeros, fb, fs, Edummy, 1, n, 1.0, cE, dF, loss)
        return math.sqrt(loss[1].item())

    for name, pot, tc in (("sw", sw, False), ("learned_tc", model.pot, True), ("learned_fp32", model.pot, False)):
        J.md_bp_set_tensor_cores(tc)
        nl = J.NeighborList(space, N, SW_RC, 0.3, 64, device=device)
        r = torch.from_numpy(si.r).to(device)
        v = torch.from_numpy(si.v).to(device)
        f = torch.zeros_like(r)
        nl.build(r, st)
        J.md_energy_forces(space, pot, r, nl.plan, f, None, st)
        J.md_integrate_nve(space, pot, r, v, f, MASS_SI, dt, warmup, nl.plan, None, None, True, st)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        J.md_integrate_nve(space, pot, r, v, f, MASS_SI, dt, steps, nl.plan, None, None, True, st)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        out[name + "_particle_steps_per_s"] = N * steps / (ms * 1e-3)
        if name == "learned_tc":
            out["force_rmse_vs_sw_final_eV_per_A"] = rmse(r, nl)
    J.md_bp_set_tensor_cores(False)
    r0 = torch.from_numpy(si.r).to(device)
    nl = J.NeighborList(space, N, SW_RC, 0.3, 64, device=device)
    nl.build(r0, st)
    out["force_rmse_vs_sw_start_eV_per_A"] = rmse(r0, nl)
    code = J.md_status_poll(st)
    if code:
        raise J.MDError(code, "deploy_compare")
    return out


def gnn_deploy_compare(params, H=64, T=2, n_side=20, temp=1000.0, steps=200, warmup=20, dt=1.0, seed=0,
                       device="cuda"):
    """NVE of the n_side^3-cell diamond at temperature temp with the trained
    graph network, FP32 kernels and tcgen05 kernels (the latter hold the
    weights rounded to BF16).  Returns particle-steps/s of each and the
    force RMSE against plain SW on the final configurations."""
    torch = _t()
    import workloads as W
    si = W.sw_silicon(n_side, T_K=temp, seed=seed)
    N, L = si.N, si.L
    space = J.md_space_periodic(3, [L] * 3)
    st = torch.zeros(1, dtype=torch.int32, device=device)
    model = J.GNNModel(params, N, 64, H, T, BP_RC, device=device)
    sw = J.sw_pot(SW_SI)
    cE = torch.zeros(N, dtype=torch.float32, device=device)
    dF = torch.zeros((N, 4), dtype=torch.float32, device=device)
    loss = torch.zeros(2, dtype=torch.float64, device=device)
    zeros = torch.zeros(N, dtype=torch.float32, device=device)
    Edummy = torch.zeros(1, dtype=torch.float64, device=device)
    out = {"N": N, "T_K": temp, "steps": steps, "dt_fs": dt, "H": H, "T": T}
    for name, tc in (("gnn_fp32", False), ("gnn_tc", True)):
        J.md_gnn_set_tensor_cores(tc)
        nl = J.NeighborList(space, N, BP_RC, 0.3, 64, device=device)
        r = torch.from_numpy(si.r).to(device)
        v = torch.from_numpy(si.v).to(device)
        f = torch.zeros_like(r)
        nl.build(r, st)
        J.md_energy_forces(space, model.pot, r, nl.plan, f, None, st)
        J.md_integrate_nve(space, model.pot, r, v, f, MASS_SI, dt, warmup, nl.plan, None, None, True, st)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        J.md_integrate_nve(space, model.pot, r, v, f, MASS_SI, dt, steps, nl.plan, None, None, True, st)
        e1.record()
        e1.synchronize()
        out[name + "_particle_steps_per_s"] = N * steps / (e0.elapsed_time(e1) * 1e-3)
        fs = torch.zeros((N, 4), dtype=torch.float32, device=device)
        fg = torch.zeros((N, 4), dtype=torch.float32, device=device)
        J.md_energy_forces(space, sw, r, nl.plan, fs, None, st)
        J.md_energy_forces(space, model.pot, r, nl.plan, fg, None, st)
        J.md_bp_loss_prep(zeros, fg, fs, Edummy, 1, N, 1.0, cE, dF, loss)
        out[name + "_force_rmse_vs_sw_final_eV_per_A"] = math.sqrt(loss[1].item())
    J.md_gnn_set_tensor_cores(False)
    code = J.md_status_poll(st)
    if code:
        raise J.MDError(code, "gnn_deploy_compare")
    return out
