#!/usr/bin/env python
"""Benchmark: Lennard-Jones NVE particle-steps/s on one B300 (per rank).

A bench step is one whole LJ NVE job of the N = 256,000 workload (FCC
4*40^3 start at density 0.84, T* = 1, r_c = 2.5 shifted, skin 0.3,
dt = 0.005): neighbor-list build, initial forces and 1,000 velocity-Verlet
steps with device-side rebuild decisions, all inside libjmd (one CUDA graph
with a device-controlled WHILE loop).  `value` = particle-steps per second
over K timed bench steps (inputs resident in HBM; L2 flushed between bench
steps), summed over ranks (weak scaling: each rank runs its own seeded
replica, no data-path collective).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl jmd|reference]

`--impl reference` times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (LJ N=256k); learned vs plain SW at stated force RMSE"
UNIT = "particle-steps/s"
# CUDA graphs for the MD loops of the sections (off with --no-graph, for profiling)
USE_GRAPH = True


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="jmd", choices=["jmd", "reference"])
    ap.add_argument("--workload", default="lj256k", choices=["lj256k", "lj4096"])
    ap.add_argument("--md-steps", type=int, default=None, help="MD steps per bench step (default: the workload's)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--tpp", type=int, default=0)
    ap.add_argument("--pair-opt", type=int, default=-1, help="pair-kernel variant (md_set_pair_options)")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch every kernel from the host, in every section (profiling)")
    ap.add_argument("--no-fp32-peak", action="store_true", help="skip the FP32 FMA probe")
    ap.add_argument("--sort", type=int, default=1,
                    help="1: Z-order sort of the particles at the start of each job (md_sort_particles)")
    ap.add_argument("--nve-fusion", type=int, default=1, help="1: kick-drift fused into the force kernel (md_set_nve_fusion)")
    ap.add_argument("--tiles", type=int, default=0,
                    help="1: the tile engine (MD_NBR_TILES) runs the NVE loop; 0: the int32-row engine")
    ap.add_argument("--tile-tpp", type=int, default=0, help="lanes per particle of the tile step kernel (1, 4 or 8; 0 = by tile size)")
    ap.add_argument("--local-rows", type=int, default=0,
                    help="1: cell-centred forces over 16-bit local rows (MD_NBR_LOCAL_ROWS); 0: int32 rows")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-vs-plain-SW section")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-replica section")
    ap.add_argument("--no-fire", action="store_true", help="skip the FIRE minimisation section")
    ap.add_argument("--no-order", action="store_true", help="skip the particle-order sensitivity section")
    ap.add_argument("--no-table1", action="store_true", help="skip the paper's Table 1 configurations")
    ap.add_argument("--no-packing", action="store_true",
                    help="skip the packing section (Fig. 3 ensemble, gradient descent and its adjoint)")
    ap.add_argument("--no-nhc", action="store_true", help="skip the Nose-Hoover NVT section")
    ap.add_argument("--no-flock", action="store_true", help="skip the flocking section")
    ap.add_argument("--no-gnn", action="store_true", help="skip the graph-network potential section")
    ap.add_argument("--no-alu", action="store_true", help="skip the ALU rooflines of k_sw and the rebuild chain")
    ap.add_argument("--no-tiles-job", action="store_true", help="skip the bench job on the tile engine")
    ap.add_argument("--probe", default=None, choices=["learned-kernels", "train-step", "batch-steps"],
                    help="print the per-kernel timings of the learned potential's deployment (64,000 Si atoms), "
                         "of one BP training step (8 snapshots of 512 atoms), or the 512-replica batch's NVE "
                         "steps as host launches, and exit")
    return ap.parse_args()


def workload(name, seed):
    import workloads as W
    return W.lj_large(seed) if name == "lj256k" else W.lj_small(seed)


class ClockSampler:
    """nvidia-smi clock / throttle samples taken during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for k, n in enumerate(names):
                if p[5 + k].lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


ORACLE_SERIES = {}


def oracle_sample(name, md_steps, seed=0):
    """Time the FP64 oracle on `md_steps` NVE steps of the workload (all host
    threads).  Returns (particle-steps/s, threads, seconds); the energy
    series is kept for the drift comparison."""
    import oracle as O
    c = workload(name, seed)
    t0 = time.perf_counter()
    _, _, PEo, KEo = O.nve(c.r, c.v, c.L, "lj", dt=c.dt, nsteps=md_steps)
    dt = time.perf_counter() - t0
    ORACLE_SERIES[(name, seed, md_steps)] = PEo + KEo
    return c.N * md_steps / dt, O.num_threads(), dt


def run_reference(args, rank):
    if rank != 0:
        return
    md = 5 if args.workload == "lj256k" else 50
    times = []
    N = workload(args.workload, 0).N
    thr = 1
    for k in range(args.warmup + args.steps):
        _, thr, dt = oracle_sample(args.workload, md)
        if k >= args.warmup:
            times.append(dt)
    tot = sum(times)
    val = N * md * args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "lj_fcc40_N256000" if N == 256000 else "lj_sc16_N4096", "N": N,
                   "md_steps_per_step": md},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": thr, "kind": "oracle",
                         "sample": f"{md} FP64 velocity-Verlet steps of the N={N} LJ workload per step"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def learned_section():
    """Train the BP network (and the graph network) on GPU-generated SW
    data, then run NVE at N = 64,000 atoms with plain SW and with the
    learned potentials."""
    import torch
    import paper_1912_04232_b300.learned as LP
    temps = np.linspace(500.0, 3000.0, 8)
    t0 = time.perf_counter()
    ds = LP.generate_sw_dataset(temps, n_snap=30, stride=20, equil=300, seed=1)
    LP.build_lists(ds)
    S = ds.r.shape[0]
    ntr = int(0.8 * S)
    t_data = time.perf_counter() - t0
    tr = LP.Trainer(ds, batch=8, lr=3e-3, wF=1.0, seed=0)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    tr.train(0, ntr, epochs=40, seed=0, lr_end=1e-4)
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t1
    e_rmse, f_rmse = tr.evaluate(ntr, S)
    two = LP.force_rmse_sw2body(ds, ntr, S)
    t_train = time.perf_counter() - t0
    # one training step (forward, loss, descriptor JVP, network gradient,
    # Adam) on each network path, from the same start, CUDA events
    step_ms, epoch_ms = {}, {}
    for name, tc in (("tcgen05_bf16", True), ("fp32", False)):
        tt = LP.Trainer(ds, batch=8, lr=3e-3, wF=1.0, seed=0, tensor_cores=tc)
        for _ in range(3):
            tt.step(0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(20):
            tt.step(8 * (k % max(1, ntr // 8)))
        e1.record()
        torch.cuda.synchronize()
        step_ms[name] = e0.elapsed_time(e1) / 20
        e0.record()
        tt.train(0, ntr, epochs=1, seed=1)
        e1.record()
        torch.cuda.synchronize()
        epoch_ms[name] = e0.elapsed_time(e1)
    dep = LP.deploy_compare(tr.params, tr.norm, n_side=20, T=1000.0, steps=200, warmup=20)
    kernels = learned_kernels(tr.params, tr.norm)
    # the graph network on the same data (trained by md_gnn_train_grad + Adam),
    # the training snapshots under 8 symmetry operations of the cubic box each
    t1 = time.perf_counter()
    da = LP.augment_cubic(ds, 0, ntr, 8, seed=2, keep=(ntr, S))
    LP.build_lists(da)
    na = 8 * ntr
    gt = LP.GNNTrainer(da, batch=8, lr=3e-3, wF=1.0, seed=0, H=64, T=2)
    g_untrained = gt.evaluate(na, na + S - ntr)
    gt.train(0, na, epochs=50, seed=0, lr_end=1e-4)
    g_e, g_f = gt.evaluate(na, na + S - ntr)
    t_gnn = time.perf_counter() - t1
    gdep = LP.gnn_deploy_compare(gt.params, H=64, T=2, n_side=20, temp=1000.0, steps=100, warmup=10)
    return {
        "sw_particle_steps_per_s": dep["sw_particle_steps_per_s"],
        "learned_particle_steps_per_s": dep["learned_tc_particle_steps_per_s"],
        "learned_fp32_particle_steps_per_s": dep["learned_fp32_particle_steps_per_s"],
        "learned_over_sw": dep["learned_tc_particle_steps_per_s"] / dep["sw_particle_steps_per_s"],
        "force_rmse_eV_per_A_heldout": f_rmse, "energy_rmse_eV_per_atom_heldout": e_rmse,
        "force_rmse_sw_two_body_only": two, "force_rmse_vs_sw_at_deploy": dep["force_rmse_vs_sw_final_eV_per_A"],
        "deploy": {"N": dep["N"], "T_K": 1000.0, "steps": 200, "dt_fs": 1.0, "network": "tcgen05 BF16"},
        "kernels_64000": {"us": kernels["us"], "roofline": kernels["roofline"],
                          "pairs_per_atom": kernels["pairs_per_atom"],
                          "triplets_per_atom": kernels["triplets_per_atom"]},
        "train": {"snapshots": int(S), "heldout": int(S - ntr), "epochs": 40, "seconds_incl_data": t_train,
                  "seconds_data": t_data, "seconds_fit": t_fit, "network": "tcgen05 BF16 (md_bp_mlp_train_tc)",
                  "step_ms": step_ms, "step_speedup_tc_over_fp32": step_ms["fp32"] / step_ms["tcgen05_bf16"],
                  "epoch_ms": epoch_ms, "steps_per_epoch": ntr // 8,
                  "atoms_per_step": 8 * int(ds.n)},
        "gnn": {"force_rmse_eV_per_A_heldout": g_f, "energy_rmse_eV_per_atom_heldout": g_e,
                "force_rmse_untrained": g_untrained[1], "epochs": 50, "augmentation": "8 cubic symmetry copies",
                "seconds": t_gnn, "H": 64, "T": 2,
                "deploy": gdep},
    }


def batch_setup(specs, dev, st):
    """Initial states of replicas (soft-sphere replicas relaxed by 50
    gradient-descent steps, then wrapped) and their md_replica_desc; the
    states concatenated on the GPU."""
    import torch
    import paper_1912_04232_b300 as P
    import workloads as W
    states = []
    for sp in specs:
        r, v = W.replica_initial(sp)
        if sp.kind == "soft":
            s = P.md_space_periodic(3, [sp.L] * 3)
            nl = P.NeighborList(s, sp.N, 1.4, 0.3, 128)
            rd = torch.from_numpy(r).to(dev)
            f = torch.zeros_like(rd)
            nl.build(rd, st)
            P.md_minimize(s, P.soft_pot(), 0, 0.05, 50, rd, f, nl.plan, None, st)
            x = rd.cpu().numpy()
            x[:, :3] = np.mod(x[:, :3], np.float32(sp.L)).astype(np.float32)
            x[:, :3][x[:, :3] >= np.float32(sp.L)] = 0.0
            r = x
        states.append((r, v))

    def desc(sp):
        d = P.md_replica_desc()
        d.N, d.L = sp.N, sp.L
        if sp.kind == "lj":
            pot = P.lj_pot()
            d.kind, d.eps, d.sigma, d.r_cut, d.e_shift = P.MD_LJ, pot.eps, pot.sigma, pot.r_cut, pot.e_shift
        else:
            d.kind, d.eps, d.alpha, d.r_cut = P.MD_SOFT_SPHERE, 1.0, 2.0, 1.4
        d.skin, d.dt, d.mass = 0.3, sp.dt, 1.0
        return d

    descs = [desc(sp) for sp in specs]
    r0 = torch.from_numpy(np.concatenate([s[0] for s in states])).to(dev)
    v0 = torch.from_numpy(np.concatenate([s[1] for s in states])).to(dev)
    return states, descs, r0, v0


def batched_section(steps=500, rank=0, world=1, dist=None, device=None):
    """512 LJ / soft-sphere replicas (N log-uniform in [64, 8192]) for
    `steps` NVE steps in one graph launch, against one launch per replica.
    With several ranks each runs its share of the replicas
    (`replicas.split_replicas`); the rates count every rank's particles over
    the slowest rank's time, the tuning figures are this rank's."""
    import torch
    import paper_1912_04232_b300 as P
    import workloads as W
    from paper_1912_04232_b300.replicas import split_replicas
    dev = device if device is not None else torch.device("cuda")
    specs_all = W.replica_plan(R=512, n_max=8192, seed=0)
    specs = [specs_all[i] for i in split_replicas([sp.N for sp in specs_all], world)[rank]]
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    states, descs, r0, v0 = batch_setup(specs, dev, st)
    import tempfile
    import paper_1912_04232_b300.batch_tune as BT
    r, v, f = r0.clone(), v0.clone(), torch.zeros_like(r0)

    def run_batch(b):
        r.copy_(r0)
        v.copy_(v0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        P.md_batch_build(b.plan, r, st)
        P.md_batch_forces(b.plan, r, f, st)
        P.md_batch_run_nve(b.plan, r, v, f, steps, None, None, True, st)
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1)

    def measure(b):
        run_batch(b)
        return min(run_batch(b) for _ in range(3))

    # default plan (smallest cells, 4 threads per particle), then one
    # threads-per-particle value for all (md_batch_autotune), then the
    # per-size-class cell multipliers and threads per particle (batch_tune)
    b = P.Batch(descs, cap=128)
    ms_default = measure(b)
    scratch = torch.empty((2 * b.plan.N, 4), dtype=torch.float32, device=dev)
    tpp = P.md_batch_autotune(b.plan, r, v, f, scratch, 20,
                              os.path.join(tempfile.gettempdir(), f"jmd_batch_tune_r{rank}.json"))
    ms_global = measure(b)
    del b
    tuned = BT.tune(descs, r0, v0, probe=20,
                    cache_path=os.path.join(tempfile.gettempdir(), f"jmd_batch_classes_r{rank}.json"))
    b = P.Batch(BT.with_mults(descs, tuned["cell_mult"]), cap=128)
    P.md_batch_set_class_tpp(b.plan, BT.tpp_per_replica(descs, tuned["tpp"]))
    ms_b = measure(b)
    # one launch (graph) per replica, same tuning
    P.md_set_pair_tpp(tpp)
    singles = []
    for sp, (rr, vv) in zip(specs, states):
        s = P.md_space_periodic(3, [sp.L] * 3)
        nl = P.NeighborList(s, sp.N, 2.5 if sp.kind == "lj" else 1.4, 0.3, 128)
        rd, vd = torch.from_numpy(rr).to(dev), torch.from_numpy(vv).to(dev)
        singles.append((s, nl, rd, vd, torch.zeros_like(rd), rd.clone(), vd.clone(), sp))

    def run_singles():
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for s, nl, rd, vd, f1, ri, vi, sp in singles:
            rd.copy_(ri)
            vd.copy_(vi)
            pot = P.lj_pot() if sp.kind == "lj" else P.soft_pot()
            nl.build(rd, st)
            P.md_energy_forces(s, pot, rd, nl.plan, f1, None, st)
            P.md_integrate_nve(s, pot, rd, vd, f1, 1.0, sp.dt, steps, nl.plan, None, None, True, st)
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1)

    run_singles()
    ms_s = run_singles()
    P.md_set_pair_tpp(4)
    code = P.md_status_poll(st)
    Ntot = int(b.plan.N)
    # ALU roofline of the one-launch step: every row entry is evaluated with
    # the cutoff as a select (LJ/soft sphere with the nearest-image formula:
    # 35 FLOP, FMA = 2), plus 24 FLOP of integration per particle-step;
    # rebuild work is not counted, so the fraction is a lower bound
    mean_cnt = float(b.cnt.float().clamp(max=128).mean().item())
    flop_ps = 35.0 * mean_cnt + 24.0
    pk, src = fp32_peak()
    ach = flop_ps * Ntot * steps / (ms_b * 1e-3) / 1e12
    if dist is not None:   # the whole job: every rank's particles, the slowest rank's time
        t = torch.tensor([float(Ntot)], dtype=torch.float64, device=dev)
        dist.all_reduce(t)
        Ntot = int(t.item())
        ms_b = max_over_ranks(ms_b, dist, dev)
        ms_s = max_over_ranks(ms_s, dist, dev)
        ms_default = max_over_ranks(ms_default, dist, dev)
        ms_global = max_over_ranks(ms_global, dist, dev)
    return {"replicas": len(specs_all), "ranks": world, "N_total": Ntot, "steps": steps, "tpp_autotuned": tpp,
            "one_launch_particle_steps_per_s": Ntot * steps / (ms_b * 1e-3),
            "per_replica_launches_particle_steps_per_s": Ntot * steps / (ms_s * 1e-3),
            "speedup": ms_s / ms_b, "status": code,
            "tuning": {"default_particle_steps_per_s": Ntot * steps / (ms_default * 1e-3),
                       "global_tpp_particle_steps_per_s": Ntot * steps / (ms_global * 1e-3),
                       "class_tuned_particle_steps_per_s": Ntot * steps / (ms_b * 1e-3),
                       "classes_N": ["N < 512", "512 <= N < 2048", "N >= 2048"],
                       "replicas_per_class": tuned["classes"], "cell_mult": tuned["cell_mult"],
                       "tpp": tuned["tpp"], "tuner_cached": tuned["cached"],
                       "tuned_over_default": ms_default / ms_b},
            "roofline": {"bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                         "flop_per_particle_step": flop_ps, "mean_row_entries": mean_cnt,
                         "peak_source": src}}


def alu_rooflines_section():
    """The ALU-bound kernels against the measured FP32 FMA peak: algorithmic
    FLOPs (the formulas' operations, FMA = 2, divide / sqrt / exp / pow = 1)
    counted from the configuration, over the CUDA-event time of the launch.
      k_sw (SW silicon, 64,000 atoms at 1000 K): 42 FLOP per ordered pair
        inside a*sigma (distance 9, phi2 and phi2' 24, accumulation 9), 102
        per triplet centred on the atom (the triplet 95, accumulation 7) and
        107 per triplet in which the atom is a leg (second leg's distance 9,
        the triplet 95, accumulation 3); with m_i partners of atom i inside
        a*sigma: sum m_i pairs, sum m_i (m_i - 1) / 2 centred and
        sum m_i (m_i - 1) leg triplets.
      rebuild chain (LJ, 256,000 particles, the lattice start): 9 FLOP per
        candidate test (difference 3, square and sum 5, compare 1), candidates
        = sum over cells of (own particles x particles of the 27 stencil
        cells); the time is the whole chain (binning, scan, scatter, cell
        sort, build), of which k_build_cells is about 86%."""
    import torch
    import paper_1912_04232_b300 as P
    import paper_1912_04232_b300.learned as LP
    import workloads as W
    dev = torch.device("cuda")
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    pk, src = fp32_peak()

    def timed(fn, reps=20):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e-3)
        return statistics.median(ts)

    out = {"peak_tflops": pk, "peak_source": src}
    # SW forces (k_sw_lists + k_sw, the deployed form) on the thermal
    # configuration after 200 NVE steps from the 1000 K lattice start
    si, s, r = sw_evolved_64000()
    cap = 64
    nl = P.NeighborList(s, si.N, LP.SW_RC, 0.3, cap)
    f = torch.zeros_like(r)
    nl.build(r, st)
    pot = P.sw_pot(LP.SW_SI, N=si.N)
    t = timed(lambda: P.md_energy_forces(s, pot, r, nl.plan, f, None, st))
    n = nl.cnt.clamp(max=cap).long()
    rows = nl.nbr.long().clamp(max=si.N - 1)
    d = r[rows, :3] - r[:, None, :3]
    d -= float(si.L) * torch.round(d / float(si.L))
    inside = (torch.arange(cap, device=dev)[None, :] < n[:, None]) & ((d * d).sum(-1) < LP.SW_RC ** 2)
    m = inside.sum(1).double()
    pairs, cent, legs = float(m.sum()), float((m * (m - 1) / 2).sum()), float((m * (m - 1)).sum())
    fl = 42.0 * pairs + 102.0 * cent + 107.0 * legs
    out["k_sw"] = {"N": si.N, "kernels": "k_sw_lists + k_sw", "configuration": "after 200 NVE steps from 1000 K",
                   "us": t * 1e6, "flops": fl, "pairs_per_atom": pairs / si.N,
                   "triplets_per_atom": (cent + legs) / si.N,
                   "roofline": {"bound": "alu", "achieved": fl / t / 1e12, "peak": pk, "unit": "TFLOP/s",
                                "frac": fl / t / 1e12 / pk}}
    # rebuild chain of the LJ list
    c = W.lj_large(seed=0)
    s = P.md_space_periodic(3, [c.L] * 3)
    nl = P.NeighborList(s, c.N, c.r_cut, c.skin, 128)
    r = torch.from_numpy(c.r).to(dev)
    t = timed(lambda: nl.build(r, st))
    nc = int(nl.plan.ncell[0])
    idx = np.clip(np.floor(np.mod(c.r[:, :3].astype(np.float64), c.L) / (c.L / nc)).astype(np.int64), 0, nc - 1)
    cnt = np.bincount((idx[:, 2] * nc + idx[:, 1]) * nc + idx[:, 0], minlength=nc ** 3).reshape(nc, nc, nc)
    sten = np.zeros_like(cnt)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                sten += np.roll(cnt, (dz, dy, dx), axis=(0, 1, 2))
    cand = float((cnt * sten).sum())
    fl = 9.0 * cand
    out["rebuild_chain_lj256k"] = {"N": c.N, "us": t * 1e6, "cells_per_axis": nc, "candidates_per_particle": cand / c.N,
                                   "roofline": {"bound": "alu", "achieved": fl / t / 1e12, "peak": pk,
                                                "unit": "TFLOP/s", "frac": fl / t / 1e12 / pk}}
    out["status"] = P.md_status_poll(st)
    return out


def table1_section(steps=10000):
    """The paper's Table 1 benchmark on this GPU: LJ particles, 10,000 NVE
    steps, cutoff 3 sigma, halo (skin) 0.5 sigma, the list rebuilt when a
    particle moves more than half the halo.  N = 64,000 at density 0.84 (the
    paper's large GPU system; simple-cubic 40^3 start, T = 1, dt = 0.005) and
    N = 216 (6^3).  The paper states no density; at 0.84 a 216-particle box
    (6.36 sigma) is smaller than twice the list radius (7 sigma) that minimum
    images need, so N = 216 runs at density 0.6 (box 7.11 sigma).  One graph
    launch per run, particles Z-order sorted first; ms per step is the run
    time / steps."""
    import torch
    import paper_1912_04232_b300 as P
    import workloads as W
    dev = torch.device("cuda")
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    out = {"steps": steps, "r_cut": 3.0, "halo": 0.5,
           "paper_k80_ms_per_step": {"N216": 0.09, "N64000": 10.5}}
    for name, n_side, rho in (("N64000", 40, 0.84), ("N216", 6, 0.6)):
        c = W.lj_fluid("sc", n_side, rho=rho, seed=0)
        s = P.md_space_periodic(3, [c.L] * 3)
        pot = P.lj_pot(1.0, 1.0, 3.0, True)
        nl = P.NeighborList(s, c.N, 3.0, 0.5, 256)
        r0, v0 = torch.from_numpy(c.r).to(dev), torch.from_numpy(c.v).to(dev)
        r, v, f = torch.empty_like(r0), torch.empty_like(v0), torch.zeros_like(r0)
        PE = torch.zeros(steps, dtype=torch.float64, device=dev)
        KE = torch.zeros_like(PE)
        ts = []
        b0 = int(nl.stats()[0])
        for k in range(3):
            r.copy_(r0)
            v.copy_(v0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            nl.sort(r, v, st)
            P.md_energy_forces(s, pot, r, nl.plan, f, None, st)
            P.md_integrate_nve(s, pot, r, v, f, 1.0, c.dt, steps, nl.plan, PE, KE, True, st)
            e1.record()
            e1.synchronize()
            if k:
                ts.append(e0.elapsed_time(e1))
        ms = min(ts)
        E = (PE + KE).cpu().numpy()
        out[name] = {"N": c.N, "density": rho, "box": float(c.L), "ms": ms, "ms_per_step": ms / steps,
                     "particle_steps_per_s": c.N * steps / (ms * 1e-3),
                     "rebuilds_per_run": (int(nl.stats()[0]) - b0) / 3.0,
                     "max_abs_dE_total_per_particle": float(np.abs(E - E[0]).max() / c.N)}
    out["status"] = P.md_status_poll(st)
    return out


def order_section():
    """Sensitivity of the LJ force kernel (N = 256,000) to the particle order:
    one md_energy_forces in the generated FCC lattice order, in a random
    order, and in that random order after md_sort_particles (median of 10
    launches after 2, list rebuilt for each order)."""
    import torch
    import paper_1912_04232_b300 as P
    dev = torch.device("cuda")
    c = workload("lj256k", 0)
    s = P.md_space_periodic(3, [c.L] * 3)
    pot = P.lj_pot(c.eps, c.sigma, c.r_cut, True)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    nl = P.NeighborList(s, c.N, c.r_cut, c.skin, 128)
    out = {}
    p = np.random.default_rng(0).permutation(c.N)
    for name, r0, sort in (("lattice_order", c.r, False), ("random_order", c.r[p], False),
                           ("random_order_sorted", c.r[p], True)):
        r = torch.from_numpy(np.ascontiguousarray(r0)).to(dev)
        f = torch.zeros_like(r)
        if sort:
            nl.sort(r, None, st)
        else:
            nl.build(r, st)
        ts = []
        for k in range(12):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            P.md_energy_forces(s, pot, r, nl.plan, f, None, st)
            e1.record()
            e1.synchronize()
            if k >= 2:
                ts.append(e0.elapsed_time(e1))
        out[name + "_force_us"] = 1e3 * statistics.median(ts)
    out["status"] = P.md_status_poll(st)
    return out


def packing_section(nseed=20):
    """Sec. 4.2, Fig. 3, and the gradient-descent rows.  (i) The App. A
    system (128 disks, half of diameter D and half of diameter 1, packing
    fraction 0.9, 300 FIRE steps, reverse mode with K = 18 checkpoints) for
    D = 0.60, 0.65, ..., 1.00 and the reciprocal peak ratio 1.25, `nseed`
    seeded random starts each: the mean minimised energy (Fig. 3(b)) and
    dE_final/dD (Fig. 3(c)).  Per-start derivatives through a minimisation
    are heavy-tailed (a start near a saddle gives a huge value), so the
    median and a trimmed mean are reported beside the mean.  (ii) The
    configuration-2 packing (N = 1,024, D = 1.4, 2,000 gradient-descent
    steps of 0.05): the forward minimisation and the adjoint
    (K = ceil(sqrt(2000)) = 45) timed alone."""
    import torch
    import paper_1912_04232_b300 as P
    import workloads as W
    dev = torch.device("cuda")
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    out = {}
    N, T, K, phi = 128, 300, 18, 0.9
    wsz = P.md_fire_adjoint_workspace_size(N, T, K)
    wsb = torch.empty(wsz + 256, dtype=torch.uint8, device=dev)
    wsv = wsb[(-wsb.data_ptr()) % 256:]
    # one set of buffers for every run, so that each size ratio's runs share
    # one captured graph (the adjoint caches a graph per argument set)
    s0 = torch.zeros((N, 4), dtype=torch.float32, device=dev)
    ra, va, fa = (torch.zeros((N, 4), dtype=torch.float32, device=dev) for _ in range(3))
    o = torch.zeros(2, dtype=torch.float64, device=dev)
    rows, t_all = [], 0.0
    for D in [0.6 + 0.05 * k for k in range(9)] + [1.25]:
        L64 = W.packing_box(N, D, phi)
        s = P.md_space_periodic(2, [W.f32(L64)] * 2)
        nl = P.NeighborList(s, N, max(D, 1.0), 0.3, 64, canonical=True)
        Es, gs = [], []
        for seed in range(nseed):
            pk = W.packing_2d(N=N, D=D, phi=phi, seed=seed)
            s0[:, :2] = torch.from_numpy(pk.s0.astype(np.float32)).to(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            P.md_minimize_fire_adjoint(s, P.soft_pot(), P.fire_params(), nl.plan, s0, N // 2, D, 1.0, phi, T, K,
                                       ra, va, fa, wsv, o, st)
            e1.record()
            e1.synchronize()
            t_all += e0.elapsed_time(e1)
            oc = o.cpu().numpy()
            Es.append(float(oc[0]))
            gs.append(float(oc[1]))
        g = np.sort(np.asarray(gs))
        cut = len(g) // 10
        rows.append({"D": round(D, 3), "E_mean": float(np.mean(Es)), "E_se": float(np.std(Es) / math.sqrt(nseed)),
                     "dE_dD_median": float(np.median(g)), "dE_dD_trimmed_mean": float(np.mean(g[cut:len(g) - cut])),
                     "dE_dD_mean": float(np.mean(g))})
    scan = [r for r in rows if r["D"] <= 1.0]
    out["fig3_app_a"] = {"N": N, "fire_steps": T, "starts_per_D": nseed, "curve": rows,
                         "argmax_E_over_D_le_1": max(scan, key=lambda r: r["E_mean"])["D"],
                         "argmin_E_over_D_le_1": min(scan, key=lambda r: r["E_mean"])["D"],
                         "adjoint_runs_per_s": len(rows) * nseed / (t_all * 1e-3)}
    # configuration 2: gradient descent and its adjoint, N = 1,024
    N2, T2, K2, D2 = 1024, 2000, 45, 1.4
    pk = W.packing_2d(N=N2, D=D2, phi=phi, seed=0)
    L64 = W.packing_box(N2, D2, phi)
    L = W.f32(L64)
    s = P.md_space_periodic(2, [L, L])
    nl = P.NeighborList(s, N2, D2, 0.3, 64)
    x = np.zeros((N2, 4), np.float32)
    x[:, :2] = (pk.s0 * L).astype(np.float32)
    x[:, :2] = np.where(x[:, :2] >= L, 0.0, x[:, :2])
    x[:, 3] = pk.diam.astype(np.float32)
    x0 = torch.from_numpy(x).to(dev)
    r, f = torch.empty_like(x0), torch.zeros_like(x0)
    E = torch.zeros(T2 + 1, dtype=torch.float64, device=dev)
    tg = []
    for k in range(3):
        r.copy_(x0)
        nl.build(r, st)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        P.md_minimize(s, P.soft_pot(), 0, 0.05, T2, r, f, nl.plan, E, st)
        e1.record()
        e1.synchronize()
        if k:
            tg.append(e0.elapsed_time(e1))
    nlc = P.NeighborList(s, N2, D2, 0.3, 64, canonical=True)
    s0 = torch.zeros((N2, 4), dtype=torch.float32, device=dev)
    s0[:, :2] = torch.from_numpy(pk.s0.astype(np.float32)).to(dev)
    ws = torch.empty(P.md_adjoint_workspace_size(N2, T2, K2), dtype=torch.uint8, device=dev)
    o = torch.zeros(2, dtype=torch.float64, device=dev)
    ta = []
    for k in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        P.md_minimize_adjoint(s, P.soft_pot(), nlc.plan, s0, N2 // 2, D2, 1.0, phi, 0.05, T2, K2, r, f, ws, o, st)
        e1.record()
        e1.synchronize()
        if k:
            ta.append(e0.elapsed_time(e1))
    oc = o.cpu().numpy()
    out["cfg2_gd"] = {"N": N2, "D": D2, "gd_steps": T2, "gd_ms": min(tg),
                      "gd_particle_steps_per_s": N2 * T2 / (min(tg) * 1e-3),
                      "E_start": float(E[0].item()), "E_end": float(E[-1].item()),
                      "adjoint_ms": min(ta), "adjoint_over_forward": min(ta) / min(tg), "checkpoints": K2,
                      "E_final": float(oc[0]), "dE_dD": float(oc[1])}
    out["status"] = P.md_status_poll(st)
    return out


def fire_section():
    """FIRE minimisation: a quench of the N = 256,000 LJ liquid (200 steps,
    dt_start = the NVE dt, dt_max = 4x) and the App. A packing (128 disks,
    D = 1.4, packing fraction 0.9, 300 steps, Bitzek's parameters)."""
    import torch
    import paper_1912_04232_b300 as P
    import workloads as W
    dev = torch.device("cuda")
    out = {}
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    sb = P.md_fire_state_bytes()
    state = torch.zeros(sb + 256, dtype=torch.uint8, device=dev)
    state = state[(-state.data_ptr()) % 256:][:sb]

    def run(s, pot, prm, r0, rc, nsteps, reps):
        nl = P.NeighborList(s, r0.shape[0], rc, 0.3, 128)
        r = torch.empty_like(r0)
        v = torch.zeros_like(r0)
        f = torch.zeros_like(r0)
        E = torch.zeros(nsteps + 1, dtype=torch.float64, device=dev)
        ts = []
        for k in range(reps + 1):
            r.copy_(r0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            nl.build(r, st)
            P.md_minimize_fire(s, pot, prm, nsteps, r, v, f, nl.plan, state, True, E, st)
            e1.record()
            e1.synchronize()
            if k:
                ts.append(e0.elapsed_time(e1))
        return min(ts), E.cpu().numpy(), P.md_fire_state_read(state)

    c = W.lj_large(0)
    s = P.md_space_periodic(3, [c.L] * 3)
    r0 = torch.from_numpy(c.r).to(dev)
    ms, E, fs = run(s, P.lj_pot(), P.fire_params(dt_start=0.005, dt_max=0.02), r0, 2.5, 200, 2)
    out["lj256k_quench"] = {"N": c.N, "steps": 200, "ms": ms, "particle_steps_per_s": c.N * 200 / (ms * 1e-3),
                            "E_per_particle_start": float(E[0] / c.N), "E_per_particle_end": float(E[-1] / c.N),
                            "final_dt_alpha_count": fs}
    pk = W.packing_2d(N=128, D=1.4, phi=0.9, seed=0)
    L = W.f32(W.packing_box(pk.N, pk.D, pk.phi))
    x = np.zeros((pk.N, 4), np.float32)
    x[:, :2] = (pk.s0 * L).astype(np.float32)
    x[:, :2] = np.where(x[:, :2] >= L, 0.0, x[:, :2])
    x[:, 3] = pk.diam.astype(np.float32)
    s2 = P.md_space_periodic(2, [L, L])
    ms2, E2, fs2 = run(s2, P.soft_pot(), P.fire_params(), torch.from_numpy(x).to(dev), 1.4, 300, 5)
    out["app_a_packing"] = {"N": pk.N, "steps": 300, "ms": ms2, "us_per_step": 1e3 * ms2 / 300,
                            "E_start": float(E2[0]), "E_end": float(E2[-1])}
    # dE_final/dD through the 300 FIRE steps (reverse mode, K = 18)
    L64 = W.packing_box(pk.N, pk.D, pk.phi)
    nlc = P.NeighborList(s2, pk.N, 1.4, 0.3, 64, canonical=True)
    s0 = torch.zeros((pk.N, 4), dtype=torch.float32, device=dev)
    s0[:, :2] = torch.from_numpy(pk.s0.astype(np.float32)).to(dev)
    ra, va, fa = (torch.zeros((pk.N, 4), dtype=torch.float32, device=dev) for _ in range(3))
    wsz = P.md_fire_adjoint_workspace_size(pk.N, 300, 18)
    wsb = torch.empty(wsz + 256, dtype=torch.uint8, device=dev)
    wsv = wsb[(-wsb.data_ptr()) % 256:]
    outd = torch.zeros(2, dtype=torch.float64, device=dev)
    ta = []
    for k in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        P.md_minimize_fire_adjoint(s2, P.soft_pot(), P.fire_params(), nlc.plan, s0, pk.N // 2, pk.D, 1.0, pk.phi, 300,
                                   18, ra, va, fa, wsv, outd, st)
        e1.record()
        e1.synchronize()
        if k:
            ta.append(e0.elapsed_time(e1))
    o = outd.cpu().numpy()
    out["app_a_fire_adjoint"] = {"N": pk.N, "steps": 300, "K": 18, "ms": min(ta), "E_final": float(o[0]),
                                 "dE_dD": float(o[1])}
    code = P.md_status_poll(st)
    out["status"] = code
    return out


def tiles_section(reps=3):
    """The bench job (LJ N = 256,000 from the same seeded start: neighbor
    build, initial forces, 1,000 velocity-Verlet steps in one graph launch)
    on the tile engine (MD_NBR_TILES), L2 flushed between repetitions."""
    import torch
    import paper_1912_04232_b300 as P
    import workloads as W
    dev = torch.device("cuda")
    c = W.lj_large(seed=0)
    s = P.md_space_periodic(3, [c.L] * 3)
    nl = P.NeighborList(s, c.N, c.r_cut, c.skin, 128, tiles=True)
    pot = P.lj_pot()
    r0, v0 = torch.from_numpy(c.r).to(dev), torch.from_numpy(c.v).to(dev)
    r, v, f = r0.clone(), v0.clone(), torch.zeros_like(r0)
    PE = torch.zeros(c.steps, dtype=torch.float64, device=dev)
    KE = torch.zeros_like(PE)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)

    def job():
        r.copy_(r0)
        v.copy_(v0)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        nl.build(r, st)
        P.md_energy_forces(s, pot, r, nl.plan, f, None, st)
        P.md_integrate_nve(s, pot, r, v, f, c.mass, c.dt, c.steps, nl.plan, PE, KE, True, st)
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1)

    job()
    ms = min(job() for _ in range(reps))
    b0, _ = nl.stats()
    e = (PE + KE).cpu().numpy()
    info = P.md_tiles_info(s, nl.plan)
    return {"engine": "tiles (MD_NBR_TILES)", "N": c.N, "md_steps": c.steps, "ms_per_job": ms,
            "particle_steps_per_s": c.N * c.steps / (ms * 1e-3), "builds_since_plan": int(b0),
            "max_energy_drift_per_particle": float(np.abs(e - e[0]).max() / c.N),
            "tile": info["tile"], "ntiles": info["ntiles"], "status": P.md_status_poll(st)}


def nhc_section(steps=200):
    """Nose-Hoover chain NVT (chain length 3, tau = 100 dt): the N = 256,000
    LJ fluid at T* = 1 and Stillinger-Weber silicon, N = 64,000 atoms at
    1000 K (dt = 1 fs), each for `steps` steps in one graph launch."""
    import torch
    import paper_1912_04232_b300 as P
    import paper_1912_04232_b300.learned as LP
    import workloads as W
    dev = torch.device("cuda")
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    out = {}

    def run(s, pot, r0, v0, rc, skin, cap, mass, dt, kT, reps=2):
        nl = P.NeighborList(s, r0.shape[0], rc, skin, cap)
        r, v, f = torch.empty_like(r0), torch.empty_like(v0), torch.zeros_like(r0)
        th = torch.zeros(P.md_nhc_state_doubles(3), dtype=torch.float64, device=dev)
        H = torch.zeros(steps, dtype=torch.float64, device=dev)
        KE = torch.zeros_like(H)
        ts = []
        for k in range(reps + 1):
            r.copy_(r0)
            v.copy_(v0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            nl.build(r, st)
            P.md_energy_forces(s, pot, r, nl.plan, f, None, st)
            P.md_integrate_nhc(s, pot, r, v, f, mass, dt, kT, 100.0 * dt, 3, steps, nl.plan, th, True, None, KE, H,
                               USE_GRAPH, st)
            e1.record()
            e1.synchronize()
            if k:
                ts.append(e0.elapsed_time(e1))
        N = r0.shape[0]
        Hn = H.cpu().numpy()
        return {"N": N, "steps": steps, "ms": min(ts), "particle_steps_per_s": N * steps / (min(ts) * 1e-3),
                "max_abs_dH_per_particle": float(np.abs(Hn - Hn[0]).max() / N),
                "T_end_over_T": float(KE[-1].item() / (1.5 * N * kT))}

    c = W.lj_large(0)
    out["lj256k"] = run(P.md_space_periodic(3, [c.L] * 3), P.lj_pot(), torch.from_numpy(c.r).to(dev),
                        torch.from_numpy(c.v).to(dev), 2.5, 0.3, 128, 1.0, c.dt, 1.0)
    si = W.sw_silicon(20, T_K=1000.0, seed=0)
    out["sw_si64k_1000K"] = run(P.md_space_periodic(3, [si.L] * 3), P.sw_pot(LP.SW_SI, N=si.N),
                                torch.from_numpy(si.r).to(dev), torch.from_numpy(si.v).to(dev), float(LP.SW_RC), 0.5,
                                64, LP.MASS_SI, 1.0, W.KB_EV * 1000.0)
    out["status"] = P.md_status_poll(st)
    return out


def _hbm_peak():
    """(GB/s, source): the measured copy bandwidth, else the fallback figure."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6400.0, "fallback"


_FP32_PEAK = {}


def fp32_peak():
    """(TFLOP/s, source): FP32 FMA throughput measured with the library's
    FMA-chain probe (4 CTAs of 1,024 threads per SM, 8 independent chains
    per thread, median of 5 launches after 3 warm-ups), with the derived
    148 SMs x 128 lanes x 2 FLOP x 2,032 MHz beside it."""
    if _FP32_PEAK:
        return _FP32_PEAK["tflops"], _FP32_PEAK["source"]
    import torch
    import paper_1912_04232_b300 as P
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    blocks, threads, iters = 4 * nsm, 1024, 1 << 15
    out = torch.empty(blocks * threads, dtype=torch.float32, device="cuda")
    ts = []
    for k in range(8):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fl = P.md_fma_probe(out, blocks, threads, iters)
        e1.record()
        e1.synchronize()
        if k >= 3:
            ts.append(e0.elapsed_time(e1))
    tfl = fl / (statistics.median(ts) * 1e-3) / 1e12
    _FP32_PEAK.update(tflops=tfl, source="measured: FMA-chain probe (derived 148 x 128 x 2 x 2032 MHz = %.1f)"
                      % (148 * 128 * 2 * 2032e6 / 1e12))
    return tfl, _FP32_PEAK["source"]


def gnn_section(steps=100, H=64, T=2):
    """Graph-network potential deployed in Nose-Hoover NVT: silicon, N =
    64,000 atoms at 1000 K (dt = 1 fs, r_c = 3.77 A, hidden width H, T
    message-passing steps, seeded random weights that are BF16-representable,
    so the FP32 and the tensor-core kernels hold the same model), `steps`
    steps in one graph launch, and one energy + force evaluation timed
    alone; for the FP32 CUDA-core kernels and for the tcgen05 kernels."""
    import torch
    import paper_1912_04232_b300 as P
    import paper_1912_04232_b300.learned as LP
    import workloads as W
    dev = torch.device("cuda")
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    si = W.sw_silicon(20, T_K=1000.0, seed=0)
    N, cap, rc = si.N, 48, 3.77
    s = P.md_space_periodic(3, [si.L] * 3)
    nl = P.NeighborList(s, N, rc, 0.5, cap)
    params = torch.from_numpy(W.gnn_params(H, T, seed=0, out_scale=0.3, bf16=True)).to(dev)
    model = P.GNNModel(params, N, cap, H, T, rc)
    r0, v0 = torch.from_numpy(si.r).to(dev), torch.from_numpy(si.v).to(dev)
    r, v, f = torch.empty_like(r0), torch.empty_like(v0), torch.zeros_like(r0)
    th = torch.zeros(P.md_nhc_state_doubles(3), dtype=torch.float64, device=dev)
    Hx = torch.zeros(steps, dtype=torch.float64, device=dev)
    KE = torch.zeros_like(Hx)
    kT, dt = W.KB_EV * 1000.0, 1.0
    fp32_pk, fp32_src = fp32_peak()
    out = {"N": N, "H": H, "T": T, "steps": steps, "weights": "seeded random, BF16-representable (out_scale 0.3)"}
    for name, tc in (("fp32", 0), ("tcgen05", 1)):
        P.md_gnn_set_tensor_cores(tc)
        ts, tf = [], []
        for k in range(3):
            r.copy_(r0)
            v.copy_(v0)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record()
            nl.build(r, st)
            P.md_energy_forces(s, model.pot, r, nl.plan, f, None, st)
            e1.record()
            P.md_integrate_nhc(s, model.pot, r, v, f, LP.MASS_SI, dt, kT, 100.0 * dt, 3, steps, nl.plan, th, True,
                               None, KE, Hx, USE_GRAPH, st)
            e2.record()
            e2.synchronize()
            if k:
                ts.append(e1.elapsed_time(e2))
        for k in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            P.md_energy_forces(s, model.pot, r, nl.plan, f, None, st)
            e1.record()
            e1.synchronize()
            if k >= 2:
                tf.append(e0.elapsed_time(e1))
        # edges within r_c on the final configuration
        n = nl.cnt.clamp(max=cap).long()
        rows = nl.nbr.long().clamp(max=N - 1)
        d = r[rows, :3] - r[:, None, :3]
        d -= float(si.L) * torch.round(d / float(si.L))
        valid = (torch.arange(cap, device=dev)[None, :] < n[:, None]) & ((d * d).sum(-1) < rc * rc)
        E_edges = int(valid.sum().item())
        # FP32 path: FLOP-bound by its products, 2H^2 (2T E + (8T - 3) N)
        # (edges: A_e forward per step, A_e^T of the step above and of step
        # 0 in reverse; nodes: B, A_r, A_s, D forward, D^T, B^T, A_r^T, A_s^T
        # reverse).  Tensor-core path: bound by the per-step edge and node
        # vectors in HBM, written once and read once in each direction:
        # 16 H T (E + N) bytes.
        Hn = Hx.cpu().numpy()
        ent = {"ms": min(ts), "atom_steps_per_s": N * steps / (min(ts) * 1e-3), "force_eval_ms": min(tf),
               "edges_within_rc_per_atom": E_edges / N, "max_abs_dH_per_atom": float(np.abs(Hn - Hn[0]).max() / N),
               "T_end_over_T": float(KE[-1].item() / (1.5 * N * kT))}
        if tc:
            byts = 16.0 * H * T * (E_edges + N)
            gbs = byts / (min(tf) * 1e-3) / 1e9
            hbm, src = _hbm_peak()
            ent["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                               "bytes_per_eval": byts, "peak_source": src}
        else:
            flops = 2.0 * H * H * (E_edges * 2 * T + N * (8 * T - 3))
            tfl = flops / (min(tf) * 1e-3) / 1e12
            ent["roofline"] = {"bound": "alu", "achieved": tfl, "peak": fp32_pk, "unit": "TFLOP/s",
                               "frac": tfl / fp32_pk, "flops_per_eval": flops, "peak_source": fp32_src}
        out[name] = ent
    P.md_gnn_set_tensor_cores(0)
    out["status"] = P.md_status_poll(st)
    return out


def flock_section(N=100000, steps=200, n_pred=8):
    """Flocking energy model: N boids with ~20 neighbours within the
    alignment range, 16 disk obstacles and n_pred predators, `steps`
    forward-Euler steps (dt = 0.1) with list rebuilds."""
    import torch
    import paper_1912_04232_b300 as P
    import workloads as W
    dev = torch.device("cuda")
    fl = W.flock(N, n_obs=16, seed=0, n_pred=n_pred)
    prm = P.flock_params()
    s = P.md_space_periodic(2, [fl.L, fl.L])
    nl = P.NeighborList(s, N, max(prm.R_align, prm.R_avoid, prm.R_cohesion), 4.0, 128)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    b0 = torch.zeros((N, 4), dtype=torch.float32, device=dev)
    b0[:, :2] = torch.from_numpy(fl.R).to(dev)
    th0 = torch.from_numpy(fl.theta).to(dev)
    obs = torch.from_numpy(fl.obstacles).to(dev)
    b, th, alt = torch.empty_like(b0), torch.empty_like(th0), torch.empty_like(b0)
    p0 = torch.zeros((n_pred, 4), dtype=torch.float32, device=dev)
    p0[:, :3] = torch.from_numpy(fl.predators).to(dev)
    pr, pr_alt = torch.empty_like(p0), torch.empty_like(p0)
    E = torch.zeros(steps, dtype=torch.float64, device=dev)
    ts = []
    b1 = nl.stats()[0]
    for k in range(3):
        b.copy_(b0)
        th.copy_(th0)
        pr.copy_(p0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        nl.build(b, st)
        P.md_flock_run(s, prm, obs, obs.shape[0], pr, pr_alt, n_pred, b, th, alt, 0.1, steps, nl.plan, E, st)
        e1.record()
        e1.synchronize()
        if k:
            ts.append(e0.elapsed_time(e1))
    ms = min(ts)
    En = E.cpu().numpy()
    return {"N": N, "predators": n_pred, "steps": steps, "ms": ms, "boid_steps_per_s": N * steps / (ms * 1e-3),
            "builds_per_run": (nl.stats()[0] - b1) / 3.0, "E_start": float(En[0]), "E_end": float(En[-1]),
            "status": P.md_status_poll(st)}


def _source_sha():
    """Hash of the sources of the pair-force kernels (a stored DRAM-traffic
    figure is only reported while it still describes the built kernel)."""
    h = hashlib.sha256()
    for p in ("paper_1912_04232_b300/csrc/pair.cu", "paper_1912_04232_b300/csrc/common.cuh",
              "paper_1912_04232_b300/csrc/kernels.cuh", "paper_1912_04232_b300/csrc/reduce.cuh",
              "paper_1912_04232_b300/csrc/cells.cuh"):
        with open(os.path.join(ROOT, p), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def max_over_ranks(x, dist=None, device=None):
    """The largest value of x over all ranks (x itself without a process
    group): the whole job takes as long as its slowest rank."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(n_particles, md_steps, steps, world, ms_max):
    """Particle-steps per second of the whole job: every rank advances its
    own system of n_particles (weak scaling), timed by the slowest rank."""
    return n_particles * md_steps * steps * world / (ms_max * 1e-3)


def sw_evolved_64000(steps=200):
    """64,000 diamond-silicon atoms after `steps` SW NVE steps (1 fs) from
    the 1000 K lattice start: the thermal configuration the deployed kernels
    see (at the lattice start every atom has exactly four partners inside
    the cutoff; at 1000 K some second neighbors come inside).  Returns the
    workload, the space and the positions on the GPU."""
    import torch
    import paper_1912_04232_b300 as J
    import paper_1912_04232_b300.learned as LP
    import workloads as W
    si = W.sw_silicon(20, T_K=1000.0, seed=0)
    space = J.md_space_periodic(3, [si.L] * 3)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    sw = J.sw_pot(LP.SW_SI, N=si.N)
    nl = J.NeighborList(space, si.N, LP.SW_RC, 0.3, 64)
    r = torch.from_numpy(si.r).cuda()
    v = torch.from_numpy(si.v).cuda()
    f = torch.zeros_like(r)
    nl.build(r, st)
    J.md_energy_forces(space, sw, r, nl.plan, f, None, st)
    J.md_integrate_nve(space, sw, r, v, f, LP.MASS_SI, 1.0, steps, nl.plan, None, None, True, st)
    torch.cuda.synchronize()
    if J.md_status_poll(st):
        raise RuntimeError("SW NVE for the evolved configuration failed")
    return si, space, r


def learned_kernels(params=None, norm=None):
    """CUDA-event timings of the learned potential's kernels at 64,000 SW
    silicon atoms (after 200 SW NVE steps from the 1000 K start):
    descriptors, the network (tcgen05 and FP32), the force gather over the
    neighbor rows, a whole BP force evaluation in both forms (partner lists
    stored by the descriptor kernel, the deployed form; rows), and SW forces
    in both forms; and each kernel's fraction of its roofline.  FLOPs (FMA = 2; exp, sin/cos,
    divide = 1): the network 2 (16x64 + 64x64 + 64x64 + 64x16) = 20,480 per
    atom on the tensor cores (BF16 peak of MEASURED_PEAKS.json); the
    descriptors 44 per pair inside R_c (cutoff 4, eight Gaussians 40) and 50
    per centred triplet (legs and cosine 9, cutoffs and exponential 10, the
    powers 12, eight columns 16, sums 3); the force gather 90 per pair (both
    atoms' weights, radial derivative) and 110 per triplet, centred or as a
    leg (the triplet's scalars 50, the weight sums 32, the two leg gradients
    28), against the measured FP32 peak."""
    import torch
    import paper_1912_04232_b300 as J
    import paper_1912_04232_b300.learned as LP
    si, space, r = sw_evolved_64000()
    N, L = si.N, si.L
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    if params is None:
        rng = np.random.default_rng(0)
        params = torch.from_numpy((rng.normal(size=J.BP_NPARAMS) * 0.1).astype(np.float32)).cuda()
        norm = torch.cat([torch.zeros(16), torch.ones(16)]).float().cuda()
    model = J.BPModel(params, norm, N)
    model_rows = J.BPModel(params, norm, N, lists=False)
    nl = J.NeighborList(space, N, LP.SW_RC, 0.3, 64)
    nl.build(r, st)
    G = torch.zeros((N, 16), device="cuda")
    Ei = torch.zeros(N, device="cuda")
    dEdG = torch.zeros((N, 16), device="cuda")
    f = torch.zeros((N, 4), device="cuda")
    sw = J.sw_pot(LP.SW_SI)
    sw_lists = J.sw_pot(LP.SW_SI, N=N)

    def t(fn, K=50):
        for _ in range(5):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(K):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / K * 1000

    out = {"N": N, "us": {
        "k_bp_desc": t(lambda: J.md_bp_descriptors(space, r, nl.plan, 0, G, st)),
        "k_mlp_infer_tc": t(lambda: J.md_bp_mlp_infer_tc(params, norm, G, N, Ei, dEdG, st)),
        "k_mlp_infer_fp32": t(lambda: J.md_bp_mlp_infer(params, norm, G, N, Ei, dEdG)),
        "k_bp_force": t(lambda: J.md_bp_forces(space, r, nl.plan, 0, dEdG, Ei, f, None, st))}}
    J.md_bp_set_tensor_cores(True)
    out["us"]["bp_energy_forces_tc"] = t(lambda: J.md_energy_forces(space, model.pot, r, nl.plan, f, None, st))
    out["us"]["bp_energy_forces_tc_rows"] = t(lambda: J.md_energy_forces(space, model_rows.pot, r, nl.plan, f, None,
                                                                           st))
    J.md_bp_set_tensor_cores(False)
    out["us"]["k_sw"] = t(lambda: J.md_energy_forces(space, sw, r, nl.plan, f, None, st))
    out["us"]["sw_forces_lists"] = t(lambda: J.md_energy_forces(space, sw_lists, r, nl.plan, f, None, st))
    out["configuration"] = "after 200 SW NVE steps (1 fs) from the 1000 K lattice start"
    # partners inside R_c per atom, for the FLOP counts
    cap = nl.cap
    n = nl.cnt.clamp(max=cap).long()
    rows = nl.nbr.long().clamp(max=N - 1)
    d = r[rows, :3] - r[:, None, :3]
    d -= float(L) * torch.round(d / float(L))
    inside = (torch.arange(cap, device="cuda")[None, :] < n[:, None]) & ((d * d).sum(-1) < LP.BP_RC ** 2)
    m = inside.sum(1).double()
    pairs, cent, legs = float(m.sum()), float((m * (m - 1) / 2).sum()), float((m * (m - 1)).sum())
    fp32_pk, _ = fp32_peak()
    try:
        bf16_pk = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except (OSError, ValueError, KeyError):
        bf16_pk = 1800.0
    us = out["us"]
    fl = {"k_bp_desc": 44.0 * pairs + 50.0 * cent, "k_mlp_infer_tc": 20480.0 * N,
          "k_bp_force": 90.0 * pairs + 110.0 * (cent + legs)}
    pk = {"k_bp_desc": fp32_pk, "k_mlp_infer_tc": bf16_pk, "k_bp_force": fp32_pk}
    out["roofline"] = {k: {"bound": "tensor" if k == "k_mlp_infer_tc" else "alu",
                           "achieved_tflops": fl[k] / (us[k] * 1e-6) / 1e12, "peak_tflops": pk[k],
                           "frac": fl[k] / (us[k] * 1e-6) / 1e12 / pk[k],
                           "share_of_evaluation": us[k] / (us["k_bp_desc"] + us["k_mlp_infer_tc"] + us["k_bp_force"])}
                       for k in fl}
    out["pairs_per_atom"] = pairs / N
    out["triplets_per_atom"] = {"centred": cent / N, "leg": legs / N}
    out["status"] = J.md_status_poll(st)
    return out


def probe_batch_steps(steps=30):
    """The 512-replica batch (configuration 4) advanced `steps` NVE steps as
    host launches, so that a profiler lists every kernel of the step (the
    graph form hides the kernels of its conditional nodes); prints the
    CUDA-event time per step and the replica rebuilds."""
    import torch
    import paper_1912_04232_b300 as P
    import workloads as W
    dev = torch.device("cuda")
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    specs = W.replica_plan(R=512, n_max=8192, seed=0)
    _, descs, r0, v0 = batch_setup(specs, dev, st)
    r, v, f = r0.clone(), v0.clone(), torch.zeros_like(r0)
    b = P.Batch(descs, cap=128)
    P.md_batch_build(b.plan, r, st)
    P.md_batch_forces(b.plan, r, f, st)
    P.md_batch_run_nve(b.plan, r, v, f, 20, None, None, False, st)
    b0 = sum(P.md_batch_stats(b.plan))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    P.md_batch_run_nve(b.plan, r, v, f, steps, None, None, False, st)
    e1.record()
    e1.synchronize()
    print(json.dumps({"replicas": len(specs), "N": int(b.plan.N), "steps": steps,
                      "us_per_step": e0.elapsed_time(e1) * 1e3 / steps,
                      "replica_builds_per_step": (sum(P.md_batch_stats(b.plan)) - b0) / steps,
                      "status": P.md_status_poll(st)}), flush=True)


def probe_learned_kernels():
    print(json.dumps(learned_kernels()), flush=True)


def probe_train_step():
    """CUDA-event timings of one BP training step (8 snapshots of 512 SW
    silicon atoms): forward, descriptor JVP, network gradient on the tensor
    cores and in FP32, Adam."""
    import torch
    import paper_1912_04232_b300 as J
    import paper_1912_04232_b300.learned as LP
    ds = LP.generate_sw_dataset(np.linspace(500.0, 3000.0, 8), n_snap=4, stride=20, equil=100, seed=1)
    LP.build_lists(ds)
    tr = LP.Trainer(ds, batch=8, lr=3e-3, wF=1.0, seed=0)
    for _ in range(5):
        tr.step(0)
    torch.cuda.synchronize()
    n = ds.n
    acc = {}
    K = 50
    for _ in range(K):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        ev[0].record()
        nb, r, N = tr.forward(0, tr.B)
        ev[1].record()
        J.md_bp_jvp(tr.space, r, nb, n, tr.dF[:N], tr.V[:N], tr.status)
        ev[2].record()
        J.md_bp_mlp_train_tc(tr.params, tr.norm, tr.G[:N], tr.V[:N], tr.cE[:N], 1.0, N, tr.scratch, tr.grad,
                             tr.status)
        ev[3].record()
        J.md_bp_mlp_train(tr.params, tr.norm, tr.G[:N], tr.V[:N], tr.cE[:N], 1.0, N, tr.scratch, tr.grad)
        ev[4].record()
        tr.step_count += 1
        J.md_adam_step(tr.params, tr.grad, tr.m, tr.v, LP.N_PARAMS, tr.lr, 0.9, 0.999, 1e-8, tr.step_count)
        ev[5].record()
        torch.cuda.synchronize()
        for k, name in enumerate(["forward", "jvp", "network_gradient_tc", "network_gradient_fp32", "adam"]):
            acc[name] = acc.get(name, 0.0) + ev[k].elapsed_time(ev[k + 1]) * 1000 / K
    print(json.dumps({"atoms": int(N), "us": acc, "status": J.md_status_poll(tr.status)}), flush=True)


def main():
    args = parse()
    if args.probe == "learned-kernels":
        probe_learned_kernels()
        return
    if args.probe == "train-step":
        probe_train_step()
        return
    if args.probe == "batch-steps":
        probe_batch_steps()
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    # CPU baseline first (before any CUDA work), rank 0 at N=1 only
    cpu_baseline = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        md = 20 if args.workload == "lj256k" else 200
        val, thr, dt = oracle_sample(args.workload, md)
        Nw = workload(args.workload, 0).N
        cpu_baseline = {"value": val, "unit": UNIT, "cores": thr, "kind": "oracle",
                        "sample": f"{md} FP64 NVE steps of the N={Nw} LJ workload ({dt:.1f} s)"}
        # the same oracle on one thread, over a shorter sample
        import oracle as O
        O.set_num_threads(1)
        md1 = 2 if args.workload == "lj256k" else 40
        val1, _, dt1 = oracle_sample(args.workload, md1)
        O.set_num_threads(thr)
        cpu_baseline["single_thread"] = {"value": val1, "unit": UNIT, "cores": 1,
                                         "sample": f"{md1} FP64 NVE steps of the same workload ({dt1:.1f} s)"}

    import torch
    import paper_1912_04232_b300 as P

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    c = workload(args.workload, seed=rank)
    md_steps = args.md_steps or c.steps
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    if args.tpp:
        P.md_set_pair_tpp(args.tpp)
    if args.tile_tpp:
        P.md_set_tile_tpp(args.tile_tpp)
    tiles = bool(args.tiles) and not args.local_rows
    if args.pair_opt >= 0:
        P.md_set_pair_options(args.pair_opt)
    P.md_set_nve_fusion(bool(args.nve_fusion))
    P.md_set_loop_graphs(not args.no_graph)
    global USE_GRAPH
    USE_GRAPH = not args.no_graph
    s = P.md_space_periodic(3, [c.L] * 3)
    nl = P.NeighborList(s, c.N, c.r_cut, c.skin, 128, local_rows=bool(args.local_rows), tiles=tiles)
    pot = P.lj_pot(c.eps, c.sigma, c.r_cut, True)
    r0 = torch.from_numpy(c.r).to(dev)
    v0 = torch.from_numpy(c.v).to(dev)
    r = torch.empty_like(r0)
    v = torch.empty_like(v0)
    f = torch.zeros_like(r0)
    PE = torch.zeros(md_steps, dtype=torch.float64, device=dev)
    KE = torch.zeros(md_steps, dtype=torch.float64, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 126 MB L2

    # Z-order sort of the particles at the start of each job (md_sort_particles
    # also builds the list); scratch and permutation allocated once, here
    sort_perm = torch.empty(c.N, dtype=torch.int32, device=dev)
    sort_raw = torch.empty(P.md_sort_scratch_bytes(nl.plan) + 256, dtype=torch.uint8, device=dev)
    sort_ws = sort_raw[(-sort_raw.data_ptr()) % 256:]

    def job():
        if args.sort and not tiles:
            P.md_sort_particles(s, nl.plan, r, v, sort_perm, sort_ws, st)
        else:
            nl.build(r, st)
        P.md_energy_forces(s, pot, r, nl.plan, f, None, st)
        P.md_integrate_nve(s, pot, r, v, f, c.mass, c.dt, md_steps, nl.plan, PE, KE, not args.no_graph, st)

    def one_step():
        r.copy_(r0)
        v.copy_(v0)
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        job()
        e1.record(stream)
        return e0, e1

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    code = P.md_status_poll(st)
    if code != 0:
        raise SystemExit(f"device status {code} after warm-up")
    b0, _ = nl.stats()
    launches0 = P.md_launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    evs = [one_step() for _ in range(args.steps)]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    launches = P.md_launch_count() - launches0
    builds = nl.stats()[0] - b0
    code = P.md_status_poll(st)
    if code != 0:
        raise SystemExit(f"device status {code} in the timed region")
    E = (PE + KE).cpu().numpy()
    drift = float(np.abs(E - E[0]).max() / c.N)
    # the GPU run's energies against the FP64 oracle over the oracle's sample
    # (the CPU-baseline steps, same start), per particle
    drift_vs_oracle = None
    Eo = ORACLE_SERIES.get((args.workload, 0, 20 if args.workload == "lj256k" else 200))
    if Eo is not None and rank == 0:
        m = min(len(Eo) - 1, len(E))
        drift_vs_oracle = {"steps": m, "max_abs_dE_per_particle": float(np.abs(E[:m] - Eo[1:m + 1]).max() / c.N),
                           "drift_gpu": float(np.abs(E[:m] - E[0]).max() / c.N),
                           "drift_oracle": float(np.abs(Eo[1:m + 1] - Eo[1]).max() / c.N)}

    t_max = max_over_ranks(ms, dist, dev)
    total_ps = c.N * md_steps * args.steps * world
    value = whole_job_rate(c.N, md_steps, args.steps, world, t_max)

    # end to end: host buffers in, energies out, every step
    e2e = None
    if not args.no_e2e:
        hr = torch.from_numpy(c.r).pin_memory()
        hv = torch.from_numpy(c.v).pin_memory()
        hpe = torch.empty(md_steps, dtype=torch.float64).pin_memory()
        hke = torch.empty(md_steps, dtype=torch.float64).pin_memory()
        tt = []
        for k in range(args.warmup + args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r.copy_(hr, non_blocking=True)
            v.copy_(hv, non_blocking=True)
            job()
            hpe.copy_(PE, non_blocking=True)
            hke.copy_(KE, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            if k >= args.warmup:
                tt.append(e0.elapsed_time(e1))
        e2e_ms = max_over_ranks(sum(tt), dist, dev)
        e2e = {"value": total_ps / (e2e_ms * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": int(hr.numel() * 4 + hv.numel() * 4),
               "d2h_bytes_per_step": int(hpe.numel() * 8 + hke.numel() * 8)}

    # roofline of the dominant kernel, launched alone with events on this stream
    peak, peak_src = _hbm_peak()
    traffic = None
    tr = {}
    try:
        tr = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    except (OSError, ValueError):
        pass
    if tiles:
        # the fused step kernel (k_t_step<LJ, 8, 2>): forces from the staged
        # region, closing half-kick, next kick-drift, displacement check.
        # K steps on the tiled copy with its rows fixed (md_tiles_steps: one
        # opening kick-drift launch, then K step launches); rows sized from
        # a fresh import of the start
        K = 20
        r.copy_(r0)
        v.copy_(v0)
        nl.build(r, st)
        P.md_energy_forces(s, pot, r, nl.plan, f, None, st)
        P.md_tiles_import(s, r, v, f, nl.plan, st)
        P.md_tiles_export(s, nl.plan, None, None, None, rows=True)
        torch.cuda.synchronize()
        mean_cnt = float(nl.cnt.float().clamp(max=nl.cap).mean().item())
        # row entries (16-bit), count, own position (each staged position
        # counted once), v read + write, r_ref read, next position write
        bytes_per_particle = 2.0 * mean_cnt + 4 + 16 + 32 + 16 + 16
        fe = []
        for _ in range(6):
            P.md_tiles_import(s, r, v, f, nl.plan, st)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            P.md_tiles_steps(s, pot, nl.plan, c.mass, c.dt, K, None, None, st)
            e1.record(stream)
            fe.append((e0, e1))
        torch.cuda.synchronize()
        kt = statistics.median(a.elapsed_time(b) for a, b in fe[1:]) * 1e-3 / K
        kname = ("k_t_step1<LJ,2>" if (args.tile_tpp or 1) == 1 else f"k_t_step<LJ,{args.tile_tpp},2>") + " (fused step, md_tiles_steps)"
        ent = tr.get("k_t_step_lj", {})
    else:
        mean_cnt = float(nl.cnt.float().clamp(max=nl.cap).mean().item())
        row_bytes = 2.0 if args.local_rows else 4.0              # 16-bit local or int32 row entries
        bytes_per_particle = row_bytes * mean_cnt + 4 + 16 + 16 + 16   # row, count, own r, f write, gathered r once
        fe = []
        for _ in range(30):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            P.md_energy_forces(s, pot, r, nl.plan, f, None, st)
            e1.record(stream)
            fe.append((e0, e1))
        torch.cuda.synchronize()
        kt = statistics.median(a.elapsed_time(b) for a, b in fe[5:]) * 1e-3
        kname = ("k_pair_block<LJ>" if args.local_rows else "k_pair<LJ>") + " (md_energy_forces)"
        ent = tr.get("k_pair_block_lj" if args.local_rows else "k_pair_lj", {})
    achieved = bytes_per_particle * c.N / kt / 1e9
    if ent.get("source_sha") == _source_sha() and ent.get("N") == c.N:
        traffic = ent.get("dram_bytes_per_launch")
    code = P.md_status_poll(st)
    if code & ~P.MD_ERR_NBR_OVERFLOW:
        raise SystemExit(f"device status {code} in the roofline launches")

    extra = {}
    if rank == 0 and not args.no_fp32_peak:
        pk, src = fp32_peak()
        extra["fp32_fma_peak"] = {"tflops": pk, "source": src}
    if rank == 0 and not args.no_learned:
        extra["learned_vs_sw"] = learned_section()
    if not args.no_batch and (rank == 0 or world > 1):   # the replicas split over the ranks
        out = batched_section(rank=rank, world=world, dist=dist, device=dev)
        if rank == 0:
            extra["batched"] = out
    if rank == 0 and not args.no_table1:
        extra["table1"] = table1_section()
    if rank == 0 and not args.no_order:
        extra["particle_order"] = order_section()
    if rank == 0 and not args.no_packing:
        extra["packing"] = packing_section()
    if rank == 0 and not args.no_fire:
        extra["fire"] = fire_section()
    if rank == 0 and not args.no_nhc:
        extra["nvt_nose_hoover"] = nhc_section()
    if rank == 0 and not args.no_flock:
        extra["flocking"] = flock_section()
    if rank == 0 and not args.no_gnn:
        extra["gnn_nvt"] = gnn_section()
    if rank == 0 and not args.no_alu:
        extra["alu_rooflines"] = alu_rooflines_section()
    if rank == 0 and not args.no_tiles_job and not tiles and args.workload == "lj256k":
        extra["tiles_engine_job"] = tiles_section()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"lj_fcc40_N{c.N}" if c.N == 256000 else f"lj_sc16_N{c.N}", "N": c.N,
                       "md_steps_per_step": md_steps, "density": 0.84, "T": 1.0, "r_cut": c.r_cut, "skin": c.skin,
                       "dt": c.dt, "neighbor_cap": nl.cap, "rebuilds_per_step": builds / args.steps,
                       "max_energy_drift_per_particle": drift, "energy_vs_oracle": drift_vs_oracle,
                       "l2": "flushed between bench steps",
                       "parallelism": f"replicas{world}", "pair_tpp": args.tpp or 4,
                       "neighbor_rows": ("16-bit tile-local" if tiles else
                                         "int32 + 16-bit local" if args.local_rows else "int32"),
                       "engine": "tiles (MD_NBR_TILES)" if tiles else "int32 rows",
                       "kick_drift": ("fused into the force kernel" if (tiles or (args.nve_fusion and not args.local_rows))
                                      else "separate kernel"),
                       "particle_order": ("re-sorted into half-cell order at every rebuild (tile engine)" if tiles else
                                          "Z-order sort at the start of each job, inside the timed region"
                                          if args.sort else "as generated (FCC lattice order)"),
                       "loop": "host launches" if args.no_graph else "one CUDA graph (device WHILE/IF)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": kname,
                         "bytes_per_particle": bytes_per_particle, "kernel_ms": kt * 1e3,
                         "peak_source": peak_src},
            "cpu_baseline": cpu_baseline,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clk,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
