"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws and lays out inputs (lattices, jitter, velocities,
random disk packings, replica plans). It holds none of the method's
arithmetic: no displacement, energy, force or integration code lives here.
Both the FP64 oracle (``oracle/``) and the CUDA path read their inputs from
these generators, so the two sides see bit-identical starting data.

Conventions shared with every consumer:
  * positions / velocities are float32 arrays of shape [N, 4] (x, y, z, w);
    in 2-D the z column is 0.  ``w`` of a position holds the particle
    diameter for soft spheres and 0 otherwise; ``w`` of a velocity is 0;
  * box lengths are returned as Python floats that are exactly
    representable in float32, so that the FP32 kernels and the FP64 oracle
    integrate in exactly the same box;
  * all randomness comes from ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "f32", "box_for_density", "sc_lattice", "fcc_lattice", "diamond_lattice",
    "jitter_wrap", "thermal_velocities", "LJFluid", "lj_fluid",
    "Packing2D", "packing_2d", "packing_box", "SWSilicon", "sw_silicon", "Flock", "flock",
    "ReplicaSpec", "replica_plan", "replica_initial", "uniform_box_positions",
]


def f32(x: float) -> float:
    """Round a double to the nearest float32 value and return it as a double."""
    return float(np.float32(x))


def box_for_density(n: int, rho: float, dim: int = 3) -> float:
    """Cubic (square) box edge for ``n`` particles at number density ``rho``,
    rounded to float32 (the box both sides use)."""
    return f32((n / rho) ** (1.0 / dim))


def _to4(r: np.ndarray) -> np.ndarray:
    out = np.zeros((r.shape[0], 4), dtype=np.float32)
    out[:, : r.shape[1]] = r
    return out


def sc_lattice(n_side: int, L: float, dim: int = 3) -> np.ndarray:
    """Simple-cubic (square) lattice, n_side**dim sites at (k + 1/2) L / n_side."""
    a = L / n_side
    g = (np.arange(n_side, dtype=np.float64) + 0.5) * a
    mesh = np.meshgrid(*([g] * dim), indexing="ij")
    return np.stack([m.reshape(-1) for m in mesh], axis=1)


def fcc_lattice(n_side: int, L: float) -> np.ndarray:
    """Face-centred cubic lattice of 4 n_side^3 sites in a cube of edge L."""
    a = L / n_side
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]]) + 0.25
    g = np.arange(n_side, dtype=np.float64)
    cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    return ((cells[:, None, :] + basis[None, :, :]) * a).reshape(-1, 3)


def diamond_lattice(n_side: int, a: float) -> np.ndarray:
    """Diamond-cubic lattice (8 n_side^3 sites) with cubic lattice constant a."""
    fcc = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    basis = np.concatenate([fcc, fcc + 0.25]) + 0.125
    g = np.arange(n_side, dtype=np.float64)
    cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    return ((cells[:, None, :] + basis[None, :, :]) * a).reshape(-1, 3)


def jitter_wrap(r: np.ndarray, L: float, amp: float, rng: np.random.Generator) -> np.ndarray:
    """Add uniform noise in [-amp, amp) per component, fold into [0, L) and
    round to float32 (a value that rounds up to L is folded to 0)."""
    r = r + rng.uniform(-amp, amp, size=r.shape)
    r = np.mod(r, L).astype(np.float32)
    r[r >= np.float32(L)] = 0.0
    r[r < 0] = 0.0
    return r


def thermal_velocities(n: int, dim: int, T: float, mass: float,
                       rng: np.random.Generator) -> np.ndarray:
    """Gaussian velocities at temperature T with zero net momentum, rescaled
    so the kinetic energy is exactly (dim*n - dim) T / 2 (k_B = 1)."""
    v = rng.normal(0.0, math.sqrt(T / mass), size=(n, dim))
    v -= v.mean(axis=0, keepdims=True)
    ke = 0.5 * mass * float((v * v).sum())
    target = 0.5 * (dim * n - dim) * T
    v *= math.sqrt(target / ke)
    return v.astype(np.float32)


# --------------------------------------------------------------------------
# Lennard-Jones fluid (Table 1 benchmark shape: N particles, cutoff, skin)
# --------------------------------------------------------------------------
@dataclass
class LJFluid:
    N: int
    L: float
    r: np.ndarray           # [N,4] float32
    v: np.ndarray           # [N,4] float32
    eps: float = 1.0
    sigma: float = 1.0
    r_cut: float = 2.5
    skin: float = 0.3
    dt: float = 0.005
    mass: float = 1.0
    steps: int = 100
    name: str = ""


def lj_fluid(lattice: str = "sc", n_side: int = 16, rho: float = 0.84, T: float = 1.0,
             jitter: float = 0.05, seed: int = 0, steps: int = 100) -> LJFluid:
    """3-D LJ fluid: a jittered lattice at density ``rho`` and T velocities.

    ``lattice='sc'`` with n_side=16 gives N = 4096;
    ``lattice='fcc'`` with n_side=40 gives N = 256,000.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n = n_side ** 3 if lattice == "sc" else 4 * n_side ** 3
    L = box_for_density(n, rho, 3)
    sites = sc_lattice(n_side, L, 3) if lattice == "sc" else fcc_lattice(n_side, L)
    r = _to4(jitter_wrap(sites, L, jitter, rng))
    v = _to4(thermal_velocities(n, 3, T, 1.0, rng))
    return LJFluid(N=n, L=L, r=r, v=v, steps=steps, name=f"lj_{lattice}{n_side}_N{n}")


def lj_small(seed: int = 0) -> LJFluid:
    """N = 4,096 LJ fluid (simple-cubic 16^3 start), 100 steps."""
    return lj_fluid("sc", 16, seed=seed, steps=100)


def lj_large(seed: int = 0) -> LJFluid:
    """N = 256,000 LJ fluid (FCC 4*40^3 start), 1,000 steps."""
    return lj_fluid("fcc", 40, seed=seed, steps=1000)


# --------------------------------------------------------------------------
# 2-D bidisperse soft-sphere packing (Sec. 4.2)
# --------------------------------------------------------------------------
def packing_box(N: int, D: float, phi: float) -> float:
    """Square box edge keeping packing fraction ``phi`` for N/2 disks of
    diameter D and N/2 of diameter 1 (FP64; the packing keeps FP64 L(D))."""
    return math.sqrt((N // 2) * math.pi * (D * D + 1.0) / 4.0 / phi)


@dataclass
class Packing2D:
    N: int
    D: float
    phi: float
    s0: np.ndarray          # [N,2] float64 fractional coordinates in [0,1)
    diam: np.ndarray        # [N] float64: D for the first N/2, 1 for the rest
    step: float = 0.05
    steps: int = 2000
    eps: float = 1.0
    alpha: float = 2.0
    skin: float = 0.3


def packing_2d(N: int = 1024, D: float = 1.2, phi: float = 0.90, seed: int = 0,
               steps: int = 2000, step: float = 0.05) -> Packing2D:
    rng = np.random.Generator(np.random.PCG64(seed))
    s0 = rng.uniform(0.0, 1.0, size=(N, 2))
    diam = np.ones(N)
    diam[: N // 2] = D
    return Packing2D(N=N, D=D, phi=phi, s0=s0, diam=diam, steps=steps, step=step)


# --------------------------------------------------------------------------
# Stillinger-Weber silicon (learned-potential workload)
# --------------------------------------------------------------------------
@dataclass
class SWSilicon:
    N: int
    L: float
    r: np.ndarray
    v: np.ndarray
    a: float
    T_K: float
    mass_amu: float = 28.0855


KB_EV = 8.617333262e-5          # Boltzmann constant, eV / K
AMU_A2_FS2_TO_EV = 103.6427     # 1 amu A^2 fs^-2 = 103.6427 eV


def sw_silicon(n_side: int = 4, a: float = 5.431, T_K: float = 1000.0, seed: int = 0,
               jitter: float = 0.0) -> SWSilicon:
    """Diamond-cubic Si, 8 n_side^3 atoms, velocities at T_K in A/fs."""
    rng = np.random.Generator(np.random.PCG64(seed))
    L = f32(n_side * a)
    sites = diamond_lattice(n_side, a)
    r = _to4(jitter_wrap(sites, L, jitter, rng) if jitter > 0 else
             np.mod(sites, L).astype(np.float32))
    n = sites.shape[0]
    # kT / m in (A/fs)^2: (eV) / (amu) -> divide by 103.6427
    kT_over_m = KB_EV * T_K / 28.0855 / AMU_A2_FS2_TO_EV
    v = thermal_velocities(n, 3, kT_over_m, 1.0, rng) if T_K > 0 else np.zeros((n, 3), np.float32)
    return SWSilicon(N=n, L=L, r=r, v=_to4(v), a=a, T_K=T_K)


# --------------------------------------------------------------------------
# Batched replicas (vmap over independent systems, Sec. 4.2)
# --------------------------------------------------------------------------
@dataclass
class ReplicaSpec:
    kind: str               # "lj" or "soft"
    N: int
    rho: float
    L: float
    seed: int
    dt: float
    extras: dict = field(default_factory=dict)


def replica_plan(R: int = 512, n_max: int = 8192, seed: int = 0,
                 lj_rlist: float = 2.8, soft_rlist: float = 1.7) -> list[ReplicaSpec]:
    """Half LJ, half 3-D soft-sphere replicas with log-uniform N and uniform
    density in [0.7, 0.95].  N has a lower clamp so that every box holds the
    interaction range twice over (minimum image stays valid)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(R):
        kind = "lj" if k < R // 2 else "soft"
        rho = float(rng.uniform(0.7, 0.95))
        rl = lj_rlist if kind == "lj" else soft_rlist
        n_min = max(64, int(math.ceil(rho * (2.0 * rl) ** 3)) + 1)
        N = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        N = max(N, n_min)
        out.append(ReplicaSpec(kind=kind, N=N, rho=rho, L=box_for_density(N, rho, 3),
                               seed=seed * 100003 + k, dt=0.005 if kind == "lj" else 0.01))
    return out


def replica_initial(spec: ReplicaSpec, T: float = 1.0):
    """Starting state of one replica: LJ replicas take N sites, chosen
    uniformly at random, of the smallest FCC lattice (4 m^3 sites, m =
    ceil((N/4)^(1/3))) filling the box, jittered by 0.05 sigma (sites stay at
    least about 1 sigma apart at the densities used); soft-sphere replicas are uniform random with diameters 1.0 / 1.4 (50/50)
    in the w column (they are meant to be relaxed before dynamics).  Gaussian
    velocities at T with zero net momentum.  Returns (r [N,4], v [N,4])."""
    rng = np.random.Generator(np.random.PCG64(spec.seed))
    L = spec.L
    if spec.kind == "lj":
        m = int(math.ceil((spec.N / 4.0) ** (1.0 / 3.0) - 1e-9))
        sites = fcc_lattice(m, L)
        keep = np.sort(rng.choice(sites.shape[0], size=spec.N, replace=False))
        r = _to4(jitter_wrap(sites[keep], L, 0.05, rng))
    else:
        r = _to4(uniform_box_positions(spec.N, L, 3, rng))
        d = np.where(np.arange(spec.N) % 2 == 0, 1.0, 1.4).astype(np.float32)
        r[:, 3] = d
    v = _to4(thermal_velocities(spec.N, 3, T, 1.0, rng))
    return r, v


# --------------------------------------------------------------------------
# Flocking (Sec. 4.3): boids in a periodic square
# --------------------------------------------------------------------------
@dataclass
class Flock:
    N: int
    L: float
    R: np.ndarray           # [N, 2] float32 positions
    theta: np.ndarray       # [N] float32 headings
    obstacles: np.ndarray   # [n_obs, 3] float32 (x, y, radius)
    predators: np.ndarray = None   # [n_pred, 3] float32 (x, y, theta)


def flock(N: int = 2000, neighbours: float = 20.0, R_align: float = 45.0, n_obs: int = 4,
          obstacle_radius: float = 60.0, seed: int = 0, n_pred: int = 0) -> Flock:
    """Uniform positions and headings; the box edge gives about `neighbours`
    boids within R_align of each boid; disk obstacles at uniform centres."""
    rng = np.random.Generator(np.random.PCG64(seed))
    L = f32(math.sqrt(N * math.pi * R_align * R_align / neighbours))
    R = rng.uniform(0.0, L, size=(N, 2)).astype(np.float32)
    R[R >= L] = 0.0
    theta = rng.uniform(-math.pi, math.pi, size=N).astype(np.float32)
    obs = np.zeros((n_obs, 3), np.float32)
    obs[:, :2] = rng.uniform(0.0, L, size=(n_obs, 2))
    obs[:, 2] = obstacle_radius
    pred = np.zeros((n_pred, 3), np.float32)
    pred[:, :2] = rng.uniform(0.0, L, size=(n_pred, 2))
    pred[:, 2] = rng.uniform(-math.pi, math.pi, size=n_pred)
    return Flock(N=N, L=L, R=R, theta=theta, obstacles=obs, predators=pred)


def uniform_box_positions(N: int, L: float, dim: int, rng: np.random.Generator) -> np.ndarray:
    """N uniform random positions in [0, L)^dim as float32."""
    r = np.mod(rng.uniform(0.0, L, size=(N, dim)), L).astype(np.float32)
    r[r >= np.float32(L)] = 0.0
    return r


# --------------------------------------------------------------------------
# Graph-network potential weights (Sec. 3.2.4 / 4.1): random, seeded
# --------------------------------------------------------------------------
def gnn_param_count(H: int, T: int) -> int:
    return 5 * H + T * (5 * H * H + 2 * H) + H * H + 2 * H + 1


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to the nearest BF16-representable value (ties to
    even), returned as FP32."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def gnn_params(H: int = 64, T: int = 2, seed: int = 0, out_scale: float = 0.1,
               bias_scale: float = 0.1, bf16: bool = False) -> np.ndarray:
    """Flat FP32 weights in the library's layout (W_enc, b_enc, u, T x {A, a,
    B, b}, D, d, w, c): matrices N(0, 1/fan_in), biases and u
    N(0, bias_scale^2), the read-out w N(0, out_scale^2 / H) so that
    energies are of order out_scale per atom."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = lambda n, s: rng.normal(0.0, s, size=n)
    parts = [g(3 * H, 1.0 / math.sqrt(3.0)), g(H, bias_scale), g(H, 1.0)]
    for _ in range(T):
        parts += [g(3 * H * H, 1.0 / math.sqrt(3 * H)), g(H, bias_scale), g(2 * H * H, 1.0 / math.sqrt(2 * H)),
                  g(H, bias_scale)]
    parts += [g(H * H, 1.0 / math.sqrt(H)), g(H, bias_scale), g(H, out_scale / math.sqrt(H)), np.zeros(1)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.shape[0] == gnn_param_count(H, T)
    return bf16_round(p) if bf16 else p
