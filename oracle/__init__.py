"""FP64 CPU oracle for the molecular-dynamics hot path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does, and the
oracle never imports the product package: the two share no code.  Inputs
come from ``workloads`` (seeded generators that hold no method arithmetic).

The C part (``md_oracle.c``) holds the plain FP64 definitions; ``bp.py``
holds the Behler-Parrinello descriptor / MLP oracle in plain PyTorch CPU
FP64 ops.  Each function cites the passage of the paper it follows.

Parity unpinned: none of the functions here is unpinned; see tests/test_oracle_*.py
for what pins each one.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_LIB = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_up = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = C.CDLL(path)
        L.or_neighbor_list.restype = C.c_long
        L.or_neighbor_list.argtypes = [C.c_int, C.c_int, _dp, _dp, C.c_double, C.c_int, C.c_int, C.c_int, _ip, _ip]
        L.or_lj_pair.restype = C.c_double
        L.or_lj_pair.argtypes = [C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double)]
        L.or_lj.restype = C.c_double
        L.or_lj.argtypes = [C.c_int, _dp, _dp, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, _dp, _dp]
        L.or_soft.restype = C.c_double
        L.or_soft.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, C.c_double, C.c_double, _dp, _dp]
        L.or_sw.restype = C.c_double
        L.or_sw.argtypes = [C.c_int, _dp, _dp, _dp, _dp, _dp]
        L.or_sw_phi2.restype = C.c_double
        L.or_sw_phi2.argtypes = [_dp, C.c_double, C.POINTER(C.c_double)]
        L.or_nve.restype = None
        L.or_nve.argtypes = [C.c_int, C.c_int, _dp, _dp, C.c_void_p, _dp, C.c_int, _dp, C.c_double, C.c_double,
                             C.c_int, _dp, _dp]
        L.or_gd.restype = None
        L.or_gd.argtypes = [C.c_int, C.c_int, _dp, C.c_void_p, _dp, C.c_int, _dp, C.c_double, C.c_int, _dp]
        L.or_flock_grad.restype = C.c_double
        L.or_flock_grad.argtypes = [C.c_int, _dp, _dp, _dp, _dp, C.c_int, C.c_void_p, C.c_int, C.c_void_p, _dp, _dp,
                                    C.c_void_p, _dp]
        L.or_flock_run.restype = None
        L.or_flock_run.argtypes = [C.c_int, _dp, _dp, _dp, _dp, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_double,
                                   C.c_int, _dp]
        L.or_nhc.restype = None
        L.or_nhc.argtypes = [C.c_int, C.c_int, _dp, _dp, C.c_void_p, _dp, C.c_int, _dp, C.c_double, C.c_double,
                             C.c_double, C.c_double, C.c_int, C.c_int, _dp, _dp, _dp, _dp]
        L.or_fire.restype = None
        L.or_fire.argtypes = [C.c_int, C.c_int, _dp, C.c_void_p, _dp, C.c_int, _dp, _dp, C.c_int, C.c_void_p,
                              C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_philox4x32_10.restype = None
        L.or_philox4x32_10.argtypes = [_up, _up, _up]
        L.or_normal3.restype = None
        L.or_normal3.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint64, _dp]
        L.or_langevin.restype = None
        L.or_langevin.argtypes = [C.c_int, _dp, _dp, _dp, C.c_int, _dp, C.c_double, C.c_double, C.c_double,
                                  C.c_double, C.c_uint64, C.c_int, C.c_int, _dp, _dp]
        L.or_packing_box.restype = C.c_double
        L.or_packing_box.argtypes = [C.c_int, C.c_double, C.c_double]
        L.or_gd_adjoint.restype = C.c_double
        L.or_gd_adjoint.argtypes = [C.c_int, _dp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                    C.c_int, C.POINTER(C.c_double), _dp]
        L.or_gd_final_energy.restype = C.c_double
        L.or_gd_final_energy.argtypes = [C.c_int, _dp, C.c_double, C.c_double, C.c_double, C.c_double,
                                         C.c_double, C.c_int]
        L.or_num_threads.restype = C.c_int
        L.or_set_num_threads.argtypes = [C.c_int]
        _LIB = L
    return _LIB


# ----------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------
def _pos(r, dim=3) -> np.ndarray:
    """[N, >=dim] array (float32 or float64) -> contiguous double [N, 3]."""
    r = np.asarray(r)
    out = np.zeros((r.shape[0], 3), dtype=np.float64)
    out[:, :dim] = r[:, :dim]
    return out


def _box(L, dim=3) -> np.ndarray:
    if np.isscalar(L):
        b = [float(L)] * dim
    else:
        b = [float(x) for x in L]
    while len(b) < 3:
        b.append(1.0)
    return np.asarray(b, dtype=np.float64)


def num_threads() -> int:
    return lib().or_num_threads()


def set_num_threads(n: int) -> None:
    lib().or_set_num_threads(int(n))


# Stillinger-Weber silicon constants (Stillinger & Weber 1985), eV and Angstrom:
# eps, sigma, a, lambda, gamma, A, B, p, q, cos(theta_0)
SW_SI = np.array([2.1683, 2.0951, 1.80, 21.0, 1.20, 7.049556277, 0.6022245584, 4.0, 0.0, -1.0 / 3.0])
SW_MASS_AMU = 28.0855
AMU_A2_FS2_EV = 103.6427


# ----------------------------------------------------------------------------
# Spaces / neighbor sets (Sec. 3.2.1, 3.2.3)
# ----------------------------------------------------------------------------
def neighbor_list(r, L, r_list, dim=3, cap=None, fp32_decision=True, use_cells=True):
    """Full neighbor list {j != i : r_ij < r_list} as padded sorted rows.

    Returns (cnt [N] int32, nbr [N, cap] int32 padded with N).  With
    ``fp32_decision`` the membership test is the FP32 formula of the kernels.
    """
    x = _pos(r, dim)
    N = x.shape[0]
    if cap is None:
        cnt = np.zeros(N, np.int32)
        nb = np.zeros((N, 1), np.int32)
        lib().or_neighbor_list(N, dim, x, _box(L, dim), float(r_list), int(fp32_decision), int(use_cells), 1,
                               cnt, nb)
        cap = max(1, int(cnt.max()) if N else 1)
    cnt = np.zeros(N, np.int32)
    nb = np.zeros((N, cap), np.int32)
    lib().or_neighbor_list(N, dim, x, _box(L, dim), float(r_list), int(fp32_decision), int(use_cells), int(cap),
                           cnt, nb)
    return cnt, nb


# ----------------------------------------------------------------------------
# Energies and forces (Sec. 3.2.2, 3.3.2)
# ----------------------------------------------------------------------------
def lj_pair(r, eps=1.0, sigma=1.0):
    du = C.c_double()
    u = lib().or_lj_pair(float(r), eps, sigma, C.byref(du))
    return u, du.value


def lj(r, L, eps=1.0, sigma=1.0, r_cut=2.5, shifted=True, use_cells=True):
    """(U, F [N,3], e [N]) for the (shifted) LJ fluid."""
    x = _pos(r)
    N = x.shape[0]
    f = np.zeros((N, 3))
    e = np.zeros(N)
    U = lib().or_lj(N, x, _box(L), eps, sigma, r_cut, int(shifted), int(use_cells), f, e)
    return U, f, e


def soft(r, diam, L, dim=2, eps=1.0, alpha=2.0):
    """(U, F [N,3], e [N]) for soft spheres with sigma_ij = (d_i + d_j)/2."""
    x = _pos(r, dim)
    N = x.shape[0]
    f = np.zeros((N, 3))
    e = np.zeros(N)
    U = lib().or_soft(N, dim, x, np.ascontiguousarray(diam, np.float64), _box(L, dim), eps, alpha, f, e)
    return U, f, e


def sw(r, L, params=SW_SI):
    """(U, F [N,3], e [N]) for Stillinger-Weber."""
    x = _pos(r)
    N = x.shape[0]
    f = np.zeros((N, 3))
    e = np.zeros(N)
    U = lib().or_sw(N, x, _box(L), np.ascontiguousarray(params, np.float64), f, e)
    return U, f, e


def sw_phi2(r, params=SW_SI):
    d = C.c_double()
    v = lib().or_sw_phi2(np.ascontiguousarray(params, np.float64), float(r), C.byref(d))
    return v, d.value


_POT = {"lj": 0, "soft": 1, "sw": 2}


def _pp(pot, **kw):
    if pot == "lj":
        return np.array([kw.get("eps", 1.0), kw.get("sigma", 1.0), kw.get("r_cut", 2.5),
                         1.0 if kw.get("shifted", True) else 0.0])
    if pot == "soft":
        return np.array([kw.get("eps", 1.0), kw.get("alpha", 2.0)])
    return np.ascontiguousarray(kw.get("params", SW_SI), np.float64)


# ----------------------------------------------------------------------------
# Dynamics (Sec. 3.3.1)
# ----------------------------------------------------------------------------
def nve(r, v, L, pot="lj", mass=1.0, dt=0.005, nsteps=10, dim=3, diam=None, **kw):
    """Velocity-Verlet NVE.  Returns (r, v, PE[nsteps+1], KE[nsteps+1])."""
    x = _pos(r, dim)
    vv = _pos(v, dim)
    N = x.shape[0]
    PE = np.zeros(nsteps + 1)
    KE = np.zeros(nsteps + 1)
    dptr = None
    if diam is not None:
        diam = np.ascontiguousarray(diam, np.float64)
        dptr = diam.ctypes.data
    lib().or_nve(N, dim, x, vv, dptr, _box(L, dim), _POT[pot], _pp(pot, **kw), mass, dt, nsteps, PE, KE)
    return x, vv, PE, KE


def gd(r, L, pot="soft", eta=0.05, nsteps=10, dim=2, diam=None, **kw):
    """Gradient descent r <- r + eta F.  Returns (r, E[nsteps+1])."""
    x = _pos(r, dim)
    N = x.shape[0]
    E = np.zeros(nsteps + 1)
    dptr = None
    if diam is not None:
        diam = np.ascontiguousarray(diam, np.float64)
        dptr = diam.ctypes.data
    lib().or_gd(N, dim, x, dptr, _box(L, dim), _POT[pot], _pp(pot, **kw), eta, nsteps, E)
    return x, E


def nhc(r, v, L, pot="lj", mass=1.0, dt=0.005, kT=1.0, tau=None, M=3, nsteps=10, dim=3, diam=None, therm=None,
        **kw):
    """Nose-Hoover chain NVT (tau defaults to 100 dt).  Returns (r, v, PE,
    KE, H' [nsteps+1 each], thermostat state (xi[M], w[M]))."""
    x = _pos(r, dim)
    vv = _pos(v, dim)
    N = x.shape[0]
    PE = np.zeros(nsteps + 1)
    KE = np.zeros(nsteps + 1)
    H = np.zeros(nsteps + 1)
    th = np.zeros(2 * M) if therm is None else np.ascontiguousarray(np.concatenate(therm), np.float64).copy()
    dptr = None
    if diam is not None:
        diam = np.ascontiguousarray(diam, np.float64)
        dptr = diam.ctypes.data
    tau = 100.0 * dt if tau is None else tau
    lib().or_nhc(N, dim, x, vv, dptr, _box(L, dim), _POT[pot], _pp(pot, **kw), mass, dt, kT, tau, M, nsteps, th,
                 PE, KE, H)
    return x, vv, PE, KE, H, (th[:M].copy(), th[M:].copy())


# Flocking parameters: J_align, R_align, J_avoid, R_avoid, J_cohesion,
# R_cohesion, J_obstacle, cutoff exponent, speed; predators: J_flee, R_flee
# (boids fleeing), J_chase, R_chase (predators chasing), predator speed
FLOCK_DEFAULTS = dict(J_align=1.0, R_align=45.0, J_avoid=25.0, R_avoid=30.0, J_cohesion=0.05, R_cohesion=40.0,
                      J_obstacle=10.0, alpha=2.0, speed=1.0, J_flee=10.0, R_flee=60.0, J_chase=0.2,
                      R_chase=150.0, predator_speed=0.85, sprint_period=50, sprint_steps=10, sprint_factor=2.0)
_FLOCK_KEYS = ("J_align", "R_align", "J_avoid", "R_avoid", "J_cohesion", "R_cohesion", "J_obstacle", "alpha", "speed",
               "J_flee", "R_flee", "J_chase", "R_chase", "predator_speed", "sprint_period", "sprint_steps",
               "sprint_factor")


def _flock_prm(params):
    fp = dict(FLOCK_DEFAULTS, **(params or {}))
    return np.array([fp[k] for k in _FLOCK_KEYS], np.float64)


def _rows3(x):
    if x is None or len(x) == 0:
        return 0, None, None
    o = np.ascontiguousarray(x, np.float64).reshape(-1, 3).copy()
    return o.shape[0], o, o.ctypes.data


def flock_grad(R, theta, L, params=None, obstacles=None, predators=None):
    """(E, dE/dR [N,2], dE/dtheta [N], dE/d(predator x, y, theta) [P,3],
    (E_align, E_avoid, E_cohesion, E_obstacle, E_flee, E_chase))."""
    R = np.ascontiguousarray(np.asarray(R, np.float64)[:, :2])
    th = np.ascontiguousarray(theta, np.float64)
    N = R.shape[0]
    gR = np.zeros((N, 2))
    gth = np.zeros(N)
    parts = np.zeros(6)
    n_obs, o, optr = _rows3(obstacles)
    n_p, pr, pptr = _rows3(predators)
    gP = np.zeros((max(n_p, 1), 3))
    E = lib().or_flock_grad(N, R, th, _box(L, 2), _flock_prm(params), n_obs, optr, n_p, pptr, gR, gth,
                            gP.ctypes.data, parts)
    return E, gR, gth, gP[:n_p], tuple(parts)


def flock_run(R, theta, L, dt=0.1, nsteps=10, params=None, obstacles=None, predators=None):
    """Forward-Euler flocking.  Returns (R [N,2], theta [N], predators [P,3],
    E[nsteps+1])."""
    R = np.ascontiguousarray(np.asarray(R, np.float64)[:, :2]).copy()
    th = np.ascontiguousarray(theta, np.float64).copy()
    E = np.zeros(nsteps + 1)
    n_obs, o, optr = _rows3(obstacles)
    n_p, pr, pptr = _rows3(predators)
    lib().or_flock_run(R.shape[0], R, th, _box(L, 2), _flock_prm(params), n_obs, optr, n_p, pptr, dt, nsteps, E)
    return R, th, (pr if pr is not None else np.zeros((0, 3))), E


# FIRE parameters (Bitzek et al. 2006 recommendations; dt_max = 4 dt_start)
FIRE_DEFAULTS = dict(dt_start=0.1, dt_max=0.4, f_inc=1.1, f_dec=0.5, alpha_start=0.1, f_alpha=0.99, n_min=5)


def fire(r, L, pot="soft", nsteps=10, dim=2, diam=None, fire_params=None, **kw):
    """FIRE minimisation from rest.  Returns (r, v, E[nsteps+1], dt[nsteps],
    (dt, alpha, npos) at the end)."""
    fp = dict(FIRE_DEFAULTS, **(fire_params or {}))
    prm = np.array([fp["dt_start"], fp["dt_max"], fp["f_inc"], fp["f_dec"], fp["alpha_start"], fp["f_alpha"],
                    fp["n_min"]], np.float64)
    x = _pos(r, dim)
    N = x.shape[0]
    E = np.zeros(nsteps + 1)
    dts = np.zeros(max(nsteps, 1))
    v = np.zeros((N, 3))
    st = np.zeros(3)
    dptr = None
    if diam is not None:
        diam = np.ascontiguousarray(diam, np.float64)
        dptr = diam.ctypes.data
    lib().or_fire(N, dim, x, dptr, _box(L, dim), _POT[pot], _pp(pot, **kw), prm, nsteps, E.ctypes.data,
                  dts.ctypes.data, v.ctypes.data, st.ctypes.data)
    return x, v, E, dts[:nsteps], (float(st[0]), float(st[1]), int(st[2]))


def philox4x32_10(ctr, key):
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def normal3(i, step, stream, seed):
    z = np.zeros(3)
    lib().or_normal3(i, step, stream, seed, z)
    return z


def langevin(r, v, L, pot="sw", mass=1.0, dt=1.0, gamma=0.01, kT=0.0, seed=0, step0=0, nsteps=10, **kw):
    """BAOAB Langevin.  Returns (r, v, PE[nsteps], KE[nsteps])."""
    x = _pos(r)
    vv = _pos(v)
    N = x.shape[0]
    PE = np.zeros(max(nsteps, 1))
    KE = np.zeros(max(nsteps, 1))
    lib().or_langevin(N, x, vv, _box(L), _POT[pot], _pp(pot, **kw), mass, dt, gamma, kT, seed, step0, nsteps,
                      PE, KE)
    return x, vv, PE[:nsteps], KE[:nsteps]


# ----------------------------------------------------------------------------
# Differentiation through minimisation (Sec. 4.2, App. A)
# ----------------------------------------------------------------------------
def packing_box(N, D, phi):
    return lib().or_packing_box(N, D, phi)


def gd_adjoint(s0, D, phi=0.9, eps=1.0, alpha=2.0, eta=0.05, T=100):
    """Reverse-mode dE_final/dD.  Returns (E_final, dE/dD, r_T [N,3])."""
    s0 = np.ascontiguousarray(s0, np.float64)
    N = s0.shape[0]
    g = C.c_double()
    rT = np.zeros((N, 3))
    E = lib().or_gd_adjoint(N, s0, D, phi, eps, alpha, eta, T, C.byref(g), rT)
    return E, g.value, rT


def gd_final_energy(s0, D, phi=0.9, eps=1.0, alpha=2.0, eta=0.05, T=100):
    s0 = np.ascontiguousarray(s0, np.float64)
    return lib().or_gd_final_energy(s0.shape[0], s0, D, phi, eps, alpha, eta, T)
