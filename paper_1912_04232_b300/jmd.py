"""Thin ctypes binding over libjmd (include/jmd.h).

Argument marshalling only: every step of the hot path runs in the CUDA
kernels of libjmd.so.  torch tensors serve as device storage; the binding
passes their data pointers and the current CUDA stream.  There is no CPU
fallback: if libjmd.so is missing the import fails, and every call checks
that its tensors live on a CUDA device.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libjmd.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"libjmd.so not found at {LIB_PATH}: build it with `python -m paper_1912_04232_b300.build` "
        "(nvcc, sm_103a). There is no fallback implementation.")

_lib = C.CDLL(LIB_PATH)

# status bits (md_status)
MD_OK = 0
MD_ERR_INVALID = 1
MD_ERR_BOX_TOO_SMALL = 2
MD_ERR_NBR_OVERFLOW = 4
MD_ERR_NONFINITE = 8
MD_ERR_TIMEOUT = 16
MD_ERR_BOUNDS = 32
MD_ERR_CUDA = 64

MD_LJ, MD_SOFT_SPHERE, MD_SW, MD_BP, MD_GNN = 0, 1, 2, 3, 4
MD_NBR_CANONICAL = 1
MD_NBR_LOCAL_ROWS = 2
MD_NBR_TILES = 4

STATUS_NAMES = {MD_ERR_INVALID: "INVALID", MD_ERR_BOX_TOO_SMALL: "BOX_TOO_SMALL",
                MD_ERR_NBR_OVERFLOW: "NBR_OVERFLOW", MD_ERR_NONFINITE: "NONFINITE",
                MD_ERR_TIMEOUT: "TIMEOUT", MD_ERR_BOUNDS: "BOUNDS", MD_ERR_CUDA: "CUDA"}


class MDError(RuntimeError):
    def __init__(self, code: int, where: str):
        names = [n for b, n in STATUS_NAMES.items() if code & b] or [str(code)]
        super().__init__(f"{where}: md_status {code} ({'|'.join(names)})")
        self.code = code


class md_space(C.Structure):
    _fields_ = [("dim", C.c_int), ("L", C.c_float * 3), ("Linv", C.c_float * 3), ("L64", C.c_double * 3)]


class md_nbr(C.Structure):
    _fields_ = [("dim", C.c_int), ("N", C.c_int), ("cap", C.c_int), ("ncell", C.c_int * 3),
                ("ncell_total", C.c_int), ("r_cut", C.c_float), ("skin", C.c_float), ("r_list", C.c_float),
                ("r_list2", C.c_float), ("half_skin2", C.c_float), ("cell_scale", C.c_float * 3),
                ("ws_bytes", C.c_size_t), ("nbr", C.c_void_p), ("cnt", C.c_void_p), ("rref", C.c_void_p),
                ("ws", C.c_void_p), ("flags", C.c_int)]


class md_pot(C.Structure):
    _fields_ = [("kind", C.c_int), ("eps", C.c_float), ("sigma", C.c_float), ("r_cut", C.c_float),
                ("e_shift", C.c_float), ("alpha", C.c_float), ("sw", C.c_float * 10), ("model", C.c_void_p)]


class md_bp_model(C.Structure):
    _fields_ = [("params", C.c_void_p), ("norm", C.c_void_p), ("G", C.c_void_p), ("dEdG", C.c_void_p),
                ("Ei", C.c_void_p), ("sys_n", C.c_int), ("lists", C.c_void_p)]


class md_gnn_model(C.Structure):
    _fields_ = [("params", C.c_void_p), ("H", C.c_int), ("T", C.c_int), ("r_cut", C.c_float), ("ws", C.c_void_p),
                ("ws_bytes", C.c_size_t), ("sys_n", C.c_int)]


class md_fire_params(C.Structure):
    _fields_ = [("dt_start", C.c_float), ("dt_max", C.c_float), ("f_inc", C.c_float), ("f_dec", C.c_float),
                ("alpha_start", C.c_float), ("f_alpha", C.c_float), ("n_min", C.c_int)]


def fire_params(dt_start=0.1, dt_max=0.4, f_inc=1.1, f_dec=0.5, alpha_start=0.1, f_alpha=0.99, n_min=5):
    """FIRE parameters (Bitzek et al. 2006 recommendations, dt_max = 4 dt_start)."""
    return md_fire_params(dt_start, dt_max, f_inc, f_dec, alpha_start, f_alpha, n_min)


class md_flock_params(C.Structure):
    _fields_ = [(n, C.c_float) for n in ("J_align", "R_align", "J_avoid", "R_avoid", "J_cohesion", "R_cohesion",
                                         "J_obstacle", "alpha", "speed", "J_flee", "R_flee", "J_chase", "R_chase",
                                         "predator_speed")] + [("sprint_period", C.c_int), ("sprint_steps", C.c_int),
                                                               ("sprint_factor", C.c_float)]


def flock_params(J_align=1.0, R_align=45.0, J_avoid=25.0, R_avoid=30.0, J_cohesion=0.05, R_cohesion=40.0,
                 J_obstacle=10.0, alpha=2.0, speed=1.0, J_flee=10.0, R_flee=60.0, J_chase=0.2, R_chase=150.0,
                 predator_speed=0.85, sprint_period=50, sprint_steps=10, sprint_factor=2.0):
    return md_flock_params(J_align, R_align, J_avoid, R_avoid, J_cohesion, R_cohesion, J_obstacle, alpha, speed,
                           J_flee, R_flee, J_chase, R_chase, predator_speed, int(sprint_period), int(sprint_steps),
                           sprint_factor)


class md_replica_desc(C.Structure):
    _fields_ = [("N", C.c_int), ("L", C.c_double), ("kind", C.c_int), ("eps", C.c_float), ("sigma", C.c_float),
                ("r_cut", C.c_float), ("e_shift", C.c_float), ("alpha", C.c_float), ("skin", C.c_float),
                ("dt", C.c_float), ("mass", C.c_float), ("cell_mult", C.c_float)]


class md_batch(C.Structure):
    _fields_ = [("R", C.c_int), ("N", C.c_int), ("cap", C.c_int), ("ncell_total", C.c_int), ("tpp", C.c_int),
                ("ws_bytes", C.c_size_t), ("nbr", C.c_void_p), ("cnt", C.c_void_p), ("rref", C.c_void_p),
                ("ws", C.c_void_p), ("host", C.c_void_p)]


_P = C.POINTER
_vp = C.c_void_p
_SIGS = {
    "md_space_periodic": [C.c_int, _P(C.c_double), _P(md_space)],
    "md_nbr_plan": [_P(md_space), C.c_int, C.c_float, C.c_float, C.c_int, _P(md_nbr)],
    "md_nbr_set_flags": [_P(md_nbr), C.c_int],
    "md_nbr_bind": [_P(md_nbr), _vp, _vp, _vp, _vp, _vp],
    "md_neighbor_list_build": [_P(md_space), _vp, _P(md_nbr), _vp, _vp],
    "md_neighbor_list_update": [_P(md_space), _vp, _P(md_nbr), _vp, _vp],
    "md_nbr_stats": [_P(md_nbr), _P(C.c_int64), _P(C.c_int32), _vp],
    "md_energy_forces": [_P(md_space), _P(md_pot), _vp, _P(md_nbr), _vp, _vp, _vp, _vp],
    "md_set_pair_tpp": [C.c_int],
    "md_set_pair_options": [C.c_int],
    "md_set_nve_fusion": [C.c_int],
    "md_set_loop_graphs": [C.c_int],
    "md_integrate_nve": [_P(md_space), _P(md_pot), _vp, _vp, _vp, C.c_float, C.c_float, C.c_int, _P(md_nbr),
                         _vp, _vp, C.c_int, _vp, _vp],
    "md_integrate_langevin": [_P(md_space), _P(md_pot), _vp, _vp, _vp, C.c_float, C.c_float, C.c_float, C.c_float,
                              C.c_uint64, C.c_uint32, C.c_int, _P(md_nbr), _vp, _vp, C.c_int, _vp, _vp],
    "md_minimize": [_P(md_space), _P(md_pot), C.c_int, C.c_float, C.c_int, _vp, _vp, _P(md_nbr), _vp, _vp, _vp],
    "md_minimize_fire": [_P(md_space), _P(md_pot), _P(md_fire_params), C.c_int, _vp, _vp, _vp, _P(md_nbr), _vp, C.c_int,
                         _vp, _vp, _vp],
    "md_fire_state_read": [_vp, _P(C.c_double), _vp],
    "md_flock_run": [_P(md_space), _P(md_flock_params), _vp, C.c_int, _vp, _vp, C.c_int, _vp, _vp, _vp, C.c_float,
                     C.c_int, _P(md_nbr), _vp, _vp, _vp],
    "md_integrate_nhc": [_P(md_space), _P(md_pot), _vp, _vp, _vp, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int,
                         C.c_int, _P(md_nbr), _vp, C.c_int, _vp, _vp, _vp, C.c_int, _vp, _vp],
    "md_status_poll": [_vp, _P(C.c_uint32), _vp],
    "md_bounded_wait": [_vp, C.c_uint64, _vp, _vp],
    "md_sort_particles": [_P(md_space), _P(md_nbr), _vp, _vp, _vp, _vp, C.c_size_t, _vp, _vp],
    "md_fma_probe": [_vp, C.c_int, C.c_int, C.c_int, _P(C.c_uint64), _vp],
    "md_bp_descriptors": [_P(md_space), _vp, _P(md_nbr), C.c_int, _vp, _vp, _vp],
    "md_bp_mlp_infer": [_vp, _vp, _vp, C.c_int, _vp, _vp, _vp],
    "md_bp_mlp_infer_tc": [_vp, _vp, _vp, C.c_int, _vp, _vp, _vp, _vp],
    "md_bp_set_tensor_cores": [C.c_int],
    "md_gnn_set_group": [C.c_int],
    "md_gnn_set_tensor_cores": [C.c_int],
    "md_gnn_train_grad": [_P(md_space), _vp, _P(md_nbr), _P(md_gnn_model), _vp, _vp, _vp, C.c_size_t, _vp, _vp,
                          _vp],
    "md_bp_forces": [_P(md_space), _vp, _P(md_nbr), C.c_int, _vp, _vp, _vp, _vp, _vp, _vp],
    "md_bp_jvp": [_P(md_space), _vp, _P(md_nbr), C.c_int, _vp, _vp, _vp, _vp],
    "md_bp_mlp_train": [_vp, _vp, _vp, _vp, _vp, C.c_float, C.c_int, _vp, _vp, _vp],
    "md_bp_mlp_train_tc": [_vp, _vp, _vp, _vp, _vp, C.c_float, C.c_int, _vp, _vp, _vp, _vp],
    "md_bp_loss_prep": [_vp, _vp, _vp, _vp, C.c_int, C.c_int, C.c_float, _vp, _vp, _vp, _vp],
    "md_column_stats": [_vp, C.c_int, C.c_int, _vp, _vp],
    "md_adam_step": [_vp, _vp, _vp, _vp, C.c_int, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int, _vp],
    "md_batch_plan": [_P(md_replica_desc), C.c_int, C.c_int, _P(md_batch)],
    "md_batch_bind": [_P(md_batch), _vp, _vp, _vp, _vp, _vp],
    "md_batch_build": [_P(md_batch), _vp, _vp, _vp],
    "md_batch_forces": [_P(md_batch), _vp, _vp, _vp, _vp],
    "md_batch_run_nve": [_P(md_batch), _vp, _vp, _vp, C.c_int, _vp, _vp, C.c_int, _vp, _vp],
    "md_batch_stats": [_P(md_batch), _P(C.c_uint32), _vp],
    "md_batch_autotune": [_P(md_batch), _vp, _vp, _vp, _vp, C.c_int, C.c_char_p, _P(C.c_int), _vp],
    "md_batch_set_class_tpp": [_P(md_batch), _vp, _vp],
    "md_packing_space": [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, _P(md_space), _P(C.c_double)],
    "md_minimize_adjoint": [_P(md_space), _P(md_pot), _P(md_nbr), _vp, C.c_int, C.c_float, C.c_float, C.c_double,
                            C.c_float, C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp],
    "md_minimize_fire_adjoint": [_P(md_space), _P(md_pot), _P(md_fire_params), _P(md_nbr), _vp, C.c_int, C.c_float,
                                 C.c_float, C.c_double, C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "md_tiles_import": [_P(md_space), _vp, _vp, _vp, _P(md_nbr), _vp, _vp],
    "md_tiles_forces": [_P(md_space), _P(md_pot), _P(md_nbr), _vp, _vp, _vp],
    "md_tiles_export": [_P(md_space), _P(md_nbr), _vp, _vp, _vp, C.c_int, _vp],
    "md_tiles_info": [_P(md_space), _P(md_nbr), _P(C.c_int32)],
    "md_tiles_steps": [_P(md_space), _P(md_pot), _P(md_nbr), C.c_float, C.c_float, C.c_int, _vp, _vp, _vp, _vp],
    "md_set_tile_tpp": [C.c_int],
    "md_neighbor_list_build_noalloc": [_P(md_space), _vp, C.c_int, C.c_float, C.c_float, C.c_int, _vp, _vp, _vp,
                                       _vp],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
_lib.md_launch_count.restype = C.c_uint64
_lib.md_launch_count.argtypes = []
_lib.md_bp_train_scratch_size.restype = C.c_size_t
_lib.md_bp_train_scratch_size.argtypes = [C.c_int]
_lib.md_batch_free.restype = None
_lib.md_batch_free.argtypes = [_P(md_batch)]
_lib.md_adjoint_workspace_size.restype = C.c_size_t
_lib.md_adjoint_workspace_size.argtypes = [C.c_int, C.c_int, C.c_int]
_lib.md_fire_adjoint_workspace_size.restype = C.c_size_t
_lib.md_fire_adjoint_workspace_size.argtypes = [C.c_int, C.c_int, C.c_int]
_lib.md_sort_scratch_bytes.restype = C.c_size_t
_lib.md_sort_scratch_bytes.argtypes = [_P(md_nbr)]
_lib.md_noalloc_scratch_bytes.restype = C.c_size_t
_lib.md_noalloc_scratch_bytes.argtypes = []
_lib.md_fire_state_bytes.restype = C.c_size_t
_lib.md_fire_state_bytes.argtypes = []
_lib.md_bp_lists_bytes.restype = C.c_size_t
_lib.md_bp_lists_bytes.argtypes = [C.c_int]
_lib.md_sw_lists_bytes.restype = C.c_size_t
_lib.md_sw_lists_bytes.argtypes = [C.c_int]
_lib.md_nhc_state_doubles.restype = C.c_size_t
_lib.md_nhc_state_doubles.argtypes = [C.c_int]
_lib.md_gnn_param_count.restype = C.c_size_t
_lib.md_gnn_param_count.argtypes = [C.c_int, C.c_int]
_lib.md_gnn_train_scratch_bytes.restype = C.c_size_t
_lib.md_gnn_train_scratch_bytes.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int]
_lib.md_gnn_workspace_bytes.restype = C.c_size_t
_lib.md_gnn_workspace_bytes.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int]
_lib.md_version.restype = C.c_char_p
_lib.md_version.argtypes = []


def lib():
    return _lib


def _check(code: int, where: str):
    if code != MD_OK:
        raise MDError(code, where)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libjmd needs CUDA tensors (no CPU fallback)")
    if not t.is_contiguous():
        raise ValueError("libjmd needs contiguous tensors")
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


# ----------------------------------------------------------------------------
# C ABI, same names (Sec. 3.2.1 - 3.3.2)
# ----------------------------------------------------------------------------
def md_space_periodic(dim: int, box) -> md_space:
    vals = [float(x) for x in (box if hasattr(box, "__len__") else [box] * dim)]
    b = (C.c_double * 3)(*(vals + [1.0, 1.0, 1.0])[:3])
    out = md_space()
    _check(_lib.md_space_periodic(int(dim), b, C.byref(out)), "md_space_periodic")
    return out


def md_nbr_plan(space: md_space, N: int, r_cut: float, skin: float, cap: int) -> md_nbr:
    out = md_nbr()
    _check(_lib.md_nbr_plan(C.byref(space), int(N), float(r_cut), float(skin), int(cap), C.byref(out)),
           "md_nbr_plan")
    return out


def md_nbr_set_flags(nb: md_nbr, flags: int):
    _check(_lib.md_nbr_set_flags(C.byref(nb), int(flags)), "md_nbr_set_flags")


def md_nbr_bind(nb: md_nbr, nbr, cnt, rref, ws, stream=None):
    _check(_lib.md_nbr_bind(C.byref(nb), _ptr(nbr), _ptr(cnt), _ptr(rref), _ptr(ws), _stream(stream)),
           "md_nbr_bind")


def md_neighbor_list_build(space, r, nb, status, stream=None):
    _check(_lib.md_neighbor_list_build(C.byref(space), _ptr(r), C.byref(nb), _ptr(status), _stream(stream)),
           "md_neighbor_list_build")


def md_neighbor_list_update(space, r, nb, status, stream=None):
    _check(_lib.md_neighbor_list_update(C.byref(space), _ptr(r), C.byref(nb), _ptr(status), _stream(stream)),
           "md_neighbor_list_update")


def md_nbr_stats(nb, stream=None):
    b = C.c_int64()
    m = C.c_int32()
    _check(_lib.md_nbr_stats(C.byref(nb), C.byref(b), C.byref(m), _stream(stream)), "md_nbr_stats")
    return b.value, m.value


def md_energy_forces(space, pot, r, nb, f, E=None, status=None, stream=None):
    _check(_lib.md_energy_forces(C.byref(space), C.byref(pot), _ptr(r), C.byref(nb), _ptr(f), _ptr(E),
                                 _ptr(status), _stream(stream)), "md_energy_forces")


def md_set_pair_options(opt: int):
    _check(_lib.md_set_pair_options(int(opt)), "md_set_pair_options")


def md_set_loop_graphs(on: bool):
    _check(_lib.md_set_loop_graphs(int(bool(on))), "md_set_loop_graphs")


def md_set_nve_fusion(on: bool):
    _check(_lib.md_set_nve_fusion(int(bool(on))), "md_set_nve_fusion")


def md_set_pair_tpp(tpp: int):
    _check(_lib.md_set_pair_tpp(int(tpp)), "md_set_pair_tpp")


def md_integrate_nve(space, pot, r, v, f, mass, dt, nsteps, nb, PE=None, KE=None, use_graph=True, status=None,
                     stream=None):
    _check(_lib.md_integrate_nve(C.byref(space), C.byref(pot), _ptr(r), _ptr(v), _ptr(f), float(mass), float(dt),
                                 int(nsteps), C.byref(nb), _ptr(PE), _ptr(KE), int(bool(use_graph)), _ptr(status),
                                 _stream(stream)), "md_integrate_nve")


def md_tiles_import(space, r, v, f, nb, status=None, stream=None):
    _check(_lib.md_tiles_import(C.byref(space), _ptr(r), _ptr(v), _ptr(f), C.byref(nb), _ptr(status),
                                _stream(stream)), "md_tiles_import")


def md_tiles_forces(space, pot, nb, E=None, status=None, stream=None):
    _check(_lib.md_tiles_forces(C.byref(space), C.byref(pot), C.byref(nb), _ptr(E), _ptr(status), _stream(stream)),
           "md_tiles_forces")


def md_tiles_export(space, nb, r=None, v=None, f=None, rows=False, stream=None):
    _check(_lib.md_tiles_export(C.byref(space), C.byref(nb), _ptr(r), _ptr(v), _ptr(f), int(bool(rows)),
                                _stream(stream)), "md_tiles_export")


def md_tiles_steps(space, pot, nb, mass, dt, nsteps, PE=None, KE=None, status=None, stream=None):
    _check(_lib.md_tiles_steps(C.byref(space), C.byref(pot), C.byref(nb), float(mass), float(dt), int(nsteps),
                               _ptr(PE), _ptr(KE), _ptr(status), _stream(stream)), "md_tiles_steps")


def md_tiles_info(space, nb):
    """Half-cells per axis, tile extent (x, y, z), number of tiles, region capacity."""
    out = (C.c_int32 * 8)()
    _check(_lib.md_tiles_info(C.byref(space), C.byref(nb), out), "md_tiles_info")
    return {"H": tuple(out[0:3]), "tile": tuple(out[3:6]), "ntiles": out[6], "region_cap": out[7]}


def md_set_tile_tpp(tpp: int):
    _check(_lib.md_set_tile_tpp(int(tpp)), "md_set_tile_tpp")


def md_integrate_langevin(space, pot, r, v, f, mass, dt, gamma, kT, seed, step0, nsteps, nb, PE=None, KE=None,
                          use_graph=True, status=None, stream=None):
    _check(_lib.md_integrate_langevin(C.byref(space), C.byref(pot), _ptr(r), _ptr(v), _ptr(f), float(mass),
                                      float(dt), float(gamma), float(kT), int(seed), int(step0), int(nsteps),
                                      C.byref(nb), _ptr(PE), _ptr(KE), int(bool(use_graph)), _ptr(status),
                                      _stream(stream)), "md_integrate_langevin")


def md_minimize(space, pot, kind, step, nsteps, r, f, nb, E=None, status=None, stream=None):
    _check(_lib.md_minimize(C.byref(space), C.byref(pot), int(kind), float(step), int(nsteps), _ptr(r), _ptr(f),
                            C.byref(nb), _ptr(E), _ptr(status), _stream(stream)), "md_minimize")


def md_nhc_state_doubles(M: int) -> int:
    return int(_lib.md_nhc_state_doubles(int(M)))


def md_integrate_nhc(space, pot, r, v, f, mass, dt, kT, tau, M, nsteps, nb, therm, reset=True, PE=None, KE=None,
                     H=None, use_graph=True, status=None, stream=None):
    _check(_lib.md_integrate_nhc(C.byref(space), C.byref(pot), _ptr(r), _ptr(v), _ptr(f), float(mass), float(dt),
                                 float(kT), float(tau), int(M), int(nsteps), C.byref(nb), _ptr(therm),
                                 int(bool(reset)), _ptr(PE), _ptr(KE), _ptr(H), int(bool(use_graph)), _ptr(status),
                                 _stream(stream)), "md_integrate_nhc")


def md_flock_run(space, params, obs, n_obs, pred, pred_alt, n_pred, b, theta, b_alt, dt, nsteps, nb, E=None,
                 status=None, stream=None):
    _check(_lib.md_flock_run(C.byref(space), C.byref(params), _ptr(obs), int(n_obs), _ptr(pred), _ptr(pred_alt),
                             int(n_pred), _ptr(b), _ptr(theta), _ptr(b_alt), float(dt), int(nsteps), C.byref(nb),
                             _ptr(E), _ptr(status), _stream(stream)), "md_flock_run")


def md_fire_state_bytes() -> int:
    return int(_lib.md_fire_state_bytes())


def md_minimize_fire(space, pot, params, nsteps, r, v, f, nb, state, restart=True, E=None, status=None, stream=None):
    _check(_lib.md_minimize_fire(C.byref(space), C.byref(pot), C.byref(params), int(nsteps), _ptr(r), _ptr(v), _ptr(f),
                                 C.byref(nb), _ptr(state), int(bool(restart)), _ptr(E), _ptr(status), _stream(stream)),
           "md_minimize_fire")


def md_fire_state_read(state, stream=None):
    """(dt, alpha, count of consecutive P > 0 steps) of a FIRE state."""
    out = (C.c_double * 3)()
    _check(_lib.md_fire_state_read(_ptr(state), out, _stream(stream)), "md_fire_state_read")
    return float(out[0]), float(out[1]), int(out[2])


def md_neighbor_list_build_noalloc(space, r, N, r_cut, skin, cap, nbr, cnt, status=None, stream=None):
    """Neighbor-list build on the library's fixed scratch pool: for callers
    that can pass only their input and output buffers (see include/jmd.h)."""
    _check(_lib.md_neighbor_list_build_noalloc(C.byref(space), _ptr(r), int(N), float(r_cut), float(skin), int(cap),
                                               _ptr(nbr), _ptr(cnt), _ptr(status), _stream(stream)),
           "md_neighbor_list_build_noalloc")


def md_sort_scratch_bytes(nb) -> int:
    return int(_lib.md_sort_scratch_bytes(C.byref(nb)))


def md_sort_particles(space, nb, r, v, perm, scratch, status=None, stream=None):
    """Renumber the particles along the Z-order curve of the list's cells;
    perm[new] = old.  scratch: a 256-byte aligned uint8 tensor of at least
    md_sort_scratch_bytes(nb) bytes."""
    _check(_lib.md_sort_particles(C.byref(space), C.byref(nb), _ptr(r), _ptr(v), _ptr(perm), _ptr(scratch),
                                  int(scratch.numel() * scratch.element_size()), _ptr(status), _stream(stream)),
           "md_sort_particles")


def md_noalloc_scratch_bytes() -> int:
    return int(_lib.md_noalloc_scratch_bytes())


# ----------------------------------------------------------------------------
# Learned potential (Sec. 3.2.4, 4.1)
# ----------------------------------------------------------------------------
BP_NPARAMS = 5313


def md_bp_descriptors(space, r, nb, sys_n, G, status=None, stream=None):
    _check(_lib.md_bp_descriptors(C.byref(space), _ptr(r), C.byref(nb), int(sys_n), _ptr(G), _ptr(status),
                                  _stream(stream)), "md_bp_descriptors")


def md_bp_mlp_infer(params, norm, G, N, Ei, dEdG, stream=None):
    _check(_lib.md_bp_mlp_infer(_ptr(params), _ptr(norm), _ptr(G), int(N), _ptr(Ei), _ptr(dEdG), _stream(stream)),
           "md_bp_mlp_infer")


def md_bp_mlp_infer_tc(params, norm, G, N, Ei, dEdG, status=None, stream=None):
    _check(_lib.md_bp_mlp_infer_tc(_ptr(params), _ptr(norm), _ptr(G), int(N), _ptr(Ei), _ptr(dEdG), _ptr(status),
                                   _stream(stream)), "md_bp_mlp_infer_tc")


def md_bp_set_tensor_cores(on: bool):
    _check(_lib.md_bp_set_tensor_cores(int(bool(on))), "md_bp_set_tensor_cores")


def md_bp_forces(space, r, nb, sys_n, dEdG, Ei, f, E=None, status=None, stream=None):
    _check(_lib.md_bp_forces(C.byref(space), _ptr(r), C.byref(nb), int(sys_n), _ptr(dEdG), _ptr(Ei), _ptr(f), _ptr(E),
                             _ptr(status), _stream(stream)), "md_bp_forces")


def md_bp_jvp(space, r, nb, sys_n, dF, V, status=None, stream=None):
    _check(_lib.md_bp_jvp(C.byref(space), _ptr(r), C.byref(nb), int(sys_n), _ptr(dF), _ptr(V), _ptr(status),
                          _stream(stream)), "md_bp_jvp")


def md_bp_train_scratch_size(N) -> int:
    return int(_lib.md_bp_train_scratch_size(int(N)))


def md_bp_mlp_train(params, norm, G, V, cE, cF, N, scratch, grad, stream=None):
    _check(_lib.md_bp_mlp_train(_ptr(params), _ptr(norm), _ptr(G), _ptr(V), _ptr(cE), float(cF), int(N),
                                _ptr(scratch), _ptr(grad), _stream(stream)), "md_bp_mlp_train")


def md_bp_mlp_train_tc(params, norm, G, V, cE, cF, N, scratch, grad, status=None, stream=None):
    """md_bp_mlp_train on the tensor cores (tcgen05, BF16 operands)."""
    _check(_lib.md_bp_mlp_train_tc(_ptr(params), _ptr(norm), _ptr(G), _ptr(V), _ptr(cE), float(cF), int(N),
                                   _ptr(scratch), _ptr(grad), _ptr(status), _stream(stream)), "md_bp_mlp_train_tc")


def md_bp_loss_prep(Ei, F, Fref, Eref, S, n, wF, cE, dF, loss, stream=None):
    _check(_lib.md_bp_loss_prep(_ptr(Ei), _ptr(F), _ptr(Fref), _ptr(Eref), int(S), int(n), float(wF), _ptr(cE),
                                _ptr(dF), _ptr(loss), _stream(stream)), "md_bp_loss_prep")


def md_column_stats(X, N, D, out, stream=None):
    _check(_lib.md_column_stats(_ptr(X), int(N), int(D), _ptr(out), _stream(stream)), "md_column_stats")


def md_adam_step(params, grad, m, v, n, lr, beta1, beta2, eps, step, stream=None):
    _check(_lib.md_adam_step(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(n), float(lr), float(beta1),
                             float(beta2), float(eps), int(step), _stream(stream)), "md_adam_step")


class BPModel:
    """Device buffers of a learned potential for N atoms and the md_pot that
    points at them (kind MD_BP).  params [5313] and norm [32] are FP32 CUDA
    tensors owned by the caller."""

    def __init__(self, params, norm, N, sys_n=0, device="cuda", lists=True):
        import torch
        self.params, self.norm = params, norm
        self.G = torch.zeros((N, 16), dtype=torch.float32, device=device)
        self.dEdG = torch.zeros((N, 16), dtype=torch.float32, device=device)
        self.Ei = torch.zeros(N, dtype=torch.float32, device=device)
        lp = None
        if lists:   # partner-list scratch: the two-kernel triplet sweep of the force gather
            self._lists = torch.empty(md_bp_lists_bytes(N) + 256, dtype=torch.uint8, device=device)
            lp = (self._lists.data_ptr() + 255) // 256 * 256
        self.model = md_bp_model(_ptr(params).value, _ptr(norm).value, _ptr(self.G).value, _ptr(self.dEdG).value,
                                 _ptr(self.Ei).value, int(sys_n), lp)
        self.pot = md_pot()
        self.pot.kind = MD_BP
        self.pot.model = C.cast(C.pointer(self.model), C.c_void_p)


def md_gnn_param_count(H, T):
    return int(_lib.md_gnn_param_count(int(H), int(T)))


def md_gnn_set_tensor_cores(on):
    _check(_lib.md_gnn_set_tensor_cores(int(bool(on))), "md_gnn_set_tensor_cores")


def md_gnn_set_group(G):
    _check(_lib.md_gnn_set_group(int(G)), "md_gnn_set_group")


def md_gnn_workspace_bytes(N, cap, H, T):
    return int(_lib.md_gnn_workspace_bytes(int(N), int(cap), int(H), int(T)))


def md_gnn_train_scratch_bytes(N, cap, H, T):
    return int(_lib.md_gnn_train_scratch_bytes(int(N), int(cap), int(H), int(T)))


def md_gnn_train_grad(space, r, nb, model, cE, dF, scratch, grad, status=None, stream=None):
    """model: a GNNModel (its md_gnn_model is passed); scratch: a 256-byte
    aligned uint8 tensor."""
    _check(_lib.md_gnn_train_grad(C.byref(space), _ptr(r), C.byref(nb), C.byref(model.model), _ptr(cE), _ptr(dF),
                                  _ptr(scratch), int(scratch.numel()), _ptr(grad), _ptr(status), _stream(stream)),
           "md_gnn_train_grad")


class GNNModel:
    """Workspace of the graph-network potential for a list of N atoms with
    row capacity cap, and the md_pot that points at the model (kind
    MD_GNN).  params: FP32 CUDA tensor of md_gnn_param_count(H, T) floats,
    owned by the caller."""

    def __init__(self, params, N, cap, H=64, T=2, r_cut=3.77, device="cuda", sys_n=0):
        import torch
        n = md_gnn_param_count(H, T)
        if n == 0 or params.numel() != n:
            raise MDError(MD_ERR_INVALID, "GNNModel: parameter count")
        nbytes = md_gnn_workspace_bytes(N, cap, H, T)
        if nbytes == 0:
            raise MDError(MD_ERR_INVALID, "GNNModel: unsupported N, cap, H or T")
        self.params = params
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.model = md_gnn_model(_ptr(params).value, int(H), int(T), float(r_cut), _ptr(self.ws).value, nbytes,
                                  int(sys_n))
        self.pot = md_pot()
        self.pot.kind = MD_GNN
        self.pot.model = C.cast(C.pointer(self.model), C.c_void_p)


# ----------------------------------------------------------------------------
# Batched replicas (Sec. 4.2 vmap over systems)
# ----------------------------------------------------------------------------
def md_batch_plan(descs, cap) -> md_batch:
    arr = (md_replica_desc * len(descs))(*descs)
    out = md_batch()
    _check(_lib.md_batch_plan(arr, len(descs), int(cap), C.byref(out)), "md_batch_plan")
    return out


def md_batch_free(bt):
    _lib.md_batch_free(C.byref(bt))


def md_batch_bind(bt, nbr, cnt, rref, ws, stream=None):
    _check(_lib.md_batch_bind(C.byref(bt), _ptr(nbr), _ptr(cnt), _ptr(rref), _ptr(ws), _stream(stream)),
           "md_batch_bind")


def md_batch_build(bt, r, status=None, stream=None):
    _check(_lib.md_batch_build(C.byref(bt), _ptr(r), _ptr(status), _stream(stream)), "md_batch_build")


def md_batch_forces(bt, r, f, status=None, stream=None):
    _check(_lib.md_batch_forces(C.byref(bt), _ptr(r), _ptr(f), _ptr(status), _stream(stream)), "md_batch_forces")


def md_batch_run_nve(bt, r, v, f, nsteps, PE=None, KE=None, use_graph=True, status=None, stream=None):
    _check(_lib.md_batch_run_nve(C.byref(bt), _ptr(r), _ptr(v), _ptr(f), int(nsteps), _ptr(PE), _ptr(KE),
                                 int(bool(use_graph)), _ptr(status), _stream(stream)), "md_batch_run_nve")


def md_batch_stats(bt, stream=None):
    h = (C.c_uint32 * bt.R)()
    _check(_lib.md_batch_stats(C.byref(bt), h, _stream(stream)), "md_batch_stats")
    return list(h)


def md_batch_autotune(bt, r, v, f, scratch, probe, cache_path=None, stream=None) -> int:
    t = C.c_int()
    _check(_lib.md_batch_autotune(C.byref(bt), _ptr(r), _ptr(v), _ptr(f), _ptr(scratch), int(probe),
                                  cache_path.encode() if cache_path else None, C.byref(t), _stream(stream)),
           "md_batch_autotune")
    return t.value


def md_batch_set_class_tpp(bt, tpp_of_rep, stream=None):
    """Threads per particle of the force kernel per replica (4, 8 or 16);
    None returns to one launch with bt.tpp."""
    if tpp_of_rep is None:
        _check(_lib.md_batch_set_class_tpp(C.byref(bt), None, _stream(stream)), "md_batch_set_class_tpp")
        return
    arr = (C.c_int * len(tpp_of_rep))(*[int(t) for t in tpp_of_rep])
    _check(_lib.md_batch_set_class_tpp(C.byref(bt), arr, _stream(stream)), "md_batch_set_class_tpp")


class Batch:
    """Plans, allocates (torch storage) and binds a replica batch."""

    def __init__(self, descs, cap=128, device="cuda", stream=None):
        import torch
        self.plan = md_batch_plan(descs, cap)
        N = self.plan.N
        self.nbr = torch.zeros((N, cap), dtype=torch.int32, device=device)
        self.cnt = torch.zeros(N, dtype=torch.int32, device=device)
        self.rref = torch.zeros((N, 4), dtype=torch.float32, device=device)
        self.ws = torch.empty(int(self.plan.ws_bytes) + 256, dtype=torch.uint8, device=device)
        off = (-self.ws.data_ptr()) % 256
        self.ws_view = self.ws[off: off + int(self.plan.ws_bytes)]
        md_batch_bind(self.plan, self.nbr, self.cnt, self.rref, self.ws_view, stream)

    def __del__(self):
        try:
            md_batch_free(self.plan)
        except Exception:
            pass


def md_adjoint_workspace_size(N, T, K) -> int:
    return int(_lib.md_adjoint_workspace_size(int(N), int(T), int(K)))


def md_packing_space(N, nA, D, dB, phi):
    """(space, dL/dD) of the bidisperse disk packing at packing fraction phi."""
    out = md_space()
    lp = C.c_double()
    _check(_lib.md_packing_space(int(N), int(nA), float(D), float(dB), float(phi), C.byref(out), C.byref(lp)),
           "md_packing_space")
    return out, lp.value


def md_minimize_adjoint(space, pot, nb, s0, nA, D, dB, phi, eta, T, K, r, f, ws, out, status=None, stream=None):
    _check(_lib.md_minimize_adjoint(C.byref(space), C.byref(pot), C.byref(nb), _ptr(s0), int(nA), float(D),
                                    float(dB), float(phi), float(eta), int(T), int(K), _ptr(r), _ptr(f), _ptr(ws),
                                    _ptr(out), _ptr(status), _stream(stream)), "md_minimize_adjoint")


def md_fire_adjoint_workspace_size(N, T, K) -> int:
    return int(_lib.md_fire_adjoint_workspace_size(int(N), int(T), int(K)))


def md_minimize_fire_adjoint(space, pot, fire, nb, s0, nA, D, dB, phi, T, K, r, v, f, ws, out, status=None,
                             stream=None):
    _check(_lib.md_minimize_fire_adjoint(C.byref(space), C.byref(pot), C.byref(fire), C.byref(nb), _ptr(s0), int(nA),
                                         float(D), float(dB), float(phi), int(T), int(K), _ptr(r), _ptr(v), _ptr(f),
                                         _ptr(ws), _ptr(out), _ptr(status), _stream(stream)),
           "md_minimize_fire_adjoint")


def md_status_poll(status, stream=None) -> int:
    h = C.c_uint32()
    _check(_lib.md_status_poll(_ptr(status), C.byref(h), _stream(stream)), "md_status_poll")
    return h.value


def md_bounded_wait(flag, limit, status, stream=None):
    _check(_lib.md_bounded_wait(_ptr(flag), int(limit), _ptr(status), _stream(stream)), "md_bounded_wait")


def md_fma_probe(out, blocks, threads, iters, stream=None) -> int:
    """Launch the FP32 FMA throughput probe; returns the launch's FLOP count."""
    fl = C.c_uint64(0)
    _check(_lib.md_fma_probe(_ptr(out), int(blocks), int(threads), int(iters), C.byref(fl), _stream(stream)),
           "md_fma_probe")
    return int(fl.value)


def md_launch_count() -> int:
    return int(_lib.md_launch_count())


def md_version() -> str:
    return _lib.md_version().decode()


# ----------------------------------------------------------------------------
# Potential descriptors
# ----------------------------------------------------------------------------
def lj_pot(eps=1.0, sigma=1.0, r_cut=2.5, shifted=True) -> md_pot:
    """LJ (Sec. 3.3.2): e_shift = u(r_cut) evaluated in FP64 when shifted."""
    p = md_pot()
    p.kind = MD_LJ
    p.eps, p.sigma, p.r_cut = eps, sigma, r_cut
    sr6 = (sigma / r_cut) ** 6
    p.e_shift = 4.0 * eps * (sr6 * sr6 - sr6) if shifted else 0.0
    return p


def soft_pot(eps=1.0, alpha=2.0) -> md_pot:
    p = md_pot()
    p.kind = MD_SOFT_SPHERE
    p.eps, p.alpha = eps, alpha
    return p


def md_bp_lists_bytes(N: int) -> int:
    return int(_lib.md_bp_lists_bytes(int(N)))


def md_sw_lists_bytes(N: int) -> int:
    return int(_lib.md_sw_lists_bytes(int(N)))


def sw_pot(params, N=None, device="cuda") -> md_pot:
    """Stillinger-Weber potential; with N, the partner-list scratch for N
    atoms is allocated (torch, kept alive by the returned struct) and the
    two-kernel form is used."""
    p = md_pot()
    p.kind = MD_SW
    for k, v in enumerate(params):
        p.sw[k] = float(v)
    if N is not None:
        import torch
        p._lists = torch.empty(md_sw_lists_bytes(N) + 256, dtype=torch.uint8, device=device)
        base = p._lists.data_ptr()
        p.model = (base + 255) // 256 * 256
    return p


# ----------------------------------------------------------------------------
# Device-memory plumbing (torch tensors) for a neighbor list
# ----------------------------------------------------------------------------
class NeighborList:
    """Plans a list, allocates its caller-owned tensors with torch and binds them."""

    def __init__(self, space: md_space, N: int, r_cut: float, skin: float, cap: int, device="cuda", stream=None,
                 canonical: bool = False, local_rows: bool = False, tiles: bool = False):
        import torch
        self.space = space
        self.plan = md_nbr_plan(space, N, r_cut, skin, cap)
        flags = ((MD_NBR_CANONICAL if canonical else 0) | (MD_NBR_LOCAL_ROWS if local_rows else 0)
                 | (MD_NBR_TILES if tiles else 0))
        if flags:
            md_nbr_set_flags(self.plan, flags)
        self.nbr = torch.empty((N, cap), dtype=torch.int32, device=device)
        self.cnt = torch.zeros(N, dtype=torch.int32, device=device)
        self.rref = torch.zeros((N, 4), dtype=torch.float32, device=device)
        self.ws = torch.empty(int(self.plan.ws_bytes) + 256, dtype=torch.uint8, device=device)
        off = (-self.ws.data_ptr()) % 256
        self.ws_view = self.ws[off: off + int(self.plan.ws_bytes)]
        md_nbr_bind(self.plan, self.nbr, self.cnt, self.rref, self.ws_view, stream)

    @property
    def N(self):
        return self.plan.N

    @property
    def cap(self):
        return self.plan.cap

    def build(self, r, status, stream=None):
        md_neighbor_list_build(self.space, r, self.plan, status, stream)

    def update(self, r, status, stream=None):
        md_neighbor_list_update(self.space, r, self.plan, status, stream)

    def stats(self, stream=None):
        return md_nbr_stats(self.plan, stream)

    def sort(self, r, v, status, stream=None):
        """Spatially sort r and v in place (md_sort_particles) and rebuild
        the list; returns perm (int32, perm[new] = old).  The scratch is a
        torch tensor kept with the list."""
        import torch
        nbytes = md_sort_scratch_bytes(self.plan)
        if getattr(self, "_sort_ws", None) is None or self._sort_ws_bytes < nbytes:
            raw = torch.empty(nbytes + 256, dtype=torch.uint8, device=r.device)
            off = (-raw.data_ptr()) % 256
            self._sort_raw, self._sort_ws, self._sort_ws_bytes = raw, raw[off:off + nbytes], nbytes
        perm = torch.empty(self.N, dtype=torch.int32, device=r.device)
        md_sort_particles(self.space, self.plan, r, v, perm, self._sort_ws, status, stream)
        return perm
