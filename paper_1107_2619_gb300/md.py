"""Thin ctypes binding of libmd.so (include/md.h): argument marshalling only.

Functions carry the C names (md_create, md_build_neighbours, md_eam_forces, md_step,
md_energy, md_get, md_set_state, md_last_error, md_destroy).  Arrays are numpy
arrays (host) or CUDA torch tensors (device, passed by data_ptr with on_device=1).
Every computation runs in the library's CUDA kernels; there is no fallback: if the
library has not been built, the first call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import inputs as _inputs

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmd.so")

MD_OK, MD_ERR_ARG, MD_ERR_SPECIES, MD_ERR_BOX, MD_ERR_NBR_OVERFLOW = 0, 1, 2, 3, 4
MD_ERR_SKIN, MD_ERR_NONFINITE, MD_ERR_TABLE_RANGE, MD_ERR_TIMEOUT = 5, 6, 7, 8
MD_ERR_CUDA, MD_ERR_OOM, MD_ERR_STATE, MD_ERR_CAPACITY = 9, 10, 11, 12
MD_NOALLOC_MAX_ATOMS, MD_NOALLOC_MAX_CELLS = 131072, 65536
MD_POT_FS_ANALYTIC, MD_POT_TABLES, MD_POT_SURROGATE, MD_POT_KNOTS = 1, 2, 3, 4
MD_SUR_FP32, MD_SUR_BF16 = 0, 1
MD_SUR_GET_G, MD_SUR_GET_DEDG = 0, 1
MD_SUR_NB, MD_SUR_H1, MD_SUR_H2, MD_SUR_PARAMS = 32, 64, 64, 6337
MD_PREC_FP64, MD_PREC_MIXED, MD_PREC_DF = 0, 1, 2
PRECISIONS = {"fp64": MD_PREC_FP64, "mixed": MD_PREC_MIXED, "df": MD_PREC_DF}
(MD_GET_POS, MD_GET_VEL, MD_GET_FORCE, MD_GET_RHO, MD_GET_EATOM, MD_GET_DF, MD_GET_NBR_COUNT,
 MD_GET_NBR_LIST, MD_GET_SPECIES, MD_GET_IMAGE) = range(10)

# functions declared in include/md.h (checked by the CPU test-suite)
EXPORTS = ["md_abi_version", "md_status_string", "md_create", "md_create_batch", "md_build_neighbours",
           "md_eam_forces", "md_step", "md_step_io", "md_set_graph", "md_energy", "md_replica_energies", "md_get",
           "md_set_state", "md_tune", "md_set_profiling", "md_get_profile", "md_get_passes", "md_selftest_timeout",
           "md_neighbours_noalloc", "md_set_thermostat", "md_get_thermostat", "md_set_surrogate", "md_sur_get_params", "md_sur_standardize",
           "md_sur_get", "md_sur_set_reference", "md_sur_loss_grad", "md_sur_train", "md_measure_fp64_peak",
           "md_last_error", "md_destroy"]


class md_potential(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_species", C.c_int32),
                ("atomic_numbers", C.POINTER(C.c_int32)), ("masses_amu", C.POINTER(C.c_double)),
                ("fs", C.c_double * 7), ("n_knots", C.c_int32), ("r_min", C.c_double),
                ("r_cut", C.c_double), ("rho_min", C.c_double), ("rho_max", C.c_double),
                ("tables", C.POINTER(C.c_double))]


class md_config(C.Structure):
    _fields_ = [("n_atoms", C.c_int64), ("h", C.c_double * 9), ("skin", C.c_double),
                ("k_max", C.c_int32), ("rebuild_every", C.c_int32), ("dt_fs", C.c_double),
                ("precision", C.c_int32), ("strict_skin", C.c_int32), ("strain_rate_zz", C.c_double),
                ("stream", C.c_void_p), ("lanes_per_atom", C.c_int32), ("passes", C.c_int32),
                ("integrator", C.c_int32)]


MD_PASSES_AUTO, MD_PASSES_LIST, MD_PASSES_STAGED, MD_PASSES_CELLS, MD_PASSES_HALF = 0, 1, 2, 3, 4
MD_INTEGRATOR_VERLET, MD_INTEGRATOR_PC3 = 0, 1
INTEGRATORS = {"verlet": MD_INTEGRATOR_VERLET, "pc3": MD_INTEGRATOR_PC3}
PASSES = {"auto": MD_PASSES_AUTO, "list": MD_PASSES_LIST, "staged": MD_PASSES_STAGED, "cells": MD_PASSES_CELLS,
          "half": MD_PASSES_HALF}
WALKS = {v: k for k, v in PASSES.items()}


class md_passes(C.Structure):
    _fields_ = [("walk", C.c_int32), ("cells_per_group", C.c_int32), ("groups", C.c_int32),
                ("capacity", C.c_int32), ("last_max", C.c_int32), ("active", C.c_int32),
                ("stage_buffers", C.c_int32)]


class md_surrogate(C.Structure):
    _fields_ = [("nb", C.c_int32), ("h1", C.c_int32), ("h2", C.c_int32), ("net", C.c_int32),
                ("mu0", C.c_double), ("dmu", C.c_double), ("width", C.c_double), ("rd", C.c_double)]


class md_energies(C.Structure):
    _fields_ = [("pe", C.c_double), ("ke", C.c_double), ("te", C.c_double), ("temperature", C.c_double),
                ("virial", C.c_double * 9), ("pressure_gpa", C.c_double), ("momentum", C.c_double * 3),
                ("volume", C.c_double), ("box", C.c_double * 3), ("step", C.c_int64),
                ("n_rebuilds", C.c_int64), ("max_neighbours", C.c_int32), ("pad", C.c_int32),
                ("range_violations", C.c_int64)]


class md_profile(C.Structure):
    _fields_ = [("launches", C.c_int64), ("n_kick", C.c_int64), ("n_rebuild", C.c_int64),
                ("n_density", C.c_int64), ("n_force", C.c_int64), ("ms_kick", C.c_double),
                ("ms_rebuild", C.c_double), ("ms_density", C.c_double), ("ms_force", C.c_double),
                ("ms_rebuild_part", C.c_double * 9)]


class MDError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{status_string(status)} ({status}): {message}")
        self.status = status


_lib = None


def lib():
    """Load libmd.so; raises if it has not been built (no CPU fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        P, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        L.md_abi_version.restype = i32
        L.md_status_string.restype = C.c_char_p
        L.md_status_string.argtypes = [C.c_int]
        L.md_create.restype = C.c_int
        L.md_create.argtypes = [C.POINTER(md_config), C.POINTER(md_potential), P, P, P, i32, C.POINTER(P)]
        L.md_create_batch.restype = C.c_int
        L.md_create_batch.argtypes = [i32, C.POINTER(md_config), C.POINTER(md_potential), P, P, P, i32,
                                      C.POINTER(P)]
        L.md_replica_energies.restype = C.c_int
        L.md_replica_energies.argtypes = [P, C.POINTER(md_energies)]
        L.md_selftest_timeout.restype = C.c_int
        L.md_selftest_timeout.argtypes = [P]
        L.md_set_graph.restype = C.c_int
        L.md_set_graph.argtypes = [P, i32]
        L.md_build_neighbours.restype = C.c_int
        L.md_build_neighbours.argtypes = [P]
        L.md_eam_forces.restype = C.c_int
        L.md_eam_forces.argtypes = [P, C.POINTER(C.c_double)]
        L.md_step.restype = C.c_int
        L.md_step.argtypes = [P, i32]
        L.md_energy.restype = C.c_int
        L.md_energy.argtypes = [P, C.POINTER(md_energies)]
        L.md_get.restype = C.c_int
        L.md_get.argtypes = [P, i32, P, i32]
        L.md_set_state.restype = C.c_int
        L.md_set_state.argtypes = [P, P, P, P, i32]
        L.md_step_io.restype = C.c_int
        L.md_step_io.argtypes = [P, i32, P, P, P, P, P, P, C.POINTER(md_energies), i32]
        L.md_tune.restype = C.c_int
        L.md_tune.argtypes = [P, C.POINTER(C.c_int32)]
        L.md_set_profiling.restype = C.c_int
        L.md_set_profiling.argtypes = [P, i32]
        L.md_get_profile.restype = C.c_int
        L.md_get_profile.argtypes = [P, C.POINTER(md_profile)]
        L.md_get_passes.restype = C.c_int
        L.md_get_passes.argtypes = [P, C.POINTER(md_passes)]
        L.md_neighbours_noalloc.restype = C.c_int
        L.md_neighbours_noalloc.argtypes = [P, i64, P, C.c_double, i32, P, P, P]
        L.md_set_thermostat.restype = C.c_int
        L.md_set_thermostat.argtypes = [P, i32, P, P]
        L.md_get_thermostat.restype = C.c_int
        L.md_get_thermostat.argtypes = [P, P]
        L.md_set_surrogate.restype = C.c_int
        L.md_set_surrogate.argtypes = [P, C.POINTER(md_surrogate), P, P, P]
        L.md_sur_get_params.restype = C.c_int
        L.md_sur_get_params.argtypes = [P, P, P, P]
        L.md_sur_standardize.restype = C.c_int
        L.md_sur_standardize.argtypes = [P]
        L.md_sur_get.restype = C.c_int
        L.md_sur_get.argtypes = [P, i32, P, i32]
        L.md_sur_set_reference.restype = C.c_int
        L.md_sur_set_reference.argtypes = [P, P, P, i32]
        L.md_sur_loss_grad.restype = C.c_int
        L.md_sur_loss_grad.argtypes = [P, i32, i32, C.c_double, C.c_double, P, P]
        L.md_sur_train.restype = C.c_int
        L.md_sur_train.argtypes = [P, i32, i32, i32, i32, C.c_double, C.c_double, C.c_double, C.c_uint64, P]
        L.md_measure_fp64_peak.restype = C.c_int
        L.md_measure_fp64_peak.argtypes = [i64, C.POINTER(C.c_double), C.POINTER(C.c_double), P]
        L.md_last_error.restype = C.c_char_p
        L.md_last_error.argtypes = [P]
        L.md_destroy.restype = None
        L.md_destroy.argtypes = [P]
        _lib = L
    return _lib


def status_string(s: int) -> str:
    return lib().md_status_string(int(s)).decode()


def _ptr(a):
    """(pointer, on_device, keepalive) for a numpy array, a torch tensor or None."""
    if a is None:
        return None, 0, None
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr()), (1 if a.is_cuda else 0), a
    return C.c_void_p(a.ctypes.data), 0, a


def _check(ctx, status):
    if status != MD_OK:
        msg = lib().md_last_error(ctx).decode() if ctx else ""
        raise MDError(status, msg)


def md_create(config: md_config, potential: md_potential, pos, vel=None, species=None):
    p, dev, _k1 = _ptr(pos)
    v, dev_v, _k2 = _ptr(vel)
    s, dev_s, _k3 = _ptr(species)
    if vel is not None and dev_v != dev or species is not None and dev_s != dev:
        raise ValueError("pos, vel and species must all be host or all device arrays")
    out = C.c_void_p()
    st = lib().md_create(C.byref(config), C.byref(potential), p, v, s, dev, C.byref(out))
    if st != MD_OK:
        raise MDError(st, "md_create failed")
    return out


def md_create_batch(configs, potential: md_potential, positions, velocities=None, species=None):
    """One context for a batch of replicas: configs is a sequence of md_config, the others
    sequences of host arrays (one per replica)."""
    n = len(configs)
    cfgs = (md_config * n)(*configs)
    keep = [np.ascontiguousarray(a, dtype=np.float64) for a in positions]
    pp = (C.c_void_p * n)(*[a.ctypes.data for a in keep])
    vv = ss = None
    if velocities is not None:
        keep_v = [np.ascontiguousarray(a, dtype=np.float64) for a in velocities]
        vv = (C.c_void_p * n)(*[a.ctypes.data for a in keep_v])
    if species is not None:
        keep_s = [np.ascontiguousarray(a, dtype=np.int32) for a in species]
        ss = (C.c_void_p * n)(*[a.ctypes.data for a in keep_s])
    out = C.c_void_p()
    st = lib().md_create_batch(n, cfgs, C.byref(potential), pp, vv, ss, 0, C.byref(out))
    if st != MD_OK:
        raise MDError(st, "md_create_batch failed")
    return out


def md_replica_energies(ctx, n_replicas: int) -> list:
    arr = (md_energies * n_replicas)()
    _check(ctx, lib().md_replica_energies(ctx, arr))
    return [dict(pe=e.pe, ke=e.ke, te=e.te, temperature=e.temperature, momentum=np.array(e.momentum[:]),
                 box=np.array(e.box[:]), volume=e.volume) for e in arr]


def md_selftest_timeout(ctx) -> int:
    """Run the bounded-wait self-test; returns the md_status (MD_ERR_TIMEOUT expected)."""
    return lib().md_selftest_timeout(ctx)


def md_set_graph(ctx, on: bool):
    _check(ctx, lib().md_set_graph(ctx, 1 if on else 0))


def md_build_neighbours(ctx):
    _check(ctx, lib().md_build_neighbours(ctx))


def md_eam_forces(ctx) -> float:
    pe = C.c_double()
    _check(ctx, lib().md_eam_forces(ctx, C.byref(pe)))
    return pe.value


def md_step(ctx, n_steps: int):
    _check(ctx, lib().md_step(ctx, int(n_steps)))


def _energy_dict(e) -> dict:
    return dict(pe=e.pe, ke=e.ke, te=e.te, temperature=e.temperature,
                virial=np.array(e.virial[:]).reshape(3, 3), pressure_gpa=e.pressure_gpa,
                momentum=np.array(e.momentum[:]), volume=e.volume, box=np.array(e.box[:]),
                step=e.step, n_rebuilds=e.n_rebuilds, max_neighbours=e.max_neighbours,
                range_violations=e.range_violations)


def md_energy(ctx) -> dict:
    e = md_energies()
    _check(ctx, lib().md_energy(ctx, C.byref(e)))
    return _energy_dict(e)


def md_step_io(ctx, n_steps: int, pos_in=None, vel_in=None, force_in=None, pos_out=None, vel_out=None,
               force_out=None) -> dict:
    """State in, n_steps steps, state out and the energies, with one synchronisation."""
    arrs = (pos_in, vel_in, force_in, pos_out, vel_out, force_out)
    ptrs = [_ptr(a) for a in arrs]
    flags = {p[1] for p, a in zip(ptrs, arrs) if a is not None}
    if len(flags) > 1:
        raise ValueError("state arrays must all be host or all device arrays")
    e = md_energies()
    _check(ctx, lib().md_step_io(ctx, int(n_steps), *[p[0] for p in ptrs], C.byref(e), flags.pop() if flags else 0))
    return _energy_dict(e)


def md_get(ctx, what: int, dst):
    p, dev, _k = _ptr(dst)
    _check(ctx, lib().md_get(ctx, int(what), p, dev))
    return dst


def md_set_state(ctx, pos=None, vel=None, force=None):
    devs = [_ptr(a) for a in (pos, vel, force)]
    flags = {d[1] for d, a in zip(devs, (pos, vel, force)) if a is not None}
    if len(flags) > 1:
        raise ValueError("state arrays must all be host or all device arrays")
    _check(ctx, lib().md_set_state(ctx, devs[0][0], devs[1][0], devs[2][0], flags.pop() if flags else 0))


def md_tune(ctx) -> int:
    lanes = C.c_int32()
    _check(ctx, lib().md_tune(ctx, C.byref(lanes)))
    return lanes.value


def md_set_profiling(ctx, on: bool):
    _check(ctx, lib().md_set_profiling(ctx, 1 if on else 0))


def md_get_profile(ctx) -> dict:
    p = md_profile()
    _check(ctx, lib().md_get_profile(ctx, C.byref(p)))
    d = {k: getattr(p, k) for k, _ in md_profile._fields_}
    d["ms_rebuild_part"] = list(p.ms_rebuild_part)
    return d


def md_get_passes(ctx) -> dict:
    p = md_passes()
    _check(ctx, lib().md_get_passes(ctx, C.byref(p)))
    d = {k: getattr(p, k) for k, _ in md_passes._fields_}
    d["walk"] = WALKS[d["walk"]]
    return d


def md_neighbours_noalloc(pos, box, r_list: float, k_max: int, count, nbr_list, stream=None) -> int:
    """Neighbour list into caller-owned device tensors, with no device allocation by the
    library (for callers that cannot allocate); returns the md_status code."""
    b = np.ascontiguousarray(box, dtype=np.float64)
    return lib().md_neighbours_noalloc(C.c_void_p(pos.data_ptr()), int(pos.shape[0]), C.c_void_p(b.ctypes.data),
                                       float(r_list), int(k_max), C.c_void_p(count.data_ptr()),
                                       C.c_void_p(nbr_list.data_ptr()), C.c_void_p(stream) if stream else None)


def md_set_thermostat(ctx, on: bool, t_kelvin=None, tau_fs=None):
    if not on:
        _check(ctx, lib().md_set_thermostat(ctx, 0, None, None))
        return
    t = np.ascontiguousarray(np.atleast_1d(t_kelvin), dtype=np.float64)
    tau = np.ascontiguousarray(np.atleast_1d(tau_fs), dtype=np.float64)
    _check(ctx, lib().md_set_thermostat(ctx, 1, t.ctypes.data, tau.ctypes.data))


def md_get_thermostat(ctx, n_replicas: int = 1):
    out = np.zeros((n_replicas, 4))
    _check(ctx, lib().md_get_thermostat(ctx, out.ctypes.data))
    return out


def md_set_surrogate(ctx, spec: md_surrogate, theta, gmu=None, ginv=None):
    th = np.ascontiguousarray(theta, dtype=np.float32)
    mu = None if gmu is None else np.ascontiguousarray(gmu, dtype=np.float32)
    iv = None if ginv is None else np.ascontiguousarray(ginv, dtype=np.float32)
    _check(ctx, lib().md_set_surrogate(ctx, C.byref(spec), th.ctypes.data,
                                       None if mu is None else mu.ctypes.data,
                                       None if iv is None else iv.ctypes.data))


def md_sur_get_params(ctx):
    th, mu, iv = (np.empty(MD_SUR_PARAMS, np.float32), np.empty(MD_SUR_NB, np.float32),
                  np.empty(MD_SUR_NB, np.float32))
    _check(ctx, lib().md_sur_get_params(ctx, th.ctypes.data, mu.ctypes.data, iv.ctypes.data))
    return th, mu, iv


def md_sur_standardize(ctx):
    _check(ctx, lib().md_sur_standardize(ctx))


def md_sur_get(ctx, what: int, dst):
    p, dev, _k = _ptr(dst)
    _check(ctx, lib().md_sur_get(ctx, int(what), p, dev))
    return dst


def md_sur_set_reference(ctx, e_ref, f_ref):
    e = np.ascontiguousarray(e_ref, dtype=np.float64)
    f = np.ascontiguousarray(f_ref, dtype=np.float64)
    _check(ctx, lib().md_sur_set_reference(ctx, e.ctypes.data, f.ctypes.data, 0))


def md_sur_loss_grad(ctx, rep_begin: int, rep_end: int, w_e: float, w_f: float):
    loss, grad = np.zeros(2), np.empty(MD_SUR_PARAMS, np.float32)
    _check(ctx, lib().md_sur_loss_grad(ctx, int(rep_begin), int(rep_end), float(w_e), float(w_f),
                                       loss.ctypes.data, grad.ctypes.data))
    return loss, grad


def md_sur_train(ctx, n_iter: int, rep_begin: int, rep_end: int, batch_reps: int, lr: float, w_e: float,
                 w_f: float, seed: int):
    loss = np.zeros(2)
    _check(ctx, lib().md_sur_train(ctx, int(n_iter), int(rep_begin), int(rep_end), int(batch_reps), float(lr),
                                   float(w_e), float(w_f), int(seed) & 0xFFFFFFFFFFFFFFFF, loss.ctypes.data))
    return loss


def md_measure_fp64_peak(iters: int = 20000, stream=None):
    """(TFLOP/s, ms) of the library's FP64 FMA-chain kernel on the current device."""
    tf, ms = C.c_double(), C.c_double()
    st = lib().md_measure_fp64_peak(int(iters), C.byref(tf), C.byref(ms), C.c_void_p(stream) if stream else None)
    if st != MD_OK:
        raise MDError(st, "md_measure_fp64_peak failed")
    return tf.value, ms.value


def md_last_error(ctx) -> str:
    return lib().md_last_error(ctx).decode()


def md_destroy(ctx):
    if ctx:
        lib().md_destroy(ctx)


# ---------------------------------------------------------------------------
def make_potential(pot: _inputs.Potential):
    """md_potential view of an inputs.Potential (returns the struct and the arrays it points to)."""
    an = np.ascontiguousarray(pot.atomic_numbers, dtype=np.int32)
    ms = np.ascontiguousarray(pot.masses, dtype=np.float64)
    tb = np.ascontiguousarray(pot.tables if pot.tables.size else np.zeros(1), dtype=np.float64)
    s = md_potential()
    s.kind, s.n_species = int(pot.kind), int(pot.n_species)
    s.atomic_numbers = an.ctypes.data_as(C.POINTER(C.c_int32))
    s.masses_amu = ms.ctypes.data_as(C.POINTER(C.c_double))
    for k in range(7):
        s.fs[k] = float(pot.fs[k])
    s.n_knots = int(pot.n_knots)
    s.r_min, s.r_cut = float(pot.r_min), float(pot.r_cut)
    s.rho_min, s.rho_max = float(pot.rho_min), float(pot.rho_max)
    s.tables = tb.ctypes.data_as(C.POINTER(C.c_double))
    return s, (an, ms, tb)


def make_config(n_atoms, box, skin, k_max, dt_fs, precision=MD_PREC_FP64, rebuild_every=0,
                strict_skin=False, strain_rate_zz=0.0, stream=None, lanes_per_atom=0, passes="auto",
                integrator="verlet"):
    c = md_config()
    c.n_atoms = int(n_atoms)
    for k in range(9):
        c.h[k] = 0.0
    for k in range(3):
        c.h[4 * k] = float(box[k])
    c.skin, c.k_max, c.rebuild_every, c.dt_fs = float(skin), int(k_max), int(rebuild_every), float(dt_fs)
    c.precision, c.strict_skin, c.strain_rate_zz = int(precision), int(bool(strict_skin)), float(strain_rate_zz)
    c.stream = C.c_void_p(stream) if stream else None
    c.lanes_per_atom = int(lanes_per_atom)
    c.passes = PASSES[passes]
    c.integrator = INTEGRATORS[integrator]
    return c


class System:
    """One simulated system on the GPU (a context of libmd.so)."""

    def __init__(self, w: _inputs.Workload, precision: str = "fp64", rebuild_every: int = 0,
                 strict_skin: bool = False, stream=None, device_inputs: bool = False, k_max=None,
                 lanes_per_atom: int = 0, passes: str = "auto", integrator: str = "verlet"):
        prec = PRECISIONS[precision]
        self.n = w.n_atoms
        self.k_max = int(k_max or w.k_max)
        self.config = make_config(w.n_atoms, w.box, w.skin, self.k_max, w.dt_fs, prec, rebuild_every,
                                  strict_skin, w.strain_rate_zz, stream, lanes_per_atom, passes, integrator)
        pot, keep = make_potential(w.potential)
        pos = np.ascontiguousarray(w.pos, dtype=np.float64)
        vel = np.ascontiguousarray(w.vel, dtype=np.float64)
        spc = np.ascontiguousarray(w.species, dtype=np.int32)
        if device_inputs:
            import torch
            pos, vel, spc = (torch.from_numpy(a).cuda() for a in (pos, vel, spc))
            torch.cuda.synchronize()
        self.ctx = md_create(self.config, pot, pos, vel, spc)
        self.n_replicas = 1
        del keep

    def build_neighbours(self):
        md_build_neighbours(self.ctx)

    def eam_forces(self) -> float:
        return md_eam_forces(self.ctx)

    def step(self, n: int = 1):
        md_step(self.ctx, n)

    def energy(self) -> dict:
        return md_energy(self.ctx)

    def get(self, what: int, out=None):
        if out is None:
            if what in (MD_GET_POS, MD_GET_VEL, MD_GET_FORCE, MD_GET_IMAGE):
                out = np.empty((self.n, 3), np.float64)
            elif what in (MD_GET_RHO, MD_GET_EATOM, MD_GET_DF):
                out = np.empty(self.n, np.float64)
            elif what in (MD_GET_NBR_COUNT, MD_GET_SPECIES):
                out = np.empty(self.n, np.int32)
            elif what == MD_GET_NBR_LIST:
                out = np.empty((self.n, self.k_max), np.int32)
            else:
                raise ValueError(what)
        return md_get(self.ctx, what, out)

    def positions(self):
        return self.get(MD_GET_POS)

    def velocities(self):
        return self.get(MD_GET_VEL)

    def forces(self):
        return self.get(MD_GET_FORCE)

    def neighbours(self):
        return self.get(MD_GET_NBR_COUNT), self.get(MD_GET_NBR_LIST)

    def tune(self) -> int:
        return md_tune(self.ctx)

    def set_graph(self, on: bool = True):
        md_set_graph(self.ctx, on)

    def replica_energies(self) -> list:
        return md_replica_energies(self.ctx, self.n_replicas)

    def set_profiling(self, on: bool = True):
        md_set_profiling(self.ctx, on)

    def profile(self) -> dict:
        return md_get_profile(self.ctx)

    def passes(self) -> dict:
        """The step kernel's neighbour walk: walk ("list", "staged", "cells" or "half": the walk prepared),
        cells_per_group, groups, capacity (atoms per stage buffer), last_max (largest group
        neighbourhood at the last build), active (the next md_step walks the prepared groups),
        stage_buffers (2 to 4: the next groups are staged while one is computed)."""
        return md_get_passes(self.ctx)

    def set_state(self, pos=None, vel=None, force=None):
        md_set_state(self.ctx, pos, vel, force)

    def step_io(self, n: int = 1, pos_in=None, vel_in=None, force_in=None, pos_out=None, vel_out=None,
                force_out=None) -> dict:
        """md_step_io: set the state, take n steps, read the state back; returns the energies."""
        return md_step_io(self.ctx, n, pos_in, vel_in, force_in, pos_out, vel_out, force_out)

    def set_thermostat(self, t_kelvin, tau_fs):
        """Nose-Hoover thermostat at t_kelvin with relaxation time tau_fs (scalars or one per
        replica); the library sets the thermal inertia Q (see thermostat())."""
        t = np.broadcast_to(np.asarray(t_kelvin, dtype=np.float64), (self.n_replicas,)).copy()
        tau = np.broadcast_to(np.asarray(tau_fs, dtype=np.float64), (self.n_replicas,)).copy()
        md_set_thermostat(self.ctx, True, t, tau)

    def thermostat(self):
        """[n_replicas][4]: pi (1/fs), xi, Q (eV fs^2), the conserved H' (eV)."""
        return md_get_thermostat(self.ctx, self.n_replicas)

    def close(self):
        if self.ctx:
            md_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch(System):
    """A batch of independent replicas in one context (md_create_batch)."""

    def __init__(self, workloads, precision: str = "mixed", rebuild_every: int = 0, stream=None,
                 k_max=None, lanes_per_atom: int = 0, integrator: str = "verlet", passes: str = "auto"):
        prec = PRECISIONS[precision]
        w0 = workloads[0]
        self.k_max = int(k_max or max(w.k_max for w in workloads))
        cfgs = [make_config(w.n_atoms, w.box, w0.skin, self.k_max, w0.dt_fs, prec, rebuild_every, False,
                            w0.strain_rate_zz, stream, lanes_per_atom, passes=passes, integrator=integrator)
                for w in workloads]
        pot, keep = make_potential(w0.potential)
        self.ctx = md_create_batch(cfgs, pot, [w.pos for w in workloads], [w.vel for w in workloads],
                                   [w.species for w in workloads])
        self.n = sum(w.n_atoms for w in workloads)
        self.n_replicas = len(workloads)
        self.offsets = np.concatenate([[0], np.cumsum([w.n_atoms for w in workloads])])
        del keep


# ----------------------------------------------------------------------------- surrogate
def make_surrogate(spec, net: str = "bf16"):
    s = md_surrogate()
    s.nb, s.h1, s.h2 = int(spec["nb"]), int(spec["h1"]), int(spec["h2"])
    s.net = MD_SUR_BF16 if net == "bf16" else MD_SUR_FP32
    s.mu0, s.dmu, s.width, s.rd = float(spec["mu0"]), float(spec["dmu"]), float(spec["width"]), float(spec["rd"])
    return s


class _SurrogateMixin:
    def set_surrogate(self, theta, gmu=None, ginv=None, net: str = "bf16"):
        self.sur_net = net
        md_set_surrogate(self.ctx, make_surrogate(self.sur_spec, net), theta, gmu, ginv)

    def sur_params(self):
        return md_sur_get_params(self.ctx)

    def standardize(self):
        md_sur_standardize(self.ctx)

    def descriptors(self):
        return md_sur_get(self.ctx, MD_SUR_GET_G, np.empty((self.n, MD_SUR_NB), np.float32))

    def dE_dG(self):
        return md_sur_get(self.ctx, MD_SUR_GET_DEDG, np.empty((self.n, MD_SUR_NB), np.float32))

    def set_reference(self, e_ref, f_ref):
        md_sur_set_reference(self.ctx, e_ref, f_ref)

    def loss_grad(self, rep_begin=0, rep_end=None, w_e=1.0, w_f=1.0):
        return md_sur_loss_grad(self.ctx, rep_begin, self.n_replicas if rep_end is None else rep_end, w_e, w_f)

    def train(self, n_iter, batch_reps, lr, w_e=1.0, w_f=1.0, seed=0, rep_begin=0, rep_end=None):
        rep_end = self.n_replicas if rep_end is None else rep_end
        return md_sur_train(self.ctx, n_iter, rep_begin, rep_end, batch_reps, lr, w_e, w_f, seed)


class SurrogateSystem(_SurrogateMixin, System):
    """A system whose force field is the learned surrogate (kind MD_POT_SURROGATE)."""

    def __init__(self, w: _inputs.Workload, theta=None, gmu=None, ginv=None, net: str = "bf16",
                 spec=None, **kw):
        self.sur_spec = dict(spec or _inputs.SUR_FE)
        super().__init__(_inputs.as_surrogate(w, self.sur_spec), **kw)
        if theta is not None:
            self.set_surrogate(theta, gmu, ginv, net)


class SurrogateBatch(_SurrogateMixin, Batch):
    """Training frames as a batch of replicas with the surrogate force field."""

    def __init__(self, workloads, theta=None, gmu=None, ginv=None, net: str = "fp32", spec=None, **kw):
        self.sur_spec = dict(spec or _inputs.SUR_FE)
        super().__init__([_inputs.as_surrogate(w, self.sur_spec) for w in workloads], **kw)
        if theta is not None:
            self.set_surrogate(theta, gmu, ginv, net)
