"""FP64 CPU oracle for the EAM hot path (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package.  It loads oracle/_build/liboracle.so (plain C, see moldy_oracle.c),
which shares no code with the CUDA library.  Inputs are numpy arrays; the
potential is the data object from paper_1107_2619_gb300.inputs (plain data).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class OrcPotential(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_species", C.c_int32), ("n_knots", C.c_int32),
                ("pad", C.c_int32), ("fs", C.c_double * 7), ("r_min", C.c_double),
                ("r_cut", C.c_double), ("rho_min", C.c_double), ("rho_max", C.c_double),
                ("tables", C.POINTER(C.c_double))]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        i64, i32, dbl, P = C.c_int64, C.c_int32, C.c_double, C.c_void_p
        L.orc_neighbours_brute.restype = i32
        L.orc_neighbours_brute.argtypes = [i64, P, P, dbl, i32, P, P]
        L.orc_neighbours_cells.restype = i32
        L.orc_neighbours_cells.argtypes = [i64, P, P, dbl, i32, P, P]
        L.orc_eam_forces.restype = i64
        L.orc_eam_forces.argtypes = [i64, P, P, P, P, P, P, i32, P, P, P, P, P, P]
        L.orc_run_pc3.restype = i64
        L.orc_run_pc3.argtypes = [i64, P, P, P, P, P, P, dbl, i32, dbl, i32, i32, P, i32, P, P, P]
        L.orc_eam_error_scales.restype = None
        L.orc_eam_error_scales.argtypes = [i64, P, P, P, P, P, P, i32, P, P, P, P, P]
        L.orc_eam_forces_half.restype = i64
        L.orc_eam_forces_half.argtypes = [i64, P, P, P, P, P, P, i32, P, P]
        L.orc_kinetic.restype = None
        L.orc_kinetic.argtypes = [i64, P, P, P, P, P, P, P]
        L.orc_pressure_gpa.restype = dbl
        L.orc_pressure_gpa.argtypes = [P, P, P]
        L.orc_run_vv.restype = i64
        L.orc_run_vv.argtypes = [i64, P, P, P, P, P, P, dbl, i32, dbl, i32, i32, dbl, P, i32, P, P, P]
        L.orc_pair_value.restype = dbl
        L.orc_pair_value.argtypes = [P, C.c_int, C.c_int, C.c_int, dbl, P]
        L.orc_embed_value.restype = dbl
        L.orc_embed_value.argtypes = [P, C.c_int, dbl, P]
        L.orc_sur_descriptors.restype = None
        L.orc_sur_descriptors.argtypes = [i64, P, P, P, P, i32, P, P]
        L.orc_sur_mlp.restype = None
        L.orc_sur_mlp.argtypes = [i64, P, P, P, P, P]
        L.orc_sur_forces.restype = None
        L.orc_sur_forces.argtypes = [i64, P, P, P, P, i32, P, P, P]
        L.orc_sur_loss_grad.restype = C.c_double
        L.orc_sur_loss_grad.argtypes = [i32, P, P, P, P, P, i32, P, P, P, P, C.c_double, C.c_double, P, P]
        L.orc_run_nvt.restype = i64
        L.orc_run_nvt.argtypes = [i64, P, P, P, P, P, P, dbl, i32, dbl, i32, dbl, P, P, i32, P]
        L.orc_num_threads.restype = C.c_int
        L.orc_set_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class _Pot:
    """Keeps the C struct and the table array it points to alive together."""

    def __init__(self, pot):
        self.tables = _f64(pot.tables if pot.tables.size else np.zeros(1))
        self.s = OrcPotential()
        self.s.kind = int(pot.kind)
        self.s.n_species = int(pot.n_species)
        self.s.n_knots = int(pot.n_knots)
        for k in range(7):
            self.s.fs[k] = float(pot.fs[k])
        self.s.r_min, self.s.r_cut = float(pot.r_min), float(pot.r_cut)
        self.s.rho_min, self.s.rho_max = float(pot.rho_min), float(pot.rho_max)
        self.s.tables = self.tables.ctypes.data_as(C.POINTER(C.c_double))

    @property
    def ref(self):
        return C.cast(C.pointer(self.s), C.c_void_p)


def num_threads() -> int:
    return lib().orc_num_threads()


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def neighbours(pos, box, r_list, k_max, method="cells"):
    """Full neighbour list: (count[N], list[N,k_max] padded with -1, max_count).
    method 'brute' is the O(N^2) definition; 'cells' the link-cell method."""
    pos, box = _f64(pos), _f64(box)
    n = pos.shape[0]
    count = np.zeros(n, np.int32)
    nl = np.full((n, k_max), -1, np.int32)
    f = lib().orc_neighbours_brute if method == "brute" else lib().orc_neighbours_cells
    m = f(n, _p(pos), _p(box), float(r_list), int(k_max), _p(count), _p(nl))
    if m < 0:
        raise ValueError("link cells need at least 3 cells per box edge")
    return count, nl, int(m)


def eam_forces(pos, species, box, pot, count, nl):
    pos, box, species, count, nl = _f64(pos), _f64(box), _i32(species), _i32(count), _i32(nl)
    n, k_max = nl.shape
    P = _Pot(pot)
    out = dict(rho=np.zeros(n), dF=np.zeros(n), force=np.zeros((n, 3)), e_atom=np.zeros(n),
               virial=np.zeros(9), pe=np.zeros(1))
    viol = lib().orc_eam_forces(n, _p(pos), _p(species), _p(box), P.ref, _p(count), _p(nl), k_max,
                                _p(out["rho"]), _p(out["dF"]), _p(out["force"]), _p(out["e_atom"]),
                                _p(out["virial"]), _p(out["pe"]))
    out["pe"] = float(out["pe"][0])
    out["virial"] = out["virial"].reshape(3, 3)
    out["range_violations"] = int(viol)
    return out


def eam_error_scales(pos, species, box, pot, count, nl, dF):
    """Per-atom scales of the force sum (moldy_oracle.c orc_eam_error_scales): m (sum of the
    absolute pair terms), q (their radial sensitivity r |d/dr|), e (through F'') and c (the
    quadratic and cubic terms of the table cubics' derivatives, knot tables only)."""
    pos, box, species, count, nl, dF = _f64(pos), _f64(box), _i32(species), _i32(count), _i32(nl), _f64(dF)
    n, k_max = nl.shape
    P = _Pot(pot)
    m, q, e, c = np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(n)
    lib().orc_eam_error_scales(n, _p(pos), _p(species), _p(box), P.ref, _p(count), _p(nl), k_max, _p(dF),
                               _p(m), _p(q), _p(e), _p(c))
    return dict(m=m, q=q, e=e, c=c)


def eam_forces_half(pos, species, box, pot, count, nl):
    pos, box, species, count, nl = _f64(pos), _f64(box), _i32(species), _i32(count), _i32(nl)
    n, k_max = nl.shape
    P = _Pot(pot)
    force, pe = np.zeros((n, 3)), np.zeros(1)
    lib().orc_eam_forces_half(n, _p(pos), _p(species), _p(box), P.ref, _p(count), _p(nl), k_max,
                              _p(force), _p(pe))
    return force, float(pe[0])


def forces(pos, species, box, pot, skin=0.3, k_max=64, method="cells"):
    """Neighbour list + Eq. (1) forces in one call."""
    count, nl, m = neighbours(pos, box, pot.r_cut + skin, k_max, method)
    if m > k_max:
        raise ValueError(f"neighbour list overflow: {m} > {k_max}")
    out = eam_forces(pos, species, box, pot, count, nl)
    out["count"], out["list"] = count, nl
    return out


def kinetic(vel, species, masses):
    vel, species, masses = _f64(vel), _i32(species), _f64(masses)
    ke, t = np.zeros(1), np.zeros(1)
    p, kt = np.zeros(3), np.zeros(9)
    lib().orc_kinetic(vel.shape[0], _p(vel), _p(species), _p(masses), _p(ke), _p(t), _p(p), _p(kt))
    return dict(ke=float(ke[0]), temperature=float(t[0]), momentum=p, kin_tensor=kt.reshape(3, 3))


def pressure_gpa(kin_tensor, virial, box):
    return float(lib().orc_pressure_gpa(_p(_f64(kin_tensor)), _p(_f64(virial)), _p(_f64(box))))


def run_vv(pos, vel, species, masses, box, pot, dt_fs, n_steps, skin, k_max, rebuild_every=0,
           strain_rate_zz=0.0, force=None):
    """Velocity Verlet from (pos, vel); returns the final state and per-step (PE, KE)."""
    pos, vel, box = _f64(pos).copy(), _f64(vel).copy(), _f64(box).copy()
    species, masses = _i32(species), _f64(masses)
    n = pos.shape[0]
    f = np.zeros((n, 3)) if force is None else _f64(force).copy()
    energies = np.zeros((max(n_steps, 1), 2))
    nreb, mc = np.zeros(1, np.int32), np.zeros(1, np.int32)
    P = _Pot(pot)
    viol = lib().orc_run_vv(n, _p(pos), _p(vel), _p(species), _p(masses), _p(box), P.ref, float(dt_fs),
                            int(n_steps), float(skin), int(k_max), int(rebuild_every),
                            float(strain_rate_zz), _p(f), 0 if force is None else 1, _p(energies),
                            _p(nreb), _p(mc))
    if int(mc[0]) > k_max:
        raise ValueError(f"neighbour list overflow: {int(mc[0])} > {k_max}")
    return dict(pos=pos, vel=vel, force=f, box=box, energies=energies[:n_steps],
                n_rebuilds=int(nreb[0]), max_count=int(mc[0]), range_violations=int(viol))


def pair_value(pot, which, a, b, r):
    P = _Pot(pot)
    d = np.zeros(1)
    v = lib().orc_pair_value(P.ref, which, a, b, float(r), _p(d))
    return float(v), float(d[0])


def embed_value(pot, a, rho):
    P = _Pot(pot)
    d = np.zeros(1)
    v = lib().orc_embed_value(P.ref, a, float(rho), _p(d))
    return float(v), float(d[0])


# ----------------------------------------------------------------------------- surrogate
class OrcSurSpec(C.Structure):
    _fields_ = [("nb", C.c_int32), ("h1", C.c_int32), ("h2", C.c_int32), ("pad", C.c_int32),
                ("mu0", C.c_double), ("dmu", C.c_double), ("width", C.c_double), ("rd", C.c_double)]


def _sur_spec(spec):
    s = OrcSurSpec()
    s.nb, s.h1, s.h2 = int(spec["nb"]), int(spec["h1"]), int(spec["h2"])
    s.mu0, s.dmu, s.width, s.rd = float(spec["mu0"]), float(spec["dmu"]), float(spec["width"]), float(spec["rd"])
    return s


def sur_descriptors(pos, box, count, nl, spec):
    pos, box, count, nl = _f64(pos), _f64(box), _i32(count), _i32(nl)
    n, k_max = nl.shape
    sp = _sur_spec(spec)
    G = np.zeros((n, sp.nb))
    lib().orc_sur_descriptors(n, _p(pos), _p(box), _p(count), _p(nl), k_max, C.byref(sp), _p(G))
    return G


def sur_mlp(G, spec, weights):
    G, w = _f64(G), _f64(weights)
    n = G.shape[0]
    sp = _sur_spec(spec)
    E, g = np.zeros(n), np.zeros((n, sp.nb))
    lib().orc_sur_mlp(n, _p(G), C.byref(sp), _p(w), _p(E), _p(g))
    return E, g


def sur_forces(pos, box, count, nl, spec, grad):
    pos, box, count, nl, grad = _f64(pos), _f64(box), _i32(count), _i32(nl), _f64(grad)
    n, k_max = nl.shape
    sp = _sur_spec(spec)
    F = np.zeros((n, 3))
    lib().orc_sur_forces(n, _p(pos), _p(box), _p(count), _p(nl), k_max, C.byref(sp), _p(grad), _p(F))
    return F


def surrogate(pos, box, spec, weights, k_max=64, method="cells"):
    """Energy (sum of E_i), per-atom energies, descriptors and forces of the surrogate."""
    count, nl, m = neighbours(pos, box, float(spec["rd"]) + float(spec.get("skin", 0.3)), k_max, method)
    if m > k_max:
        raise ValueError(f"neighbour list overflow: {m} > {k_max}")
    G = sur_descriptors(pos, box, count, nl, spec)
    E, g = sur_mlp(G, spec, weights)
    F = sur_forces(pos, box, count, nl, spec, g)
    return dict(energy=float(E.sum()), e_atom=E, G=G, grad=g, force=F, count=count, list=nl)


def sur_n_params(spec):
    nb, h1, h2 = int(spec["nb"]), int(spec["h1"]), int(spec["h2"])
    return h1 * nb + h1 + h2 * h1 + h2 + h2 + 1


def sur_loss_grad(frames, spec, weights, w_e=1.0, w_f=1.0, k_max=64):
    """Loss and parameter gradient over frames = [(pos, box, e_ref, f_ref), ...]."""
    off = np.zeros(len(frames) + 1, dtype=np.int64)
    pos, box, cnt, lists, eref, fref = [], [], [], [], [], []
    r_list = float(spec["rd"]) + float(spec.get("skin", 0.3))
    for s, (p, b, e, f) in enumerate(frames):
        c, nl, m = neighbours(p, b, r_list, k_max, "cells")
        if m > k_max:
            raise ValueError(f"neighbour list overflow: {m} > {k_max}")
        off[s + 1] = off[s] + len(p)
        pos.append(_f64(p)); box.append(_f64(b)); cnt.append(_i32(c)); lists.append(_i32(nl))
        eref.append(float(e)); fref.append(_f64(f))
    pos, box = np.ascontiguousarray(np.concatenate(pos)), np.ascontiguousarray(np.concatenate(box))
    cnt, lists = np.ascontiguousarray(np.concatenate(cnt)), np.ascontiguousarray(np.concatenate(lists))
    eref, fref = np.array(eref), np.ascontiguousarray(np.concatenate(fref))
    sp = _sur_spec(spec)
    w = _f64(weights)
    grad, parts = np.zeros(sur_n_params(spec)), np.zeros(2)
    loss = lib().orc_sur_loss_grad(len(frames), _p(off), _p(pos), _p(box), _p(cnt), _p(lists), k_max,
                                   _p(eref), _p(fref), C.byref(sp), _p(w), float(w_e), float(w_f),
                                   _p(grad), _p(parts))
    return dict(loss=float(loss), loss_e=float(parts[0]), loss_f=float(parts[1]), grad=grad)


def run_pc3(pos, vel, species, masses, box, pot, dt_fs, n_steps, skin, k_max, rebuild_every=0, force=None,
            gear3=None):
    """Third-order predictor-corrector (moldy_oracle.c orc_run_pc3) from (pos, vel); gear3 the
    third-derivative term (dt^3/6) da/dt of a previous call (None: zero).  Returns the final
    state (force at the last predicted positions, gear3) and per-step (PE, KE)."""
    pos, vel, box = _f64(pos).copy(), _f64(vel).copy(), _f64(box).copy()
    species, masses = _i32(species), _f64(masses)
    n = pos.shape[0]
    f = np.zeros((n, 3)) if force is None else _f64(force).copy()
    g3 = np.zeros((n, 3)) if gear3 is None else _f64(gear3).copy()
    energies = np.zeros((max(n_steps, 1), 2))
    nreb = np.zeros(1, np.int32)
    P = _Pot(pot)
    lib().orc_run_pc3(n, _p(pos), _p(vel), _p(species), _p(masses), _p(box), P.ref, float(dt_fs), int(n_steps),
                      float(skin), int(k_max), int(rebuild_every), _p(f), 0 if force is None else 1, _p(g3),
                      _p(energies), _p(nreb))
    return dict(pos=pos, vel=vel, force=f, gear3=g3, energies=energies[:n_steps], n_rebuilds=int(nreb[0]))


def run_nvt(pos, vel, species, masses, box, pot, dt_fs, n_steps, skin, k_max, t_kelvin, q_ev_fs2,
            pi=0.0, xi=0.0, force=None):
    """Nose-Hoover velocity Verlet; returns the final state, thermostat (pi, xi) and per-step
    (PE, KE, extended energy H')."""
    pos, vel, box = _f64(pos).copy(), _f64(vel).copy(), _f64(box).copy()
    species, masses = _i32(species), _f64(masses)
    n = pos.shape[0]
    f = np.zeros((n, 3)) if force is None else _f64(force).copy()
    energies = np.zeros((max(n_steps, 1), 3))
    th = np.array([pi, xi, q_ev_fs2], dtype=np.float64)
    P = _Pot(pot)
    lib().orc_run_nvt(n, _p(pos), _p(vel), _p(species), _p(masses), _p(box), P.ref, float(dt_fs), int(n_steps),
                      float(skin), int(k_max), float(t_kelvin), _p(th), _p(f), 0 if force is None else 1,
                      _p(energies))
    return dict(pos=pos, vel=vel, force=f, box=box, energies=energies[:n_steps], pi=float(th[0]), xi=float(th[1]))


def adam_step(w, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, Algorithm 1): returns new (w, m, v); t counts from 1."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
