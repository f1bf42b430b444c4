"""Thin Python binding of the C ABI in ``include/vpath.h`` (argument
marshalling only: every step of the path runs in the CUDA library).

The module-level functions carry the C names (``sim_create``,
``sim_step_batch``, ``bias_functional``, ``energy_forces``, ...);
:class:`TrialBatch` wraps a handle for convenience.  There is no CPU
fallback: if the compiled library is missing, loading raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import systems as _systems

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libvpath.so")

SIM_OK = 0
SIM_EINVAL = -1
SIM_ECUDA = -2
SIM_ELIST_OVERFLOW = -3
SIM_ESKIN = -4
SIM_ENONFINITE = -5
SIM_ETIMEOUT = -6
SIM_STRICT_SKIN = 1
SIM_NO_GRAPH = 2
SIM_FIXED_INTERVAL = 4

_ERRNAMES = {SIM_EINVAL: "SIM_EINVAL", SIM_ECUDA: "SIM_ECUDA", SIM_ELIST_OVERFLOW: "SIM_ELIST_OVERFLOW",
             SIM_ESKIN: "SIM_ESKIN", SIM_ENONFINITE: "SIM_ENONFINITE", SIM_ETIMEOUT: "SIM_ETIMEOUT"}


class SimError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class SimSystem(C.Structure):
    _fields_ = [
        ("n_atoms", C.c_int32), ("n_solute", C.c_int32), ("n_cv", C.c_int32),
        ("pos", C.c_void_p), ("vel", C.c_void_p), ("mass", C.c_void_p), ("charge", C.c_void_p),
        ("lj_type", C.c_void_p), ("n_types", C.c_int32), ("sigma", C.c_void_p), ("epsilon", C.c_void_p),
        ("n_bonds", C.c_int32), ("bonds", C.c_void_p), ("bond_r0", C.c_void_p), ("bond_k", C.c_void_p),
        ("n_angles", C.c_int32), ("angles", C.c_void_p), ("angle_t0", C.c_void_p), ("angle_k", C.c_void_p),
        ("n_excl", C.c_int32), ("excl", C.c_void_p),
        ("box", C.c_double), ("native_pos", C.c_void_p), ("gamma", C.c_void_p),
    ]


class SimParams(C.Structure):
    _fields_ = [
        ("dt", C.c_double), ("temperature", C.c_double), ("gamma", C.c_double), ("r_cut", C.c_double),
        ("skin", C.c_double), ("nstlist", C.c_int32), ("eps_rf", C.c_double), ("k_ratchet", C.c_double),
        ("cv_r0", C.c_double), ("cv_r_switch", C.c_double), ("cv_r_cut", C.c_double), ("cv_min_sep", C.c_int32),
        ("seed", C.c_uint64), ("flags", C.c_int32),
    ]


class Toy2dParamsC(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("A1", "A2", "A3", "s1", "s2", "s3", "w", "xm", "ym", "mass", "gamma", "kT",
                                          "dt", "x0", "y0", "z_product")] + [("bias", C.c_int32), ("s_power", C.c_int32)]


_lib = None

# every symbol the header declares, with its ctypes signature
_SIGS = {
    "sim_create": ([C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "sim_step_batch": ([C.c_void_p, C.c_int32], C.c_int),
    "bias_functional": ([C.c_void_p, C.c_double, C.c_void_p, C.c_void_p], C.c_int),
    "energy_forces": ([C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p], C.c_int),
    "sim_get_state": ([C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "sim_set_state": ([C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "sim_step_count": ([C.c_void_p], C.c_int64),
    "sim_set_step_count": ([C.c_void_p, C.c_int64], C.c_int),
    "sim_set_noise_offset": ([C.c_void_p, C.c_int32, C.c_int64], C.c_int),
    "sim_trial_seed": ([C.c_void_p, C.c_int32, C.c_void_p], C.c_int),
    "sim_num_trials": ([C.c_void_p], C.c_int32),
    "sim_num_atoms": ([C.c_void_p, C.c_int32], C.c_int32),
    "sim_record": ([C.c_void_p, C.c_int32], C.c_int),
    "sim_get_record": ([C.c_void_p, C.c_int32, C.c_void_p], C.c_int),
    "sim_record_frames": ([C.c_void_p, C.c_int32, C.c_int32], C.c_int),
    "sim_frame_shape": ([C.c_void_p, C.c_void_p], C.c_int),
    "sim_get_frames": ([C.c_void_p, C.c_void_p, C.c_int64], C.c_int),
    "sim_noise_offset": ([C.c_void_p, C.c_int32, C.c_void_p], C.c_int),
    "sim_set_variants": ([C.c_void_p, C.c_int32, C.c_int32], C.c_int),
    "phi_frames_adjoint": ([C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                            C.c_void_p], C.c_int),
    "phi_adjoint_coefficients": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p], C.c_int),
    "sim_pairlist": ([C.c_void_p, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p], C.c_int),
    "sim_diagnostics": ([C.c_void_p, C.c_void_p], C.c_int),
    "sim_list_positions": ([C.c_void_p, C.c_int32, C.c_void_p], C.c_int),
    "sim_rebuild": ([C.c_void_p], C.c_int),
    "sim_potential_device": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "sim_autotune": ([C.c_void_p, C.c_int32, C.c_char_p, C.c_void_p], C.c_int),
    "sim_set_timing": ([C.c_void_p, C.c_int32], C.c_int),
    "sim_tune_classes": ([C.c_void_p, C.c_void_p, C.c_int32], C.c_int32),
    "sim_set_class_variants": ([C.c_void_p, C.c_void_p, C.c_int32], C.c_int),
    "sim_set_step_mode": ([C.c_void_p, C.c_int32], C.c_int),
    "sim_step_mode": ([C.c_void_p], C.c_int32),
    "sim_autotune_step": ([C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p], C.c_int),
    "sim_kernel_times": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32], C.c_int),
    "sim_philox_normals": ([C.c_uint64, C.c_int64, C.c_uint32, C.c_int32, C.c_void_p, C.c_void_p], C.c_int),
    "cv_eval_noalloc": ([C.c_void_p, C.c_void_p, C.c_int32, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                         C.c_char_p, C.c_int32], C.c_int),
    "phi_frames_refine": ([C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_int32, C.c_double, C.c_void_p,
                           C.c_void_p], C.c_int),
    "sim_contact_tracking": ([C.c_void_p, C.c_int32], C.c_int),
    "sim_native_contacts": ([C.c_void_p, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p], C.c_int),
    "sim_contact_times": ([C.c_void_p, C.c_int32, C.c_void_p, C.c_int64], C.c_int),
    "path_similarity": ([C.c_void_p, C.c_int32, C.c_int64, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                         C.c_char_p, C.c_int32], C.c_int),
    "toy2d_run": ([C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                   C.c_void_p, C.c_int32, C.c_void_p, C.c_char_p, C.c_int32], C.c_int),
    "sim_stream": ([C.c_void_p], C.c_void_p),
    "sim_destroy": ([C.c_void_p], None),
    "sim_last_error": ([C.c_void_p], C.c_char_p),
}


def load(path: str = LIB_PATH):
    """Loads the compiled library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
        L = C.CDLL(path)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _check(h, rc):
    if rc != SIM_OK:
        msg = load().sim_last_error(h).decode() if h else ""
        raise SimError(rc, msg)


class _Marshalled:
    """Host arrays behind one SimSystem (kept alive during sim_create)."""

    def __init__(self, s: "_systems.System"):
        f64 = lambda a: None if a is None else np.ascontiguousarray(np.asarray(a, np.float64).reshape(-1))
        i32 = lambda a: None if a is None else np.ascontiguousarray(np.asarray(a, np.int32).reshape(-1))
        self.keep = k = dict(
            pos=f64(s.pos), vel=f64(s.vel), mass=f64(s.mass), charge=f64(s.charge), lj_type=i32(s.lj_type),
            sigma=f64(s.sigma), epsilon=f64(s.epsilon), bonds=i32(s.bonds), bond_r0=f64(s.bond_r0),
            bond_k=f64(s.bond_k), angles=i32(s.angles), angle_t0=f64(s.angle_t0), angle_k=f64(s.angle_k),
            excl=i32(s.excl_pairs), native=f64(s.native_pos), gamma=f64(s.gamma))
        self.c = SimSystem(
            n_atoms=s.n_atoms, n_solute=s.n_solute, n_cv=s.n_cv, pos=_ptr(k["pos"]), vel=_ptr(k["vel"]),
            mass=_ptr(k["mass"]), charge=_ptr(k["charge"]), lj_type=_ptr(k["lj_type"]), n_types=len(s.sigma),
            sigma=_ptr(k["sigma"]), epsilon=_ptr(k["epsilon"]), n_bonds=len(s.bonds), bonds=_ptr(k["bonds"]),
            bond_r0=_ptr(k["bond_r0"]), bond_k=_ptr(k["bond_k"]), n_angles=len(s.angles), angles=_ptr(k["angles"]),
            angle_t0=_ptr(k["angle_t0"]), angle_k=_ptr(k["angle_k"]),
            n_excl=0 if s.excl_pairs is None else len(s.excl_pairs), excl=_ptr(k["excl"]), box=float(s.box),
            native_pos=_ptr(k["native"]), gamma=_ptr(k["gamma"]))


def params_struct(p: "_systems.Params") -> SimParams:
    return SimParams(dt=p.dt, temperature=p.temperature, gamma=p.gamma, r_cut=p.r_cut, skin=p.skin,
                     nstlist=p.nstlist, eps_rf=p.eps_rf, k_ratchet=p.k_ratchet, cv_r0=p.cv_r0,
                     cv_r_switch=p.cv_r_switch, cv_r_cut=p.cv_r_cut, cv_min_sep=p.cv_min_sep, seed=p.seed,
                     flags=p.flags)


# ---------------------------------------------------------------------------
# C-named functions
# ---------------------------------------------------------------------------

def sim_create(systems: Sequence["_systems.System"], params: "_systems.Params", trials_per_system: Sequence[int],
               trial_seeds: Optional[Sequence[int]] = None, cuda_stream: int = 0):
    L = load()
    ms = [_Marshalled(s) for s in systems]
    arr = (SimSystem * len(ms))(*[m.c for m in ms])
    tps = np.ascontiguousarray(np.asarray(trials_per_system, np.int32))
    seeds = None if trial_seeds is None else np.ascontiguousarray(np.asarray(trial_seeds, np.uint64))
    ps = params_struct(params)
    h = C.c_void_p()
    rc = L.sim_create(C.cast(arr, C.c_void_p), len(ms), tps.ctypes.data, _ptr(seeds), C.addressof(ps),
                      C.c_void_p(cuda_stream or None), C.addressof(h))
    if rc != SIM_OK:
        msg = L.sim_last_error(h).decode() if h.value else ""
        if h.value:
            L.sim_destroy(h)
        raise SimError(rc, msg)
    return h


def sim_step_batch(h, n_steps: int):
    _check(h, load().sim_step_batch(h, int(n_steps)))


def bias_functional(h, z_max: float = -1.0):
    n = load().sim_num_trials(h)
    phi = np.zeros(n)
    am = C.c_int32(-1)
    _check(h, load().bias_functional(h, float(z_max), phi.ctypes.data, C.addressof(am)))
    return phi, int(am.value)


def energy_forces(h, trial: int, want_forces: bool = True):
    n = load().sim_num_atoms(h, trial)
    e = np.zeros(6)
    F = np.zeros((n, 3)) if want_forces else None
    _check(h, load().energy_forces(h, int(trial), e.ctypes.data, _ptr(F)))
    return e, F


def sim_get_state(h, trial: int):
    n = load().sim_num_atoms(h, trial)
    pos = np.zeros((n, 3))
    vel = np.zeros((n, 3))
    cv = np.zeros(4)
    _check(h, load().sim_get_state(h, int(trial), pos.ctypes.data, vel.ctypes.data, cv.ctypes.data))
    return pos, vel, cv


def sim_set_state(h, trial: int, pos, vel, cv_state=None):
    P = np.ascontiguousarray(np.asarray(pos, np.float64).reshape(-1))
    V = np.ascontiguousarray(np.asarray(vel, np.float64).reshape(-1))
    S = None if cv_state is None else np.ascontiguousarray(np.asarray(cv_state, np.float64).reshape(-1))
    _check(h, load().sim_set_state(h, int(trial), P.ctypes.data, V.ctypes.data, _ptr(S)))


def sim_step_count(h) -> int:
    return int(load().sim_step_count(h))


def sim_set_step_count(h, step: int):
    _check(h, load().sim_set_step_count(h, int(step)))


def sim_num_trials(h) -> int:
    return int(load().sim_num_trials(h))


def sim_num_atoms(h, trial: int) -> int:
    return int(load().sim_num_atoms(h, trial))


def sim_record(h, capacity: int):
    _check(h, load().sim_record(h, int(capacity)))


def sim_get_record(h, trial: int, capacity: int):
    """[capacity, 5]: z, z_m, a, phi, Q per step (index = step % capacity)."""
    out = np.zeros((capacity, 5))
    _check(h, load().sim_get_record(h, int(trial), out.ctypes.data))
    return out


def sim_record_frames(h, trial: int, capacity: int):
    _check(h, load().sim_record_frames(h, int(trial), int(capacity)))


def sim_frame_shape(h):
    """(trials recorded, capacity, CV atoms per frame) of the frame record."""
    sh = np.zeros(3, np.int32)
    _check(h, load().sim_frame_shape(h, sh.ctypes.data))
    return int(sh[0]), int(sh[1]), int(sh[2])


def sim_get_frames(h, capacity: Optional[int] = None, n_cv: Optional[int] = None, n_trials: int = 0):
    """The frame record: (capacity, n_cv, 3) for one recorded trial, or
    (n_trials, capacity, n_cv, 3) when every trial is recorded (n_cv then the
    largest of the batch).  The shape comes from the handle; capacity, n_cv
    and n_trials, when given, must match it."""
    nt, cap, m = sim_frame_shape(h)
    if ((capacity is not None and capacity != cap) or (n_cv is not None and n_cv != m)
            or (n_trials and n_trials != nt)):
        raise ValueError(f"the frame record holds {nt} trial(s) x {cap} frames x {m} atoms, "
                         f"not {n_trials or 1} x {capacity} x {n_cv}")
    out = np.zeros((nt, cap, m, 3) if (n_trials or nt != 1) else (cap, m, 3))
    _check(h, load().sim_get_frames(h, out.ctypes.data, out.size))
    return out


def sim_noise_offset(h, trial: int) -> int:
    v = C.c_int64(0)
    _check(h, load().sim_noise_offset(h, int(trial), C.byref(v)))
    return int(v.value)


def sim_set_variants(h, pair_variant: int, cv_variant: int = 0):
    """Fixes the launch shapes (the autotuner's numbering)."""
    _check(h, load().sim_set_variants(h, int(pair_variant), int(cv_variant)))


def sim_set_noise_offset(h, trial: int, offset: int):
    _check(h, load().sim_set_noise_offset(h, int(trial), int(offset)))


def sim_trial_seed(h, trial: int) -> int:
    v = C.c_uint64(0)
    _check(h, load().sim_trial_seed(h, int(trial), C.byref(v)))
    return int(v.value)


def phi_frames_adjoint(h, trial: int, frames, coef=None):
    """(Phi or None, z per frame, dPhi/dframes) for frames (n_frames, n_cv, 3)."""
    F = np.ascontiguousarray(np.asarray(frames, np.float64))
    nf, ncv = F.shape[0], F.shape[1]
    Cf = None if coef is None else np.ascontiguousarray(np.asarray(coef, np.float64).reshape(-1))
    phi = np.zeros(1)
    z = np.zeros(nf)
    G = np.zeros((nf, ncv, 3))
    _check(h, load().phi_frames_adjoint(h, int(trial), F.ctypes.data, nf, _ptr(Cf), phi.ctypes.data, z.ctypes.data,
                                        G.ctypes.data))
    return (None if coef is not None else float(phi[0])), z, G


def phi_adjoint_coefficients(h, z, Q):
    zz = np.ascontiguousarray(np.asarray(z, np.float64))
    qq = np.ascontiguousarray(np.asarray(Q, np.float64))
    coef = np.zeros((len(zz), 2))
    phi = np.zeros(1)
    _check(h, load().phi_adjoint_coefficients(h, zz.ctypes.data, qq.ctypes.data, len(zz), coef.ctypes.data,
                                              phi.ctypes.data))
    return coef, float(phi[0])


def sim_pairlist(h, trial: int, cap: int = 0):
    n = load().sim_num_atoms(h, trial)
    cap = cap or max(1024, 400 * n)
    pairs = np.zeros((cap, 2), np.int32)
    cnt = C.c_int64(0)
    _check(h, load().sim_pairlist(h, int(trial), pairs.ctypes.data, cap, C.addressof(cnt)))
    if cnt.value > cap:
        return sim_pairlist(h, trial, int(cnt.value))
    return pairs[: cnt.value]


def sim_diagnostics(h):
    out = np.zeros(7, np.int64)
    _check(h, load().sim_diagnostics(h, out.ctypes.data))
    return dict(skin_violations=int(out[0]), max_list_entries=int(out[1]), list_capacity=int(out[2]),
                clusters=int(out[3]), list_entries=int(out[4]), trial_rebuilds=int(out[5]),
                displacement_rebuilds=int(out[6]))


def sim_list_positions(h, trial: int):
    """(n_atoms, 3): the positions the trial's current list was built from."""
    n = load().sim_num_atoms(h, trial)
    out = np.zeros((n, 3))
    _check(h, load().sim_list_positions(h, int(trial), out.ctypes.data))
    return out


def sim_potential_device(h, d_pos: int, d_energy: int, d_forces: int, cuda_stream: int = 0):
    """U and -grad U of one configuration per trial, device pointers in and
    out (e.g. ``tensor.data_ptr()``), ordered on the given stream."""
    _check(h, load().sim_potential_device(h, C.c_void_p(d_pos or None), C.c_void_p(d_energy or None),
                                          C.c_void_p(d_forces or None), C.c_void_p(cuda_stream or None)))


def sim_rebuild(h):
    """Rebuilds every list at the current positions (state unchanged)."""
    _check(h, load().sim_rebuild(h))


def sim_autotune(h, reps: int = 5, cache_path: Optional[str] = None):
    """Picks the fastest launch shapes for this batch; returns (pair, cv) variants."""
    ch = np.zeros(2, np.int32)
    _check(h, load().sim_autotune(h, int(reps), None if cache_path is None else cache_path.encode(), ch.ctypes.data))
    return int(ch[0]), int(ch[1])


def sim_tune_classes(h):
    """The batch's size classes: a list of dicts (log2 atoms, trials, clusters,
    pair variant, whether the class has its own pair launch)."""
    n = load().sim_tune_classes(h, None, 0)
    if n < 0:
        raise SimError(n, sim_last_error(h))
    info = np.zeros(5 * max(n, 1), np.int32)
    load().sim_tune_classes(h, info.ctypes.data, n)
    return [dict(lg_atoms=int(info[5 * k]), trials=int(info[5 * k + 1]), clusters=int(info[5 * k + 2]),
                 pair_variant=int(info[5 * k + 3]), own_launch=bool(info[5 * k + 4])) for k in range(n)]


def sim_set_class_variants(h, variants):
    """One pair launch per size class, class k with variants[k]."""
    v = np.ascontiguousarray(np.asarray(variants, np.int32))
    _check(h, load().sim_set_class_variants(h, v.ctypes.data, len(v)))


STEP_MODES = 3
STEP_FORM_NAMES = ("kernel per phase", "one kernel", "kernel per phase, rebuild kernels only in rebuild steps")


def sim_set_step_mode(h, mode: int):
    """0: one kernel per phase (graph replays); 1: one cooperative kernel per
    step; 2: as 0, the rebuild kernels in conditional graph nodes opened only
    in steps in which a trial rebuilds."""
    _check(h, load().sim_set_step_mode(h, int(mode)))


def sim_step_mode(h) -> int:
    return int(load().sim_step_mode(h))


def sim_autotune_step(h, reps: int = 3, times: bool = False):
    """Times every step form on this batch, keeps the fastest; the state is
    restored.  Returns the form (and, with times, every form's ms per step)."""
    m = C.c_int32(0)
    ms = np.full(STEP_MODES, np.nan)
    _check(h, load().sim_autotune_step(h, int(reps), C.byref(m), ms.ctypes.data))
    return (int(m.value), [float(x) for x in ms]) if times else int(m.value)


def sim_set_timing(h, on):
    """0: off, 1 (or True): direct launches timed per kernel, 2: in-graph timing of the pair kernel."""
    _check(h, load().sim_set_timing(h, int(on)))


def sim_kernel_times(h):
    cap = 64
    names = (C.c_char_p * cap)()
    ms = np.zeros(cap)
    cnt = np.zeros(cap, np.int64)
    n = load().sim_kernel_times(h, C.cast(names, C.c_void_p), ms.ctypes.data, cnt.ctypes.data, cap)
    return {names[k].decode(): (float(ms[k]), int(cnt[k])) for k in range(min(n, cap))}


def sim_philox_normals(seed: int, step: int, stream: int, n: int):
    raw = np.zeros((n, 4), np.uint32)
    nor = np.zeros((n, 3))
    rc = load().sim_philox_normals(int(seed), int(step), int(stream), int(n), raw.ctypes.data, nor.ctypes.data)
    if rc != SIM_OK:
        raise SimError(rc, "sim_philox_normals failed")
    return raw, nor


def cv_eval_noalloc(d_pos: int, d_native: int, n_cv: int, box: float, params, d_z: int, d_grad: int,
                    cuda_stream: int = 0):
    """z and grad z of one configuration without any device allocation (all
    pointers are device addresses, e.g. ``tensor.data_ptr()``).  Returns the
    status code and the library's message."""
    ps = params_struct(params)
    buf = C.create_string_buffer(256)
    rc = load().cv_eval_noalloc(C.c_void_p(d_pos or None), C.c_void_p(d_native or None), int(n_cv), float(box),
                                C.addressof(ps), C.c_void_p(d_z or None), C.c_void_p(d_grad or None),
                                C.c_void_p(cuda_stream or None), buf, 256)
    return rc, buf.value.decode()


def phi_frames_refine(h, trial: int, frames, n_iter: int, step: float):
    """Descent on Phi over the inner frames of a path (n_frames, n_cv, 3);
    returns (refined frames, Phi history [n_iter + 1], accepted iterations)."""
    F = np.array(frames, dtype=np.float64, order="C", copy=True)
    hist = np.zeros(n_iter + 1)
    acc = C.c_int32(0)
    _check(h, load().phi_frames_refine(h, int(trial), F.ctypes.data, F.shape[0], int(n_iter), float(step),
                                       hist.ctypes.data, C.byref(acc)))
    return F, hist, int(acc.value)


def sim_contact_tracking(h, every: int):
    _check(h, load().sim_contact_tracking(h, int(every)))


def sim_native_contacts(h, trial: int):
    n = C.c_int64(0)
    _check(h, load().sim_native_contacts(h, int(trial), None, 0, C.byref(n)))
    pairs = np.zeros((max(n.value, 1), 2), np.int32)
    _check(h, load().sim_native_contacts(h, int(trial), pairs.ctypes.data, n.value, C.byref(n)))
    return pairs[: n.value]


def sim_contact_times(h, trial: int, n_contacts: int):
    t = np.zeros(max(n_contacts, 1), np.int64)
    _check(h, load().sim_contact_times(h, int(trial), t.ctypes.data, int(n_contacts)))
    return t[:n_contacts]


def path_similarity(times, pairs, cuda_stream: int = 0):
    """s(k, k') on the GPU for each (k, k') in pairs; times (n_paths, n_c)."""
    T = np.ascontiguousarray(times, np.int64)
    if T.ndim != 2:
        raise ValueError("times must be (n_paths, n_contacts)")
    P = np.ascontiguousarray(pairs, np.int32).reshape(-1, 2)
    out = np.zeros(len(P))
    buf = C.create_string_buffer(256)
    rc = load().path_similarity(T.ctypes.data, T.shape[0], T.shape[1], P.ctypes.data, len(P), out.ctypes.data,
                                C.c_void_p(cuda_stream or None), buf, 256)
    if rc != SIM_OK:
        raise SimError(rc, buf.value.decode())
    return out


def toy2d_run(tp, k, seeds, n_steps: int, path_every: int = 0, want_state: bool = True, cuda_stream: int = 0):
    """Trials of the two-dimensional toy model on the GPU: k[i] and seeds[i]
    per trial.  Returns (passage int64[n], phi[n], state (n, 4) or None,
    path (n, n_steps // path_every + 1, 2) or None)."""
    k = np.ascontiguousarray(k, np.float64).reshape(-1)
    sd = np.ascontiguousarray(seeds, np.uint64).reshape(-1)
    if len(k) != len(sd):
        raise ValueError("k and seeds differ in length")
    n = len(k)
    pc = Toy2dParamsC(**{f: float(getattr(tp, f)) for f, _ in Toy2dParamsC._fields_ if f not in ("bias", "s_power")},
                      bias=int(tp.bias), s_power=int(tp.s_power))
    phi = np.zeros(n)
    passage = np.zeros(n, np.int64)
    state = np.zeros((n, 4)) if want_state else None
    path = np.zeros((n, n_steps // path_every + 1, 2)) if path_every > 0 else None
    buf = C.create_string_buffer(256)
    rc = load().toy2d_run(C.addressof(pc), n, k.ctypes.data, sd.ctypes.data, int(n_steps),
                          None if state is None else state.ctypes.data, phi.ctypes.data, passage.ctypes.data,
                          None if path is None else path.ctypes.data, int(path_every), C.c_void_p(cuda_stream or None),
                          buf, 256)
    if rc != SIM_OK:
        raise SimError(rc, buf.value.decode())
    return passage, phi, state, path


def sim_stream(h) -> int:
    return int(load().sim_stream(h) or 0)


def sim_destroy(h):
    if h is not None and getattr(h, "value", h):
        load().sim_destroy(h)


def sim_last_error(h) -> str:
    return load().sim_last_error(h).decode()


class TrialBatch:
    """A batch of independent trials (owning one library handle)."""

    def __init__(self, systems, params, trials_per_system, trial_seeds=None, cuda_stream: int = 0):
        if not isinstance(systems, (list, tuple)):
            systems = [systems]
        self.systems = list(systems)
        self.params = params
        self.trials_per_system = list(trials_per_system)
        self.h = sim_create(self.systems, params, trials_per_system, trial_seeds, cuda_stream)
        self.n_trials = sim_num_trials(self.h)

    def step(self, n: int):
        sim_step_batch(self.h, n)

    def bias_functional(self, z_max: float = -1.0):
        return bias_functional(self.h, z_max)

    def energy_forces(self, trial: int = 0, want_forces: bool = True):
        return energy_forces(self.h, trial, want_forces)

    def get_state(self, trial: int = 0):
        return sim_get_state(self.h, trial)

    def set_state(self, trial, pos, vel, cv_state=None):
        sim_set_state(self.h, trial, pos, vel, cv_state)

    @property
    def step_count(self) -> int:
        return sim_step_count(self.h)

    @property
    def stream(self) -> int:
        return sim_stream(self.h)

    def close(self):
        for rb in self.__dict__.pop("_replay_batches", {}).values():
            rb.close()
        if self.h is not None:
            sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
