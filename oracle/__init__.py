"""Python access to the FP64 CPU oracle (test infrastructure only).

The oracle is plain C in ``vpath_oracle.c``.  Only the tests,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` import this package; the product path (the CUDA library
and its binding) never does.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vpath_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "toy2d_oracle.c"), os.path.join(_HERE, "contacts_oracle.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libvpath_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(f) for f in _SRCS)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               *_SRCS, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrSystem(C.Structure):
    _fields_ = [
        ("n", C.c_int32), ("n_solute", C.c_int32), ("n_cv", C.c_int32), ("n_types", C.c_int32),
        ("mass", C.c_void_p), ("charge", C.c_void_p), ("sigma", C.c_void_p), ("epsilon", C.c_void_p),
        ("gamma", C.c_void_p), ("type", C.c_void_p),
        ("n_bonds", C.c_int32), ("bonds", C.c_void_p), ("bond_r0", C.c_void_p), ("bond_k", C.c_void_p),
        ("n_angles", C.c_int32), ("angles", C.c_void_p), ("angle_t0", C.c_void_p), ("angle_k", C.c_void_p),
        ("n_excl", C.c_int32), ("excl", C.c_void_p),
        ("box", C.c_double), ("native", C.c_void_p),
    ]


class OrParams(C.Structure):
    _fields_ = [
        ("dt", C.c_double), ("temperature", C.c_double), ("gamma", C.c_double), ("r_cut", C.c_double),
        ("skin", C.c_double), ("nstlist", C.c_int32),
        ("eps_rf", C.c_double), ("k_ratchet", C.c_double), ("cv_r0", C.c_double), ("cv_r_switch", C.c_double),
        ("cv_r_cut", C.c_double), ("cv_min_sep", C.c_int32), ("list_fixed", C.c_int32),
    ]


class OrRunOut(C.Structure):
    _fields_ = [
        ("z", C.c_void_p), ("zm", C.c_void_p), ("a", C.c_void_p), ("phi_step", C.c_void_p),
        ("frames", C.c_void_p), ("record_every", C.c_int32),
        ("pos_out", C.c_void_p), ("vel_out", C.c_void_p),
        ("Phi", C.c_double), ("energies", C.c_double * 6), ("force_out", C.c_void_p),
    ]


class OrToy2dParams(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("A1", "A2", "A3", "s1", "s2", "s3", "w", "xm", "ym", "mass", "gamma", "kT",
                                          "dt", "x0", "y0", "z_product")] + [("bias", C.c_int32), ("s_power", C.c_int32)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            vp = C.c_void_p
            L.or_philox4x32_10.argtypes = [vp, vp, vp]
            L.or_normal3.argtypes = [C.c_uint64, C.c_int64, C.c_int64, C.c_uint32, vp]
            L.or_contact.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, vp]
            L.or_cv.argtypes = [vp, vp, C.c_int32, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int32, vp]
            L.or_cv.restype = C.c_double
            L.or_pairlist.argtypes = [C.POINTER(OrSystem), vp, C.c_double, vp, C.c_int64]
            L.or_pairlist.restype = C.c_int64
            L.or_forces.argtypes = [C.POINTER(OrSystem), C.POINTER(OrParams), vp, C.c_int32, vp, vp]
            L.or_forces.restype = C.c_int
            L.or_initial_velocities.argtypes = [C.POINTER(OrSystem), C.c_double, C.c_uint64, vp]
            L.or_run.argtypes = [C.POINTER(OrSystem), C.POINTER(OrParams), C.c_uint64, vp, vp, C.c_int32,
                                 C.POINTER(OrRunOut)]
            L.or_run.restype = C.c_int
            L.or_phi_frames.argtypes = [C.POINTER(OrSystem), C.POINTER(OrParams), vp, C.c_int32, vp, vp, vp]
            L.or_phi_frames.restype = C.c_double
            L.or_phi_frames_grad.argtypes = [C.POINTER(OrSystem), C.POINTER(OrParams), vp, C.c_int32, vp]
            L.or_phi_frames_grad.restype = C.c_double
            L.or_toy2d_force.argtypes = [C.POINTER(OrToy2dParams), C.c_double, C.c_double, vp, vp, vp]
            L.or_toy2d_run.argtypes = [C.POINTER(OrToy2dParams), C.c_double, C.c_uint64, C.c_int64, vp, vp, vp]
            L.or_toy2d_run.restype = C.c_int64
            L.or_toy2d_phi_path.argtypes = [C.POINTER(OrToy2dParams), C.c_double, vp, C.c_int64, vp]
            L.or_toy2d_phi_path.restype = C.c_double
            L.or_native_contacts.argtypes = [vp, C.c_int32, C.c_double, C.c_int32, vp, C.c_int64]
            L.or_native_contacts.restype = C.c_int64
            L.or_contact_times.argtypes = [vp, vp, C.c_int32, C.c_int32, C.c_double, C.c_double, vp, C.c_int64, vp]
            L.or_path_similarity.argtypes = [vp, vp, C.c_int64]
            L.or_path_similarity.restype = C.c_double
            L.or_num_threads.restype = C.c_int32
            L.or_set_num_threads.argtypes = [C.c_int32]
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


class _Sys:
    """Keeps the numpy arrays behind an OrSystem alive."""

    def __init__(self, s):
        self.keep = dict(
            mass=np.ascontiguousarray(s.mass, np.float64), charge=np.ascontiguousarray(s.charge, np.float64),
            sigma=np.ascontiguousarray(s.sigma, np.float64), epsilon=np.ascontiguousarray(s.epsilon, np.float64),
            gamma=None if s.gamma is None else np.ascontiguousarray(s.gamma, np.float64),
            type=np.ascontiguousarray(s.lj_type, np.int32),
            bonds=np.ascontiguousarray(s.bonds, np.int32).reshape(-1), bond_r0=np.ascontiguousarray(s.bond_r0, np.float64),
            bond_k=np.ascontiguousarray(s.bond_k, np.float64),
            angles=np.ascontiguousarray(s.angles, np.int32).reshape(-1),
            angle_t0=np.ascontiguousarray(s.angle_t0, np.float64), angle_k=np.ascontiguousarray(s.angle_k, np.float64),
            excl=None if s.excl_pairs is None else np.ascontiguousarray(s.excl_pairs, np.int32).reshape(-1),
            native=np.ascontiguousarray(s.native_pos, np.float64).reshape(-1),
        )
        k = self.keep
        self.c = OrSystem(
            n=s.n_atoms, n_solute=s.n_solute, n_cv=s.n_cv, n_types=len(s.sigma),
            mass=_p(k["mass"]), charge=_p(k["charge"]), sigma=_p(k["sigma"]), epsilon=_p(k["epsilon"]),
            gamma=_p(k["gamma"]), type=_p(k["type"]),
            n_bonds=len(s.bonds), bonds=_p(k["bonds"]), bond_r0=_p(k["bond_r0"]), bond_k=_p(k["bond_k"]),
            n_angles=len(s.angles), angles=_p(k["angles"]), angle_t0=_p(k["angle_t0"]), angle_k=_p(k["angle_k"]),
            n_excl=0 if s.excl_pairs is None else len(s.excl_pairs), excl=_p(k["excl"]),
            box=float(s.box), native=_p(k["native"]))


def _params(p):
    return OrParams(dt=p.dt, temperature=p.temperature, gamma=p.gamma, r_cut=p.r_cut, skin=p.skin,
                    nstlist=p.nstlist, eps_rf=p.eps_rf, k_ratchet=p.k_ratchet, cv_r0=p.cv_r0,
                    cv_r_switch=p.cv_r_switch, cv_r_cut=p.cv_r_cut, cv_min_sep=p.cv_min_sep,
                    list_fixed=int((getattr(p, "flags", 0) & 4) != 0))  # bit 4 of the flags: fixed-interval lists


# ---------------------------------------------------------------------------
# thin wrappers
# ---------------------------------------------------------------------------

def philox4x32_10(ctr, key):
    c = np.asarray(ctr, np.uint32)
    k = np.asarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def normal3(seed, atom, step, stream):
    out = np.zeros(3)
    lib().or_normal3(int(seed), int(atom), int(step), int(stream), out.ctypes.data)
    return out


def contact(r, r0=0.75, rs=1.0, rc=1.2):
    out = np.zeros(4)
    lib().or_contact(float(r), float(r0), float(rs), float(rc), out.ctypes.data)
    return out  # C, C~, dC/dr, dC~/dr


def cv(s, p, pos):
    """z and grad z (n_cv, 3) at the given positions."""
    X = np.ascontiguousarray(np.asarray(pos, np.float64)[: s.n_cv].reshape(-1))
    nat = np.ascontiguousarray(s.native_pos, np.float64).reshape(-1)
    g = np.zeros(3 * s.n_cv)
    z = lib().or_cv(X.ctypes.data, nat.ctypes.data, s.n_cv, float(s.box), p.cv_r0, p.cv_r_switch, p.cv_r_cut,
                    p.cv_min_sep, g.ctypes.data)
    return z, g.reshape(-1, 3)


def pairlist(s, posf, r_list):
    """Sorted (i<j) pairs of the FP32 list rule from float positions."""
    ss = _Sys(s)
    pf = np.ascontiguousarray(np.asarray(posf, np.float32).reshape(-1))
    cap = max(1024, s.n_atoms * 400)
    out = np.zeros(2 * cap, np.int32)
    n = lib().or_pairlist(C.byref(ss.c), pf.ctypes.data, float(r_list), out.ctypes.data, cap)
    if n > cap:
        out = np.zeros(2 * n, np.int32)
        n = lib().or_pairlist(C.byref(ss.c), pf.ctypes.data, float(r_list), out.ctypes.data, n)
    return out[: 2 * n].reshape(-1, 2)


def forces(s, p, pos, use_list=False):
    """(F (n,3), energies[4] = E_LJ, E_RF, E_bond, E_angle) of -grad U."""
    ss = _Sys(s)
    pp = _params(p)
    X = np.ascontiguousarray(np.asarray(pos, np.float64).reshape(-1))
    F = np.zeros(3 * s.n_atoms)
    e = np.zeros(4)
    rc = lib().or_forces(C.byref(ss.c), C.byref(pp), X.ctypes.data, int(bool(use_list)), F.ctypes.data,
                         e.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"or_forces failed ({rc})")
    return F.reshape(-1, 3), e


def initial_velocities(s, temperature, seed):
    ss = _Sys(s)
    v = np.zeros(3 * s.n_atoms)
    lib().or_initial_velocities(C.byref(ss.c), float(temperature), int(seed), v.ctypes.data)
    return v.reshape(-1, 3)


def run(s, p, seed, n_steps, pos=None, vel=None, record_every=0, want_force=False):
    """One trial of n_steps biased BAOAB steps.  Returns a dict with per-step
    z, z_m, a, phi, the final state, Phi and the final energies."""
    ss = _Sys(s)
    pp = _params(p)
    n = s.n_atoms
    X = np.ascontiguousarray(np.asarray(s.pos if pos is None else pos, np.float64).reshape(-1))
    V = None
    if vel is not None or s.vel is not None:
        V = np.ascontiguousarray(np.asarray(vel if vel is not None else s.vel, np.float64).reshape(-1))
    z = np.zeros(n_steps + 1)
    zm = np.zeros(n_steps + 1)
    a = np.zeros(n_steps + 1)
    ph = np.zeros(n_steps + 1)
    frames = None
    if record_every > 0:
        frames = np.zeros((n_steps // record_every + 1, 3 * n))
    po = np.zeros(3 * n)
    vo = np.zeros(3 * n)
    fo = np.zeros(3 * n) if want_force else None
    out = OrRunOut(z=z.ctypes.data, zm=zm.ctypes.data, a=a.ctypes.data, phi_step=ph.ctypes.data,
                   frames=_p(frames), record_every=record_every, pos_out=po.ctypes.data, vel_out=vo.ctypes.data,
                   force_out=_p(fo))
    rc = lib().or_run(C.byref(ss.c), C.byref(pp), int(seed), X.ctypes.data, None if V is None else V.ctypes.data,
                      int(n_steps), C.byref(out))
    res = dict(status=rc, z=z, zm=zm, a=a, phi_step=ph, Phi=out.Phi, energies=np.array(out.energies[:]),
               pos=po.reshape(-1, 3), vel=vo.reshape(-1, 3))
    if frames is not None:
        res["frames"] = frames.reshape(frames.shape[0], n, 3)
    if fo is not None:
        res["force"] = fo.reshape(-1, 3)
    return res


def phi_frames(s, p, frames):
    """Bias functional along frames (n_frames, n_cv, 3); returns (Phi, z, a, phi)."""
    ss = _Sys(s)
    pp = _params(p)
    Fr = np.ascontiguousarray(np.asarray(frames, np.float64)[:, : s.n_cv, :].reshape(-1))
    nf = int(np.asarray(frames).shape[0])
    z = np.zeros(nf)
    a = np.zeros(nf)
    ph = np.zeros(nf)
    Phi = lib().or_phi_frames(C.byref(ss.c), C.byref(pp), Fr.ctypes.data, nf, z.ctypes.data, a.ctypes.data,
                              ph.ctypes.data)
    return Phi, z, a, ph


def phi_frames_grad(s, p, frames):
    """(Phi, dPhi/dframes (n_frames, n_cv, 3)) along frames (n_frames, >= n_cv, 3)."""
    ss = _Sys(s)
    pp = _params(p)
    Fr = np.ascontiguousarray(np.asarray(frames, np.float64)[:, : s.n_cv, :].reshape(-1))
    nf = int(np.asarray(frames).shape[0])
    G = np.zeros(nf * 3 * s.n_cv)
    Phi = lib().or_phi_frames_grad(C.byref(ss.c), C.byref(pp), Fr.ctypes.data, nf, G.ctypes.data)
    return Phi, G.reshape(nf, s.n_cv, 3)


def num_threads():
    return int(lib().or_num_threads())


def set_num_threads(k):
    lib().or_set_num_threads(int(k))


# ---------------------------------------------------------------------------
# two-dimensional toy model (SM, "Illustrative Application in a Toy Model")
# ---------------------------------------------------------------------------

def _toy_params(tp):
    return OrToy2dParams(**{f: float(getattr(tp, f)) for f, _ in OrToy2dParams._fields_ if f not in ("bias", "s_power")},
                         bias=int(tp.bias), s_power=int(tp.s_power))


def toy2d_force(tp, x, y):
    """(U, Fx, Fy) at (x, y)."""
    out = np.zeros(3)
    pp = _toy_params(tp)
    lib().or_toy2d_force(C.byref(pp), float(x), float(y), out[0:].ctypes.data, out[1:].ctypes.data,
                         out[2:].ctypes.data)
    return float(out[0]), float(out[1]), float(out[2])


def toy2d_run(tp, k, seed, n_steps, want_path=False):
    """One trial: (first passage step or -1, Phi, state (x, y, vx, vy), path (n, 2) or None)."""
    pp = _toy_params(tp)
    st = np.zeros(4)
    phi = np.zeros(1)
    path = np.zeros((n_steps + 1, 2)) if want_path else None
    n = lib().or_toy2d_run(C.byref(pp), float(k), int(seed), int(n_steps), st.ctypes.data, phi.ctypes.data,
                           None if path is None else path.ctypes.data)
    if path is not None:
        path = path[: (n + 1 if n >= 0 else n_steps + 1)]
    return int(n), float(phi[0]), st, path


def toy2d_phi_path(tp, k, path):
    """(Phi, first passage index or -1) of Eq. VMDcondition along a given path (n, 2)."""
    pp = _toy_params(tp)
    P = np.ascontiguousarray(np.asarray(path, np.float64).reshape(-1, 2))
    pas = np.zeros(1, np.int64)
    Phi = lib().or_toy2d_phi_path(C.byref(pp), float(k), P.ctypes.data, len(P), pas.ctypes.data)
    return float(Phi), int(pas[0])


# ---------------------------------------------------------------------------
# order of native-contact formation and path similarity (Sec. "Results")
# ---------------------------------------------------------------------------

def native_contacts(native, n_cv, r0, min_sep):
    """(Nc, 2) int32 pairs (i < j, j - i > min_sep) formed in the native structure."""
    nat = np.ascontiguousarray(np.asarray(native, np.float64)[:n_cv].reshape(-1))
    n = lib().or_native_contacts(nat.ctypes.data, int(n_cv), float(r0), int(min_sep), None, 0)
    pairs = np.zeros((max(n, 1), 2), np.int32)
    lib().or_native_contacts(nat.ctypes.data, int(n_cv), float(r0), int(min_sep), pairs.ctypes.data, n)
    return pairs[:n]


def contact_times(frames, steps, box, r0, pairs):
    """Formation time of each contact along frames (n_frames, n_cv, 3) at the given steps (-1: not formed at the end)."""
    F = np.ascontiguousarray(np.asarray(frames, np.float64))
    st = np.ascontiguousarray(steps, np.int64)
    pr = np.ascontiguousarray(pairs, np.int32)
    t = np.zeros(len(pr), np.int64)
    lib().or_contact_times(F.ctypes.data, st.ctypes.data, F.shape[0], F.shape[1], float(box), float(r0),
                           pr.ctypes.data, len(pr), t.ctypes.data)
    return t


def path_similarity(ta, tb):
    a = np.ascontiguousarray(ta, np.int64)
    b = np.ascontiguousarray(tb, np.int64)
    return float(lib().or_path_similarity(a.ctypes.data, b.ctypes.data, len(a)))


def refine_frames(s, p, frames, n_iter, step):
    """Descent on Phi over the inner frames of a path, end frames fixed, with
    Armijo backtracking (first trial step 2x the last accepted one, halved
    until Phi drops by 1e-4 eta |g|^2): FP64 restatement of the refinement.
    A trial point's moved coordinates are rounded to FP32, the precision the
    path's frames are held in, so that the path returned is exactly the one
    scored.  Returns (frames, Phi history [n_iter + 1], accepted iterations)."""
    X = np.array(frames, dtype=np.float64)[:, : s.n_cv, :].copy()
    phi, G = phi_frames_grad(s, p, X)
    G[0] = 0.0
    G[-1] = 0.0
    gg = float((G * G).sum())
    hist = [phi]
    eta, acc = step, 0
    for it in range(n_iter):
        ok = False
        for _ in range(40):
            if gg <= 0.0:
                break
            Y = X.copy()
            Y[1:-1] = (X[1:-1] - eta * G[1:-1]).astype(np.float32).astype(np.float64)
            phi_y = phi_frames(s, p, Y)[0]
            if phi_y <= phi - 1e-4 * eta * gg:
                X, phi, ok = Y, phi_y, True
                break
            eta *= 0.5
        if ok:
            phi, G = phi_frames_grad(s, p, X)
            G[0] = 0.0
            G[-1] = 0.0
            gg = float((G * G).sum())
            acc += 1
            eta *= 2.0
        hist.append(phi)
        if not ok:
            hist += [phi] * (n_iter - it - 1)
            break
    return X, np.array(hist), acc
