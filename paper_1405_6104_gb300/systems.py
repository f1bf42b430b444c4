"""Seeded synthetic inputs: solute-in-solvent systems and run parameters.

This module produces *inputs only*.  It holds none of the method's arithmetic
(no forces, no collective variable, no bias, no integrator, no random draws
that the method itself makes): the Langevin noise and the Maxwell-Boltzmann
initial velocities are drawn by each side from its own counter-based
generator.  Both the CUDA path and the CPU oracle consume what is built here.

The paper's workloads (Fip35 and villin in TIP3P water, Sec. "Results" and the
Supplementary Material) need PDB structures and force-field files that are not
available.  The systems below are stand-ins with the same structure: a solute
chain X (the only atoms the bias acts on, Eq. VR) immersed in an explicit
solvent Y (Eq. Lang), a native (target) structure that defines the reference
contact map C(X^native) of the collective variable (SM Sec. "Collective
coordinate"), and periodic cubic boxes.

Units: nm, ps, amu, kJ/mol, e, K.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

# ---------------------------------------------------------------------------
# containers
# ---------------------------------------------------------------------------


@dataclasses.dataclass
class System:
    """One periodic system.  Atoms [0, n_solute) are the solute X, the rest
    the solvent Y.  The collective-variable atoms are [0, n_cv)."""

    pos: np.ndarray            # (n, 3) float64, nm
    mass: np.ndarray           # (n,) amu
    charge: np.ndarray         # (n,) e
    lj_type: np.ndarray        # (n,) int32
    sigma: np.ndarray          # (n_types,) nm
    epsilon: np.ndarray        # (n_types,) kJ/mol
    bonds: np.ndarray          # (nb, 2) int32
    bond_r0: np.ndarray        # (nb,) nm
    bond_k: np.ndarray         # (nb,) kJ/mol/nm^2  (V = k/2 (r - r0)^2)
    angles: np.ndarray         # (na, 3) int32, middle atom is the vertex
    angle_t0: np.ndarray       # (na,) rad
    angle_k: np.ndarray        # (na,) kJ/mol/rad^2 (V = k/2 (t - t0)^2)
    box: float                 # cubic side, nm
    native_pos: np.ndarray     # (n_cv, 3) target structure of the CV atoms
    n_solute: int
    n_cv: int
    vel: Optional[np.ndarray] = None     # (n, 3) nm/ps, None -> Maxwell-Boltzmann draw
    gamma: Optional[np.ndarray] = None   # (n,) 1/ps, None -> Params.gamma
    excl_pairs: Optional[np.ndarray] = None  # (ne, 2) extra exclusions
    name: str = ""

    @property
    def n_atoms(self) -> int:
        return int(self.pos.shape[0])

    def copy(self) -> "System":
        return dataclasses.replace(
            self, **{f.name: (getattr(self, f.name).copy() if isinstance(getattr(self, f.name), np.ndarray) else getattr(self, f.name))
                     for f in dataclasses.fields(self)})


@dataclasses.dataclass
class Params:
    """Run parameters shared by every trial of a batch."""

    dt: float = 0.002              # ps
    temperature: float = 300.0     # K
    gamma: float = 1.0             # 1/ps (atoms without their own gamma)
    r_cut: float = 1.0             # nm, LJ + reaction-field cut-off
    skin: float = 0.1              # nm, Verlet buffer (r_list = r_cut + skin)
    nstlist: int = 10              # steps between list rebuilds
    eps_rf: float = 0.0            # reaction-field dielectric; <= 0 means infinity
    k_ratchet: float = 50.0        # k_R of Eq. VR, kJ/mol
    cv_r0: float = 0.75            # r_0 of the contact function, nm (SM: 7.5 A)
    cv_r_switch: float = 1.0       # switching starts, nm
    cv_r_cut: float = 1.2          # contact contributions vanish beyond, nm (SM: 12 A)
    cv_min_sep: int = 35           # pairs with j - i > cv_min_sep (SM: |i-j| > 35)
    seed: int = 0                  # trial t uses seed + t unless seeds are given
    flags: int = 0


# force-field constants of the synthetic models (fixed once here so both sides
# read identical data)
WATER_O = dict(mass=15.9994, charge=-0.834, sigma=0.315061, epsilon=0.636386)
# the hydrogen's small Lennard-Jones sphere (CHARMM's variant of TIP3P) keeps
# a hydrogen of this flexible water from collapsing onto an atom that attracts
# it (without it a hot start of the solvated systems can blow up)
WATER_H = dict(mass=1.008, charge=0.417, sigma=0.0400013, epsilon=0.192464)
WATER_OH = dict(r0=0.09572, k=462750.0)
WATER_HOH = dict(t0=math.radians(104.52), k=836.8)
POLY_CLASSES = dict(sigma=[0.25, 0.30, 0.34, 0.37], epsilon=[0.1, 0.4, 0.5, 0.8],
                    mass=[1.008, 12.011, 14.007, 15.999])
POLY_BOND = dict(r0=0.153, k=2.5e5)
POLY_ANGLE = dict(t0=math.radians(111.0), k=450.0)


# ---------------------------------------------------------------------------
# geometry helpers (input construction only)
# ---------------------------------------------------------------------------


class _Hash:  # noqa: D101 (kept for small systems)
    """Spatial hash of accepted points for overlap rejection (periodic)."""

    def __init__(self, box: float, cell: float):
        self.box = box
        self.n = max(1, int(box // cell))
        self.cell = box / self.n
        self.cells = {}

    def _key(self, p):
        return tuple(int(math.floor(c / self.cell)) % self.n for c in p)

    def add(self, p):
        self.cells.setdefault(self._key(p), []).append(np.asarray(p, dtype=np.float64))

    def min_dist2(self, p, reach: int = 1):
        k = self._key(p)
        best = np.inf
        L = self.box
        rng = range(-reach, reach + 1)
        seen = set()
        for dx in rng:
            for dy in rng:
                for dz in rng:
                    kk = ((k[0] + dx) % self.n, (k[1] + dy) % self.n, (k[2] + dz) % self.n)
                    if kk in seen:
                        continue
                    seen.add(kk)
                    for q in self.cells.get(kk, ()):
                        d = q - p
                        d -= L * np.round(d / L)
                        best = min(best, float(d @ d))
        return best


def box_exact(box: float) -> float:
    """Box sides are multiples of 2^-10 nm, exact in both FP32 and FP64, so
    that the float and the double minimum-image shifts coincide."""
    return round(float(box) * 1024.0) / 1024.0


def _f32exact(a):
    """Positions representable in FP32 (the kernels store FP32 coordinates);
    both sides then start from bit-identical states."""
    return np.asarray(a, np.float32).astype(np.float64)


def _rand_unit(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def _chain_walk(rng, n, bond, angle, centre, radius, min_dist, max_tries=200, max_backtracks=0):
    """Self-avoiding chain with fixed bond length and bond angle, random
    dihedrals, kept inside a sphere of the given radius.  When no trial
    position of an atom keeps min_dist from the chain, the best one is taken;
    with max_backtracks > 0 only if it keeps at least 0.8 min_dist, otherwise
    (a dense walk that has trapped itself) the walk backs up 8 atoms and
    continues from there, up to max_backtracks times (the starting coil of a
    solvated system, whose atoms interact)."""
    pts = np.zeros((n, 3))
    pts[0] = np.asarray(centre, dtype=np.float64)
    if n == 1:
        return pts
    d = _rand_unit(rng)
    pts[1] = pts[0] + bond * d
    backtracks = 0
    i = 2
    while i < n:
        best, best_score, best_md = None, -np.inf, np.inf
        a, b = pts[i - 2], pts[i - 1]
        u = (b - a) / np.linalg.norm(b - a)
        perp = np.cross(u, _rand_unit(rng))
        perp /= np.linalg.norm(perp)
        w = np.cross(u, perp)
        # only points within bond + min_dist of b can come within min_dist of a
        # candidate; the minimum over them equals the minimum over all points
        # whenever it is below min_dist, the only case in which its value matters
        prev = pts[:i - 2]
        reach = (bond + min_dist) * (1.0 + 1e-9)
        prev = prev[((prev - b) ** 2).sum(1) < reach * reach]
        for _ in range(max_tries):
            phi = rng.uniform(0, 2 * np.pi)
            dirn = -math.cos(angle) * u + math.sin(angle) * (math.cos(phi) * perp + math.sin(phi) * w)
            c = b + bond * dirn
            r_out = np.linalg.norm(c - centre) - radius
            md = np.sqrt(((prev - c) ** 2).sum(1)).min() if len(prev) else np.inf
            score = min(md - min_dist, 0.0) * 10.0 - max(r_out, 0.0)
            if md >= min_dist and r_out <= 0:
                best, best_md = c, md
                break
            if score > best_score:
                best, best_score, best_md = c, score, md
        if best_md < 0.8 * min_dist and backtracks < max_backtracks and i > 2:
            backtracks += 1
            i = max(2, i - 8)
            continue
        pts[i] = best
        i += 1
    return pts


def _lattice_hamiltonian_path(rng, dims, spacing):
    """Seeded Hamiltonian path through a small cubic lattice (compact chain)."""
    sites = [(i, j, k) for i in range(dims[0]) for j in range(dims[1]) for k in range(dims[2])]
    n = len(sites)
    order = list(range(n))
    rng.shuffle(order)

    def nbrs(s):
        out = []
        for ax in range(3):
            for dd in (-1, 1):
                t = list(s)
                t[ax] += dd
                if 0 <= t[ax] < dims[ax]:
                    out.append(tuple(t))
        return out

    def dfs(path, used):
        if len(path) == n:
            return path
        cand = nbrs(path[-1])
        rng.shuffle(cand)
        for c in cand:
            if c not in used:
                used.add(c)
                r = dfs(path + [c], used)
                if r:
                    return r
                used.discard(c)
        return None

    for s in order:
        p = dfs([sites[s]], {sites[s]})
        if p:
            return np.array(p, dtype=np.float64) * spacing
    raise RuntimeError("no Hamiltonian path")


def _place_solvent_points(rng, box, n, min_dist, occupied, occ_dist=0.25):
    """n solvent sites, periodic box: the sites of a cubic lattice of spacing
    a >= min_dist, visited in random order with a random jitter of at most
    (a - min_dist)/2 (so kept sites stay min_dist apart), keeping those that
    clear the occupied (solute) positions by occ_dist."""
    from scipy.spatial import cKDTree

    m = max(1, int(box // min_dist))
    a = box / m
    grid = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"), -1).reshape(-1, 3)
    grid = (grid + 0.5) * a
    jit = 0.5 * (a - min_dist)
    cand = (grid[rng.permutation(len(grid))] + rng.uniform(-jit, jit, size=(len(grid), 3))) % box
    if len(occupied):
        tree = cKDTree(np.asarray(occupied) % box, boxsize=box)
        d, _ = tree.query(cand, k=1)
        cand = cand[d >= occ_dist]
    if len(cand) < n:
        raise RuntimeError(f"solvent placement: {len(cand)} free sites < {n}; enlarge the box")
    return cand[:n]


def _exclusions_from_topology(bonds, angles):
    """1-2 and 1-3 pairs (the synthetic models have no dihedrals)."""
    ex = set()
    for a, b in bonds:
        ex.add((min(a, b), max(a, b)))
    for a, _, c in angles:
        ex.add((min(a, c), max(a, c)))
    return ex


# ---------------------------------------------------------------------------
# systems
# ---------------------------------------------------------------------------


def tiny_chain(seed: int = 0) -> tuple:
    """12-bead chain (alternating +-0.3 e, harmonic bonds k=1e5, r0=0.38 nm)
    in 200 neutral LJ particles (sigma 0.3 nm, epsilon 0.6 kJ/mol), 3.0 nm box,
    dt 2 fs, ratchet constant 50 kJ/mol.  The target structure is a compact
    Hamiltonian path on a 2x2x3 lattice of spacing 0.38 nm."""
    rng = np.random.default_rng(seed)
    L = 3.0
    n_b, n_s = 12, 200
    native = _lattice_hamiltonian_path(rng, (2, 2, 3), 0.38)
    native = native - native.mean(0) + L / 2
    chain = _chain_walk(rng, n_b, 0.38, math.radians(150.0), np.full(3, L / 2) - 0.5, 1.4, 0.45)
    chain = chain - chain.mean(0) + L / 2
    chain %= L
    solv = _place_solvent_points(rng, L, n_s, 0.3, list(chain), occ_dist=0.3)
    pos = _f32exact(np.concatenate([chain, solv]))
    n = n_b + n_s
    charge = np.zeros(n)
    charge[:n_b] = [0.3 if i % 2 == 0 else -0.3 for i in range(n_b)]
    mass = np.full(n, 18.0)
    mass[:n_b] = 12.011
    bonds = np.array([[i, i + 1] for i in range(n_b - 1)], dtype=np.int32)
    sysm = System(
        pos=pos, mass=mass, charge=charge, lj_type=np.zeros(n, np.int32),
        sigma=np.array([0.3]), epsilon=np.array([0.6]),
        bonds=bonds, bond_r0=np.full(len(bonds), 0.38), bond_k=np.full(len(bonds), 1e5),
        angles=np.zeros((0, 3), np.int32), angle_t0=np.zeros(0), angle_k=np.zeros(0),
        box=L, native_pos=native, n_solute=n_b, n_cv=n_b, name="tiny_chain_212")
    params = Params(dt=0.002, temperature=300.0, gamma=1.0, r_cut=1.0, skin=0.1, nstlist=10,
                    eps_rf=0.0, k_ratchet=50.0, cv_min_sep=2, seed=seed)
    return sysm, params


def solvated_heteropolymer(n_solute: int = 540, n_water: int = 3500, box: Optional[float] = None,
                           seed: int = 1, native_radius: Optional[float] = None,
                           coil_radius: Optional[float] = None, name: str = "") -> System:
    """Heteropolymer of n_solute atoms (4 LJ classes, charges N(0, 0.25 e)
    neutralised, bonds 0.153 nm and angles 111 deg) in n_water flexible 3-site
    waters (O -0.834 e, H +0.417 e, O-H 0.0957 nm, H-O-H 104.5 deg).  The box
    side defaults to 33 water-equivalents per nm^3.  The target structure is a
    compact self-avoiding fold; the starting structure an open coil."""
    rng = np.random.default_rng(seed)
    if box is None:
        box = ((n_water + n_solute / 3.0) / 33.0) ** (1.0 / 3.0)
    L = box_exact(box)
    scale = (n_solute / 540.0) ** (1.0 / 3.0)
    if native_radius is None:
        native_radius = 1.1 * scale
    if coil_radius is None:
        coil_radius = min(1.8 * scale, 0.42 * L)
    centre = np.full(3, L / 2)
    native = _chain_walk(rng, n_solute, POLY_BOND["r0"], POLY_ANGLE["t0"], centre, native_radius, 0.18)
    coil = _chain_walk(rng, n_solute, POLY_BOND["r0"], POLY_ANGLE["t0"], centre, coil_radius, 0.28,
                       max_backtracks=5000)
    coil %= L
    cls = rng.integers(0, 4, size=n_solute)
    q = rng.normal(0.0, 0.25, size=n_solute)
    q -= q.mean()
    o_pos = _place_solvent_points(rng, L, n_water, 0.27, list(coil), occ_dist=0.22)
    # water hydrogens: random orientation with the fixed geometry; orientations
    # that put an H within 0.15 nm of another molecule's atom are redrawn
    from scipy.spatial import cKDTree

    r0, t0 = WATER_OH["r0"], WATER_HOH["t0"]
    nw = len(o_pos)
    h1 = np.zeros((nw, 3))
    h2 = np.zeros((nw, 3))
    heavy = np.concatenate([coil % L, o_pos]) if n_solute else o_pos
    tree = cKDTree(heavy % L, boxsize=L)
    todo = np.arange(nw)
    for _ in range(30):
        if len(todo) == 0:
            break
        u = rng.normal(size=(len(todo), 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        w = np.cross(u, rng.normal(size=(len(todo), 3)))
        w /= np.linalg.norm(w, axis=1, keepdims=True)
        o = o_pos[todo]
        h1[todo] = o + r0 * u
        h2[todo] = o + r0 * (math.cos(t0) * u + math.sin(t0) * w)
        bad = np.zeros(len(todo), bool)
        for hpos in (h1[todo], h2[todo]):
            cnt = np.array([len(x) for x in tree.query_ball_point(hpos % L, 0.15)])
            bad |= cnt > 1  # its own oxygen is always within 0.15 nm
        todo = todo[bad]
    waters = list(zip(o_pos, h1, h2))
    n = n_solute + 3 * n_water
    pos = np.zeros((n, 3))
    pos[:n_solute] = coil
    mass = np.zeros(n)
    charge = np.zeros(n)
    lj_type = np.zeros(n, np.int32)
    mass[:n_solute] = np.array(POLY_CLASSES["mass"])[cls]
    charge[:n_solute] = q
    lj_type[:n_solute] = cls
    bonds = [[i, i + 1] for i in range(n_solute - 1)]
    bond_r0 = [POLY_BOND["r0"]] * (n_solute - 1)
    bond_k = [POLY_BOND["k"]] * (n_solute - 1)
    angles = [[i, i + 1, i + 2] for i in range(n_solute - 2)]
    angle_t0 = [POLY_ANGLE["t0"]] * (n_solute - 2)
    angle_k = [POLY_ANGLE["k"]] * (n_solute - 2)
    for w, (o, h1, h2) in enumerate(waters):
        a = n_solute + 3 * w
        pos[a], pos[a + 1], pos[a + 2] = o, h1 % L, h2 % L
        mass[a], mass[a + 1], mass[a + 2] = WATER_O["mass"], WATER_H["mass"], WATER_H["mass"]
        charge[a], charge[a + 1], charge[a + 2] = WATER_O["charge"], WATER_H["charge"], WATER_H["charge"]
        lj_type[a], lj_type[a + 1], lj_type[a + 2] = 4, 5, 5
        bonds += [[a, a + 1], [a, a + 2]]
        bond_r0 += [WATER_OH["r0"]] * 2
        bond_k += [WATER_OH["k"]] * 2
        angles.append([a + 1, a, a + 2])
        angle_t0.append(WATER_HOH["t0"])
        angle_k.append(WATER_HOH["k"])
    sigma = np.array(POLY_CLASSES["sigma"] + [WATER_O["sigma"], WATER_H["sigma"]])
    epsilon = np.array(POLY_CLASSES["epsilon"] + [WATER_O["epsilon"], WATER_H["epsilon"]])
    return System(
        pos=_f32exact(pos % L), mass=mass, charge=charge, lj_type=lj_type, sigma=sigma, epsilon=epsilon,
        bonds=np.array(bonds, np.int32).reshape(-1, 2), bond_r0=np.array(bond_r0), bond_k=np.array(bond_k),
        angles=np.array(angles, np.int32).reshape(-1, 3), angle_t0=np.array(angle_t0), angle_k=np.array(angle_k),
        box=L, native_pos=native, n_solute=n_solute, n_cv=n_solute,
        name=name or f"heteropolymer{n_solute}_water{n_water}")


def protein_params(seed: int = 1, k_ratchet: float = 5e-3, dt: float = 0.001) -> Params:
    """Parameters of the solvated-heteropolymer workloads: dt 1 fs, 300 K,
    reaction field with a 1.0 nm cut-off, k_R = 5e-3 kJ/mol (the paper's
    value for its protein runs), contact pairs with |i - j| > 35."""
    return Params(dt=dt, temperature=300.0, gamma=1.0, r_cut=1.0, skin=0.1, nstlist=10,
                  eps_rf=0.0, k_ratchet=k_ratchet, cv_min_sep=35, seed=seed)


def plain_single(seed: int = 1):
    """540-atom heteropolymer + 3500 waters = 11 040 atoms in a 4.8 nm box."""
    return solvated_heteropolymer(540, 3500, box=4.8, seed=seed, name="plain_11040"), protein_params(seed)


def batched_64(seed: int = 1):
    """64 trials of the 11 040-atom system; trial t uses Philox seed 1000 + t
    and its own Maxwell-Boltzmann velocities."""
    s, p = plain_single(seed)
    p.seed = 1000
    return s, p, [1000 + t for t in range(64)]


def uneven_32(seed: int = 2, n_systems: int = 32, n_min: int = 5000, n_max: int = 60000):
    """32 systems, total atom counts log-uniform in [5k, 60k], solute sizes
    log-uniform in [200, 2000] capped at N/5, boxes at 33 water-equivalents
    per nm^3."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_systems):
        n_tot = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        n_sol = int(round(math.exp(rng.uniform(math.log(200), math.log(2000)))))
        n_sol = min(n_sol, n_tot // 5)
        n_w = (n_tot - n_sol) // 3
        out.append(solvated_heteropolymer(n_sol, n_w, seed=seed * 1000 + k, name=f"uneven{k}_{n_sol + 3 * n_w}"))
    return out, protein_params(seed)


def adjoint_30k(seed: int = 3):
    """30 000 atoms: 1800-atom solute + 9400 waters."""
    return solvated_heteropolymer(1800, 9400, seed=seed, name="adjoint_30000"), protein_params(seed)


def small_solvated(n_solute: int = 60, n_water: int = 420, seed: int = 5, cv_min_sep: int = 4):
    """A few-hundred-atom solvated chain for fast parity tests that still span
    many clusters and a ragged tail (n_atoms not a multiple of 8)."""
    s = solvated_heteropolymer(n_solute, n_water, seed=seed, name=f"small{n_solute}_{n_water}")
    p = protein_params(seed, k_ratchet=5.0, dt=0.001)
    p.cv_min_sep = cv_min_sep
    return s, p


# ---------------------------------------------------------------------------
# two-dimensional toy model (SM, "Illustrative Application in a Toy Model")
# ---------------------------------------------------------------------------

TOY_NONE, TOY_RATCHET, TOY_STEERED = 0, 1, 2


@dataclasses.dataclass
class Toy2dParams:
    """The toy model's potential and Langevin parameters as the paper gives
    them (A1 = 30, A2 = 20, A3 = 6, s1 = 1, s2 = 2, s3 = 2, w = 0.03, gate at
    (1.5, 0); gamma = 1, dt = 0.02, k_B T = 0.2; start (0, 5)).  The mass is
    not stated (m = 1); the product counts as reached when z = sqrt(x^2 + y^2)
    <= z_product (0.3: well inside the funnel, whose thermal spread at the
    bottom is about 0.04).  s_power is the exponent of s in the numerators of
    the three well terms: the section prints 2, which leaves no ring barrier
    (every plain trajectory reaches the funnel within about a thousand
    steps); 4 (amplitude A at each centre) gives the barrier and the gate the
    section describes and is the default."""
    A1: float = 30.0
    A2: float = 20.0
    A3: float = 6.0
    s1: float = 1.0
    s2: float = 2.0
    s3: float = 2.0
    w: float = 0.03
    xm: float = 1.5
    ym: float = 0.0
    mass: float = 1.0
    gamma: float = 1.0
    kT: float = 0.2
    dt: float = 0.02
    x0: float = 0.0
    y0: float = 5.0
    z_product: float = 0.3
    bias: int = TOY_RATCHET
    s_power: int = 4


def toy2d_rmd_batch(n_trials: int = 2000, k_values: Sequence[float] = (1.0,), seed0: int = 5000):
    """rMD trials of the toy model: n_trials per bias strength, trial seeds
    seed0 + index (the paper: 2000 trials of 30 000 steps per K_R)."""
    ks = np.repeat(np.asarray(k_values, np.float64), n_trials)
    seeds = seed0 + np.arange(len(ks), dtype=np.uint64)
    return Toy2dParams(bias=TOY_RATCHET), ks, seeds


def toy2d_plain_batch(n_trials: int = 20000, seed0: int = 9000):
    """Plain Langevin trials of the toy model (the paper: 20 000 trials of
    90 000 steps)."""
    return Toy2dParams(bias=TOY_NONE), np.zeros(n_trials), seed0 + np.arange(n_trials, dtype=np.uint64)
