"""Pins of the FP64 CPU oracle against facts fixed by the paper, by the
published definitions it relies on, and by mathematics -- never against the
oracle itself.  Each test names the passage it follows.  CPU only."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_1405_6104_gb300 import systems as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
KB = 0.0083144626
FCOUL = 138.935458


def tiny_system(pos, *, mass=None, charge=None, types=None, sigma=(0.3,), epsilon=(0.6,), bonds=(), bond_r0=(),
                bond_k=(), angles=(), angle_t0=(), angle_k=(), box=20.0, native=None, n_cv=None):
    pos = np.asarray(pos, np.float64)
    n = len(pos)
    n_cv = n if n_cv is None else n_cv
    return S.System(
        pos=pos, mass=np.ones(n) * 10.0 if mass is None else np.asarray(mass, float),
        charge=np.zeros(n) if charge is None else np.asarray(charge, float),
        lj_type=np.zeros(n, np.int32) if types is None else np.asarray(types, np.int32),
        sigma=np.asarray(sigma, float), epsilon=np.asarray(epsilon, float),
        bonds=np.asarray(bonds, np.int32).reshape(-1, 2), bond_r0=np.asarray(bond_r0, float),
        bond_k=np.asarray(bond_k, float), angles=np.asarray(angles, np.int32).reshape(-1, 3),
        angle_t0=np.asarray(angle_t0, float), angle_k=np.asarray(angle_k, float), box=box,
        native_pos=(pos[:n_cv].copy() if native is None else np.asarray(native, float)), n_solute=n_cv, n_cv=n_cv)


# ---------------------------------------------------------------------------
# Philox4x32-10 (noise eta of Eq. Lang; Salmon et al. SC'11)
# ---------------------------------------------------------------------------

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_normals_moments_and_ks():
    from scipy import stats
    xs = np.array([O.normal3(12345, a, st, 0) for a in range(200) for st in range(1, 101)]).reshape(-1)
    assert abs(xs.mean()) < 5 / math.sqrt(len(xs))
    assert abs(xs.var() - 1) < 5 * math.sqrt(2 / len(xs))
    assert abs(stats.kurtosis(xs)) < 0.1
    assert stats.kstest(xs, "norm").pvalue > 1e-3
    # different streams / steps / atoms give uncorrelated draws
    a = np.array([O.normal3(7, i, 3, 0)[0] for i in range(4000)])
    b = np.array([O.normal3(7, i, 3, 1)[0] for i in range(4000)])
    c = np.array([O.normal3(7, i, 4, 0)[0] for i in range(4000)])
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.06 and abs(np.corrcoef(a, c)[0, 1]) < 0.06


# ---------------------------------------------------------------------------
# contact function of the reaction coordinate (SM, "Collective coordinate")
# ---------------------------------------------------------------------------

def _C_exact(r, r0):
    """(1 - rho^6)/(1 - rho^10) in exact rational arithmetic (rho != 1)."""
    rho = Fraction(r) / Fraction(r0)
    return float((1 - rho ** 6) / (1 - rho ** 10))


@pytest.mark.parametrize("r", [0.1, 0.3, 0.5, 0.7, 0.7499, 0.7501, 0.8, 0.95, 1.3, 2.0, 5.0])
def test_contact_matches_printed_formula(r):
    c = O.contact(r, 0.75, 10.0, 11.0)  # switch far away: C~ = C
    assert c[0] == pytest.approx(_C_exact(r, 0.75), rel=1e-14, abs=1e-16)
    assert c[1] == c[0]


def test_contact_special_values():
    assert O.contact(0.75, 0.75, 1.0, 1.2)[0] == pytest.approx(0.6, abs=1e-15)   # removable singularity
    assert O.contact(1e-12, 0.75, 1.0, 1.2)[0] == pytest.approx(1.0, abs=1e-12)  # C(0) = 1
    # large r: C -> (r0/r)^4
    for r in (20.0, 80.0):
        assert O.contact(r, 0.75, 1e3, 2e3)[0] / (0.75 / r) ** 4 == pytest.approx(1.0, rel=5e-3 * (20 / r) ** 2)
    # at r0 the slope is -1.2/r0 (expansion of the printed ratio around rho = 1)
    assert O.contact(0.75, 0.75, 1.0, 1.2)[2] == pytest.approx(-1.2 / 0.75, rel=1e-12)


def test_contact_derivatives_by_finite_differences():
    h = 1e-6
    for r in np.linspace(0.2, 1.4, 49):
        c = O.contact(r, 0.75, 1.0, 1.2)
        cp, cm = O.contact(r + h, 0.75, 1.0, 1.2), O.contact(r - h, 0.75, 1.0, 1.2)
        assert c[2] == pytest.approx((cp[0] - cm[0]) / (2 * h), rel=1e-6, abs=1e-8)
        assert c[3] == pytest.approx((cp[1] - cm[1]) / (2 * h), rel=1e-6, abs=1e-8)


def test_switch_is_smooth_and_vanishes_beyond_cut():
    rs, rc = 1.0, 1.2
    assert O.contact(rc, 0.75, rs, rc)[1] == 0.0 and O.contact(1.5, 0.75, rs, rc)[1] == 0.0
    assert O.contact(rs, 0.75, rs, rc)[1] == O.contact(rs, 0.75, rs, rc)[0]
    for r in (rs, rc):  # value and slope continuous at both ends
        lo, hi = O.contact(r - 1e-9, 0.75, rs, rc), O.contact(r + 1e-9, 0.75, rs, rc)
        assert abs(lo[1] - hi[1]) < 1e-8 and abs(lo[3] - hi[3]) < 1e-6


# ---------------------------------------------------------------------------
# reaction coordinate z (SM eq. for z) and its gradient
# ---------------------------------------------------------------------------

def test_cv_worked_case():
    """Four atoms, pairs with j - i > 2: only (0, 3) counts.  Current distance
    r0 (C = 3/5), native distance r0*sqrt(3/2) = 0.919 nm, inside the
    switching radius (s = 3/2: C = 76/211), so z = (3/5 - 76/211)^2 =
    (253/1055)^2."""
    r0 = 0.75
    pos = [[0, 0, 0], [0.3, 0.2, 0], [0.5, 0.6, 0.1], [r0, 0, 0]]
    nat = [[0, 0, 0], [0.2, 0.3, 0], [0.4, 0.1, 0.5], [r0 * math.sqrt(1.5), 0, 0]]
    s = tiny_system(pos, native=nat)
    p = S.Params(cv_min_sep=2)
    z, g = O.cv(s, p, np.asarray(pos))
    assert z == pytest.approx((253 / 1055) ** 2, rel=1e-14)
    # gradient of the single pair: dz/dx_3 = 2 (3/5 - 76/211) C'(r0) x_hat = 2 (253/1055)(-1.6) x_hat
    assert g[3] == pytest.approx([2 * (253 / 1055) * (-1.6), 0, 0], rel=1e-12)
    assert np.allclose(g[1], 0) and np.allclose(g[2], 0)
    assert np.allclose(g.sum(0), 0, atol=1e-14)


def test_cv_native_is_zero_and_gradient_fd():
    s, p = S.tiny_chain(0)
    z0, g0 = O.cv(s, p, s.native_pos)
    assert z0 == 0.0 and np.all(g0 == 0.0)
    X = s.pos[: s.n_cv].copy()
    z, g = O.cv(s, p, X)
    assert z > 0
    rng = np.random.default_rng(0)
    h = 1e-6
    for _ in range(20):
        i, k = rng.integers(s.n_cv), rng.integers(3)
        Xp, Xm = X.copy(), X.copy()
        Xp[i, k] += h
        Xm[i, k] -= h
        fd = (O.cv(s, p, Xp)[0] - O.cv(s, p, Xm)[0]) / (2 * h)
        assert g[i, k] == pytest.approx(fd, rel=1e-6, abs=1e-7)
    assert np.allclose(g.sum(0), 0, atol=1e-10)  # translation invariance


def test_cv_rigid_motion_invariance_and_pair_set():
    s, p = S.tiny_chain(0)
    s.box = 50.0
    X = s.pos[: s.n_cv] + 20.0
    z = O.cv(s, p, X)[0]
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    Y = (X - X.mean(0)) @ R.T + X.mean(0) + np.array([0.31, -0.2, 0.11])
    assert O.cv(s, p, Y)[0] == pytest.approx(z, rel=1e-12)
    # moving a pair that the |i - j| rule excludes changes nothing
    p2 = S.Params(cv_min_sep=s.n_cv - 2)  # only (0, n-1)
    X2 = X.copy()
    X2[1] += 0.05
    assert O.cv(s, p2, X)[0] == O.cv(s, p2, X2)[0]


# ---------------------------------------------------------------------------
# potential U and forces (stand-in force field for Eq. Lang's U)
# ---------------------------------------------------------------------------

def _two(r, **kw):
    return tiny_system([[5, 5, 5], [5 + r, 5, 5]], **kw)


def test_lj_closed_forms_and_mixing():
    p = S.Params(r_cut=1.0)
    sig, eps = 0.3, 0.6
    shift = 4 * eps * ((sig / 1.0) ** 12 - (sig / 1.0) ** 6)
    F, e = O.forces(_two(sig), p, _two(sig).pos)
    assert e[0] == pytest.approx(-shift, abs=1e-12)
    rmin = 2 ** (1 / 6) * sig
    F, e = O.forces(_two(rmin), p, _two(rmin).pos)
    assert e[0] == pytest.approx(-eps - shift, rel=1e-12)
    assert np.abs(F).max() < 1e-9
    # Lorentz-Berthelot: sigma_ij = (0.2 + 0.4)/2, eps_ij = sqrt(0.1 * 0.9)
    s = _two(0.3, types=[0, 1], sigma=[0.2, 0.4], epsilon=[0.1, 0.9])
    F, e = O.forces(s, p, s.pos)
    eps_ij = math.sqrt(0.09)
    assert e[0] == pytest.approx(-4 * eps_ij * ((0.3 / 1.0) ** 12 - (0.3 / 1.0) ** 6), rel=1e-12)
    # beyond the cut-off nothing
    F, e = O.forces(_two(1.05), p, _two(1.05).pos)
    assert e[0] == 0 and np.all(F == 0)


def test_reaction_field_closed_form():
    p = S.Params(r_cut=1.0, eps_rf=0.0)  # eps_rf = infinity
    for r in (0.3, 0.6, 0.999999):
        s = _two(r, charge=[0.5, -0.4], epsilon=[0.0])
        F, e = O.forces(s, p, s.pos)
        qq = FCOUL * 0.5 * -0.4
        assert e[1] == pytest.approx(qq * (1 / r + r * r / 2 - 1.5), rel=1e-12)
        assert F[0, 0] == pytest.approx(-qq * (1 / r ** 2 - r), rel=1e-10, abs=1e-9)
    # potential and force both vanish at the cut-off for eps_rf = infinity
    s = _two(1.0 - 1e-9, charge=[1.0, 1.0], epsilon=[0.0])
    F, e = O.forces(s, p, s.pos)
    assert abs(e[1]) < 1e-6 and abs(F[0, 0]) < 1e-5
    # finite eps_rf = 1 is plain cut-off Coulomb shifted to zero at r_c
    p1 = S.Params(r_cut=1.0, eps_rf=1.0)
    s = _two(0.5, charge=[1.0, 1.0], epsilon=[0.0])
    assert O.forces(s, p1, s.pos)[1][1] == pytest.approx(FCOUL * (1 / 0.5 - 1.0), rel=1e-12)


def test_bond_and_angle_closed_forms():
    p = S.Params(r_cut=1.0)
    s = _two(0.41, bonds=[[0, 1]], bond_r0=[0.38], bond_k=[1e5], epsilon=[0.0])
    F, e = O.forces(s, p, s.pos)
    assert e[2] == pytest.approx(0.5 * 1e5 * 0.03 ** 2, rel=1e-10)
    assert F[0, 0] == pytest.approx(1e5 * 0.03, rel=1e-8) and F[1, 0] == pytest.approx(-1e5 * 0.03, rel=1e-8)
    th = math.radians(100.0)
    pos = [[5 + 0.1, 5, 5], [5, 5, 5], [5 + 0.1 * math.cos(th), 5 + 0.1 * math.sin(th), 5]]
    s = tiny_system(pos, angles=[[0, 1, 2]], angle_t0=[math.radians(104.52)], angle_k=[836.8], epsilon=[0.0])
    F, e = O.forces(s, p, s.pos)
    assert e[3] == pytest.approx(0.5 * 836.8 * (th - math.radians(104.52)) ** 2, rel=1e-10)
    assert np.allclose(F.sum(0), 0, atol=1e-9)
    # torque-free: the angle force on the end atom is perpendicular to its arm
    assert abs(F[0] @ (np.array(pos[0]) - pos[1])) < 1e-9


@pytest.mark.parametrize("which", ["tiny", "small"])
def test_forces_are_minus_gradient(which):
    s, p = S.tiny_chain(0) if which == "tiny" else S.small_solvated()
    X = s.pos.copy()
    F, e = O.forces(s, p, X)
    assert np.abs(F.sum(0)).max() < 1e-8 * max(1.0, np.abs(F).max())  # Newton's third law
    rng = np.random.default_rng(1)
    h = 1e-5
    idx = rng.choice(s.n_atoms, size=12, replace=False)
    for i in idx:
        for k in range(3):
            Xp, Xm = X.copy(), X.copy()
            Xp[i, k] += h
            Xm[i, k] -= h
            Up, Um = O.forces(s, p, Xp)[1].sum(), O.forces(s, p, Xm)[1].sum()
            fd = -(Up - Um) / (2 * h)
            assert F[i, k] == pytest.approx(fd, rel=1e-6, abs=1e-5 * max(1, abs(F[i, k])) + 1e-6)


def test_brute_force_equals_verlet_list_on_small_box():
    s, p = S.small_solvated()
    F1, e1 = O.forces(s, p, s.pos, use_list=False)
    F2, e2 = O.forces(s, p, s.pos, use_list=True)
    assert np.allclose(F1, F2, rtol=1e-12, atol=1e-9) and np.allclose(e1, e2, rtol=1e-12)


def test_pairlist_rule_brackets_fp64_distances():
    s, p = S.small_solvated()
    posf = s.pos.astype(np.float32)
    pairs = O.pairlist(s, posf, p.r_cut + p.skin)
    L = s.box
    d = posf[pairs[:, 1]].astype(np.float64) - posf[pairs[:, 0]]
    d -= L * np.round(d / L)
    r = np.sqrt((d ** 2).sum(1))
    assert r.max() < 1.1 + 1e-5
    # every non-excluded pair clearly inside r_list is present
    X = posf.astype(np.float64)
    dd = X[None] - X[:, None]
    dd -= L * np.round(dd / L)
    rr = np.sqrt((dd ** 2).sum(-1))
    iu = np.triu_indices(s.n_atoms, 1)
    inside = set(zip(*[a[rr[iu] < 1.1 - 1e-5] for a in iu]))
    excl = {tuple(sorted(b)) for b in s.bonds.tolist()} | {tuple(sorted((a[0], a[2]))) for a in s.angles.tolist()}
    got = set(map(tuple, pairs.tolist()))
    assert inside - excl <= got
    assert not (got & excl)


# ---------------------------------------------------------------------------
# integrator (Eq. Lang, BAOAB) and thermostat
# ---------------------------------------------------------------------------

def test_energy_conservation_without_friction_and_bias():
    s, p = S.tiny_chain(0)
    p.gamma, p.k_ratchet = 0.0, 0.0
    n = 1000
    X = s.pos.copy()
    r0 = O.run(s, p, 3, 0)
    v0 = r0["vel"]
    es = []
    for k in range(0, n + 1, 50):
        r = O.run(s, p, 3, k, pos=X, vel=v0)
        es.append(r["energies"][:5])
    es = np.array(es)
    etot = es.sum(1)
    ekin = es[:, 4]
    assert np.std(etot) < 0.01 * np.std(ekin) + 1e-9
    drift = abs(etot[-1] - etot[0]) / (n * p.dt) / s.n_atoms
    assert drift < 1e-3  # kJ/mol/ps per atom


def test_displacement_triggered_lists_give_the_cut_off_model():
    """U of Eq. Lang is the cut-off potential: every pair closer than r_cut
    interacts.  With lists rebuilt once an atom has moved skin/2 (minus
    1e-5 nm), a thin buffer of 0.02 nm must give the same trajectory as a
    0.4 nm buffer (whose lists, rebuilt every 10 steps, cover every pair that
    can come within r_cut), up to rounding; fixed 20-step intervals with the
    thin buffer miss pairs and do not."""
    s, p = S.tiny_chain(0)
    p.k_ratchet = 0.0
    n = 300
    thick = S.Params(**{**p.__dict__, "skin": 0.4, "nstlist": 10, "flags": 4})
    ref = O.run(s, thick, 5, n)
    thin = O.run(s, S.Params(**{**p.__dict__, "skin": 0.02, "nstlist": 20}), 5, n)
    fixed = O.run(s, S.Params(**{**p.__dict__, "skin": 0.02, "nstlist": 20, "flags": 4}), 5, n)
    L = s.box
    dev = lambda r: np.abs((r["pos"] - ref["pos"]) - L * np.round((r["pos"] - ref["pos"]) / L)).max()
    # the thick buffer itself: 10 steps of 2 fs move no atom 0.2 nm at 300 K
    assert all(r["status"] == 0 for r in (ref, thin, fixed))
    assert dev(thin) < 1e-8
    assert dev(fixed) > 1e-6


def test_thermostat_equipartition():
    s, p = S.tiny_chain(0)
    p.gamma, p.k_ratchet = 10.0, 0.0
    r = O.run(s, p, 11, 6000, record_every=0)
    # average kinetic energy over the second half from restarts is costly;
    # use one long run and per-species velocities at many checkpoints
    kin_s, kin_b = [], []
    X, V = r["pos"], r["vel"]
    for _ in range(20):
        r = O.run(s, p, 11 + _, 100, pos=X, vel=V)
        X, V = r["pos"], r["vel"]
        kin_b.append(0.5 * (s.mass[: s.n_solute, None] * V[: s.n_solute] ** 2).sum() / (1.5 * s.n_solute))
        kin_s.append(0.5 * (s.mass[s.n_solute:, None] * V[s.n_solute:] ** 2).sum() / (1.5 * (s.n_atoms - s.n_solute)))
    kT = KB * p.temperature
    assert np.mean(kin_s) == pytest.approx(kT, rel=0.04)
    assert np.mean(kin_b) == pytest.approx(kT, rel=0.25)


def test_initial_velocities_maxwell_boltzmann():
    s, p = S.small_solvated()
    v = O.initial_velocities(s, 300.0, 99)
    assert np.abs((s.mass[:, None] * v).sum(0)).max() < 1e-10
    kT = KB * 300.0
    assert np.mean(s.mass[:, None] * v ** 2) == pytest.approx(kT, rel=0.05)


# ---------------------------------------------------------------------------
# ratchet bias (Eq. VR) and functional (Eq. VMDcondition)
# ---------------------------------------------------------------------------

def test_functional_worked_two_frame_case():
    """Two CV atoms (min_sep 0), one pair.  Frame 0 at the native distance
    (z = 0, z_m = 0), frame 1 at r0 with native distance 0.5 r0: a = z_1,
    |grad_i z|^2 = (2 h C'(r0))^2 for both atoms, so
    Phi = dt (k_R/2)^2 a^2 (2 h C')^2 (1/(g m_0) + 1/(g m_1))."""
    r0 = 0.75
    nat = np.array([[5, 5, 5], [5 + 0.5 * r0, 5, 5]])
    s = tiny_system(nat.copy(), mass=[12.0, 16.0], native=nat)
    p = S.Params(cv_min_sep=0, k_ratchet=7.0, dt=0.002, gamma=2.0)
    f1 = np.array([[5, 5, 5], [5 + r0, 5, 5]])
    Phi, z, a, phi = O.phi_frames(s, p, np.stack([nat, f1]))
    Cn = _C_exact(0.5 * r0, r0)
    h = 0.6 - Cn
    assert z[0] == 0 and z[1] == pytest.approx(h * h, rel=1e-14)
    g2 = (2 * h * -1.6) ** 2
    expect = p.dt * (p.k_ratchet / 2) ** 2 * (h * h) ** 2 * g2 * (1 / (2.0 * 12.0) + 1 / (2.0 * 16.0))
    assert Phi == pytest.approx(expect, rel=1e-12)


def test_functional_zero_cases_and_ratchet_bookkeeping():
    s, p = S.tiny_chain(0)
    # k_R = 0: no bias, Phi exactly 0
    p0 = S.Params(**{**p.__dict__, "k_ratchet": 0.0})
    assert O.run(s, p0, 5, 200)["Phi"] == 0.0
    # a path along which z never increases carries no bias
    nat = s.native_pos
    X0 = s.pos[: s.n_cv]
    frames = np.stack([nat + (1 - t) * (X0 - nat) for t in np.linspace(0, 1, 30)])
    Phi, z, a, _ = O.phi_frames(s, p, frames)
    assert np.all(np.diff(z) <= 0) and Phi == 0.0
    # reversed path: z increases, every step is biased
    Phi_r, z_r, a_r, _ = O.phi_frames(s, p, frames[::-1])
    assert Phi_r > 0 and np.all(a_r[1:] > 0)
    # trajectory bookkeeping: z_m(0) = z(X_0), running minimum, a = (z - z_m_prev)+, Phi = dt sum phi
    r = O.run(s, p, 5, 400)
    z, zm, a = r["z"], r["zm"], r["a"]
    assert zm[0] == z[0] and a[0] == 0.0
    assert np.all(zm == np.minimum.accumulate(z))
    assert np.allclose(a[1:], np.maximum(z[1:] - zm[:-1], 0.0), rtol=0, atol=0)
    assert r["Phi"] == pytest.approx(p.dt * r["phi_step"][1:].sum(), rel=1e-12)
    assert np.all(r["phi_step"] >= 0) and r["Phi"] > 0
    # z_m updated before or after the force: identical bias (if z > z_m_old then min(z_m_old, z) = z_m_old)
    a_after = np.maximum(z[1:] - np.minimum(zm[:-1], z[1:]), 0.0)
    assert np.array_equal(a_after, a[1:])


def test_bias_force_is_minus_gradient_of_ratchet_potential():
    """At fixed z_m the printed force equals -grad of (k_R/4)(z - z_m)_+^2."""
    s, p = S.tiny_chain(0)
    X = s.pos[: s.n_cv].copy()
    z, g = O.cv(s, p, X)
    zm = z - 0.37
    a = z - zm
    Fb = -(p.k_ratchet / 2) * a * g
    h = 1e-6
    for i, k in [(0, 0), (3, 1), (7, 2), (11, 0)]:
        Xp, Xm = X.copy(), X.copy()
        Xp[i, k] += h
        Xm[i, k] -= h
        Vp = p.k_ratchet / 4 * max(O.cv(s, p, Xp)[0] - zm, 0) ** 2
        Vm = p.k_ratchet / 4 * max(O.cv(s, p, Xm)[0] - zm, 0) ** 2
        assert Fb[i, k] == pytest.approx(-(Vp - Vm) / (2 * h), rel=1e-6, abs=1e-8)


def test_full_tiny_run_is_finite():
    s, p = S.tiny_chain(0)
    r = O.run(s, p, 0, 2000)
    assert r["status"] == 0 and np.isfinite(r["Phi"]) and r["Phi"] > 0
    assert r["zm"][-1] <= r["z"][0]


# ---------------------------------------------------------------------------
# adjoint of the functional with respect to the frames
# ---------------------------------------------------------------------------

def _biased_path(s, p, n=24):
    """A path along which z rises (every step biased) with a dip in the
    middle, so that the running minimum changes and routes gradient back."""
    nat, X0 = s.native_pos, s.pos[: s.n_cv]
    ts = np.concatenate([np.linspace(0.1, 0.6, n // 2), np.linspace(0.55, 1.0, n - n // 2)])
    rng = np.random.default_rng(3)
    return np.stack([nat + t * (X0 - nat) + 0.01 * rng.normal(size=nat.shape) for t in ts])


def test_functional_adjoint_matches_finite_differences():
    s, p = S.tiny_chain(0)
    fr = _biased_path(s, p)
    Phi, G = O.phi_frames_grad(s, p, fr)
    assert Phi == pytest.approx(O.phi_frames(s, p, fr)[0], rel=1e-14)
    _, z, a, _ = O.phi_frames(s, p, fr)
    assert (a[1:] > 0).sum() >= len(a) // 2
    h = 1e-6
    rng = np.random.default_rng(4)
    checked = 0
    for _ in range(120):
        f, i, k = rng.integers(len(fr)), rng.integers(s.n_cv), rng.integers(3)
        A, Bm = fr.copy(), fr.copy()
        A[f, i, k] += h
        Bm[f, i, k] -= h
        (PA, zA, aA, _), (PB, zB, aB, _) = O.phi_frames(s, p, A), O.phi_frames(s, p, Bm)
        # skip coordinates where +-h flips a ratchet branch or the running minimum
        if not (np.array_equal(aA > 0, a > 0) and np.array_equal(aB > 0, a > 0)):
            continue
        if not (np.array_equal(np.minimum.accumulate(zA) == zA, np.minimum.accumulate(z) == z)):
            continue
        fd = (PA - PB) / (2 * h)
        assert G[f, i, k] == pytest.approx(fd, rel=1e-5, abs=1e-7 * max(1.0, np.abs(G).max()))
        checked += 1
    assert checked > 80
    # the first frame only enters through the running minimum
    assert np.abs(G[0]).max() > 0


def test_functional_adjoint_zero_cases():
    s, p = S.tiny_chain(0)
    nat, X0 = s.native_pos, s.pos[: s.n_cv]
    fr = np.stack([nat + t * (X0 - nat) for t in np.linspace(1.0, 0.1, 20)])  # toward the target
    assert np.all(np.diff(O.phi_frames(s, p, fr)[1]) < 0)
    Phi, G = O.phi_frames_grad(s, p, fr)
    assert Phi == 0.0 and np.all(G == 0.0)
    p0 = S.Params(**{**p.__dict__, "k_ratchet": 0.0})
    Phi, G = O.phi_frames_grad(s, p0, _biased_path(s, p))
    assert Phi == 0.0 and np.all(G == 0.0)
