"""Pins of the toy-model oracle (SM, "Illustrative Application in a Toy
Model") to facts that do not come from the oracle itself: the landscape the
section describes (funnel at the origin, ring barrier, gate near (1.5, 0),
flat outer region), derivatives by finite differences, energy conservation
without friction, equipartition with friction, and worked values of the
functional (Eq. VMDcondition) with the ratchet rule (Eq. VR) and the steered
pull."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_1405_6104_gb300 import systems as S


def tp(**kw):
    return dataclasses.replace(S.Toy2dParams(), **kw)


def U(p, x, y):
    return O.toy2d_force(p, x, y)[0]


def _ridge_and_moat(p, th):
    """Along the ray at angle th: the ring's maximum and the minimum outside it."""
    r = np.linspace(0.0, 5.0, 1001)
    prof = np.array([U(p, rr * np.cos(th), rr * np.sin(th)) for rr in r])
    inner = np.where((r > 0.5) & (r < 2.5))[0]
    k = inner[np.argmax(prof[inner])]
    outer = np.arange(k, len(r))
    m = outer[np.argmin(prof[outer])]
    return r[k], prof[k], r[m], prof[m]


def test_landscape_matches_the_section():
    p = tp()
    # the product (0, 0) is the lowest point of the funnel, the global minimum in r < 6
    g = np.linspace(-6, 6, 121)
    vals = np.array([[U(p, x, y) for x in g] for y in g])
    iy, ix = np.unravel_index(np.argmin(vals), vals.shape)
    assert abs(g[ix]) <= 0.1 and abs(g[iy]) <= 0.1
    # a ring barrier surrounds the funnel: in every direction a maximum near
    # r = 1-2 separates the funnel from the region outside, several k_B T high
    ridge = {}
    for th in np.linspace(0, 2 * np.pi, 13)[:-1]:
        rk, uk, rm, um = _ridge_and_moat(p, th)
        assert 0.8 < rk < 2.0 and rm > rk
        assert uk - um > 5 * p.kT and uk > U(p, 0.0, 0.0) + 10.0
        ridge[round(th, 6)] = uk
    # the gate: the ring is lowest towards (1.5, 0), far higher opposite it
    assert min(ridge, key=ridge.get) == 0.0
    assert ridge[round(np.pi, 6)] > ridge[0.0] + 10 * p.kT
    # the start (0, 5) lies in the flat outer region
    _, fx, fy = O.toy2d_force(p, 0.0, 5.0)
    assert np.hypot(fx, fy) < 0.5
    assert abs(U(p, 0.0, 5.0) - U(p, 0.0, 4.5)) < 0.5


def test_printed_numerators_leave_no_barrier():
    # the reading behind s_power = 4: with the printed s^2 numerators the
    # profile falls monotonically from the start to the funnel in every
    # direction, so the section's activated crossing could not occur
    p = tp(s_power=2)
    r = np.linspace(0.1, 5.0, 491)  # (the gate shifts the funnel's bottom a few 1e-3 off the origin)
    for th in np.linspace(0, 2 * np.pi, 13)[:-1]:
        prof = np.array([U(p, rr * np.cos(th), rr * np.sin(th)) for rr in r])
        assert np.all(np.diff(prof) > 0.0)


def test_far_field_is_the_quartic():
    p = tp()
    for x, y in [(100.0, 0.0), (0.0, -80.0), (50.0, 60.0)]:
        r2 = x * x + y * y
        assert U(p, x, y) == pytest.approx(p.w ** 2 * r2 ** 2, rel=1e-7)


def test_force_is_minus_gradient():
    p = tp()
    rng = np.random.default_rng(3)
    h = 1e-5
    for x, y in rng.uniform(-4, 4, size=(40, 2)):
        _, fx, fy = O.toy2d_force(p, x, y)
        gx = (U(p, x + h, y) - U(p, x - h, y)) / (2 * h)
        gy = (U(p, x, y + h) - U(p, x, y - h)) / (2 * h)
        assert fx == pytest.approx(-gx, rel=1e-6, abs=1e-7)
        assert fy == pytest.approx(-gy, rel=1e-6, abs=1e-7)


def test_radial_without_the_gate():
    p = tp(A3=0.0)
    for r in (0.5, 1.7, 3.2):
        vals = [U(p, r * np.cos(t), r * np.sin(t)) for t in np.linspace(0, 2 * np.pi, 9)]
        assert np.ptp(vals) < 1e-12 * max(1.0, abs(vals[0]))
        _, fx, fy = O.toy2d_force(p, r * np.cos(0.7), r * np.sin(0.7))
        assert abs(fx * np.sin(0.7) - fy * np.cos(0.7)) < 1e-12  # no tangential component


def test_energy_conservation_without_friction():
    # gamma = 0: BAOAB is velocity Verlet; the total energy stays within O(dt^2)
    p = tp(gamma=0.0, dt=0.002, bias=S.TOY_NONE, z_product=-1.0, x0=0.3, y0=2.0)
    n = 20000
    _, _, st, path = O.toy2d_run(p, 0.0, 11, n, want_path=True)
    # energy at the end vs the start (start velocity: the seeded Maxwell-Boltzmann draw)
    v0 = np.sqrt(p.kT / p.mass) * O.normal3(11, 0, 0, 1)[:2]
    e0 = 0.5 * p.mass * (v0 ** 2).sum() + U(p, p.x0, p.y0)
    e1 = 0.5 * p.mass * (st[2] ** 2 + st[3] ** 2) + U(p, st[0], st[1])
    assert abs(e1 - e0) < 2e-3 * (abs(e0) + 1.0)
    assert len(path) == n + 1


def test_equipartition_with_friction():
    # flat landscape: <v_x^2> = <v_y^2> = kT/m under the Langevin thermostat
    p = tp(A1=0.0, A2=0.0, A3=0.0, w=0.0, bias=S.TOY_NONE, z_product=-1.0, kT=0.7, mass=2.0, gamma=2.0, dt=0.05)
    vs = []
    for seed in range(1000):  # 2000 independent samples: the mean of v^2 has a 3.2% standard error
        _, _, st, _ = O.toy2d_run(p, 0.0, 100 + seed, 200)
        vs.append(st[2:])
    vs = np.array(vs)
    assert np.mean(vs ** 2) == pytest.approx(p.kT / p.mass, rel=0.12)
    assert abs(np.mean(vs)) < 4 * np.sqrt(p.kT / p.mass / vs.size)


def test_ratchet_functional_worked_example():
    # z along the path: 2, 3, 2.5, 4, 1, 0.2 (all on the y axis); z_m: 2, 2, 2, 2, 1
    # a = 1, 0.5, 2, 0 and the product (0.2 <= 0.3) at index 5, where a = 0
    p = tp(bias=S.TOY_RATCHET)
    zs = [2.0, 3.0, 2.5, 4.0, 1.0, 0.2, 5.0]
    path = np.array([[0.0, z] for z in zs])
    k = 3.0
    Phi, passage = O.toy2d_phi_path(p, k, path)
    assert passage == 5
    assert Phi == pytest.approx(p.dt * (k / 2) ** 2 * (1.0 + 0.25 + 4.0) / (p.gamma * p.mass), rel=1e-14)


def test_steered_functional_worked_example():
    # |F| = k z for the harmonic pull towards z = 0
    p = tp(bias=S.TOY_STEERED, gamma=2.0, mass=0.5)
    zs = [3.0, 2.0, 1.5, 0.25]
    path = np.array([[z * np.cos(0.3), z * np.sin(0.3)] for z in zs])
    k = 0.7
    Phi, passage = O.toy2d_phi_path(p, k, path)
    assert passage == 3
    want = p.dt * sum((k * z) ** 2 for z in zs[1:]) / (p.gamma * p.mass)
    assert Phi == pytest.approx(want, rel=1e-12)


def test_no_bias_cases():
    p = tp(bias=S.TOY_RATCHET)
    # k = 0: the ratchet trial is the plain Langevin trial, Phi = 0
    n1, phi1, st1, _ = O.toy2d_run(p, 0.0, 21, 3000)
    n0, phi0, st0, _ = O.toy2d_run(tp(bias=S.TOY_NONE), 5.0, 21, 3000)
    assert phi1 == 0.0 and phi0 == 0.0 and n1 == n0 and np.array_equal(st1, st0)
    # a path whose z never rises has Phi = 0 under the ratchet
    path = np.array([[0.0, 5.0 - 0.01 * k] for k in range(300)])
    assert O.toy2d_phi_path(p, 4.0, path)[0] == 0.0


def test_run_bookkeeping():
    # the functional of a run equals the functional re-evaluated on its path,
    # and the ratchet never pushes outwards
    p = tp(bias=S.TOY_RATCHET)
    for seed in (1, 2, 3):
        n, phi, st, path = O.toy2d_run(p, 2.0, seed, 30000, want_path=True)
        Phi, pas = O.toy2d_phi_path(p, 2.0, path)
        assert pas == n and Phi == pytest.approx(phi, rel=1e-13, abs=0.0)
        if n > 0:
            assert np.hypot(*path[n]) <= p.z_product < np.hypot(*path[n - 1])
