"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the
same seeded inputs.  Tolerances: forces 1e-5 relative RMS, positions after
100 steps 1e-4 nm, bias functional 1e-6 relative, neighbour lists
bit-exact, Philox raw outputs bit-exact."""
import numpy as np
import pytest

import oracle as O
from paper_1405_6104_gb300 import binding as B
from paper_1405_6104_gb300 import systems as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1405_6104_gb300 import build
    build.build()
    B.load()


def min_image(d, L):
    return d - L * np.round(d / L)


def rel_rms(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


SYSTEMS = {
    "tiny": lambda: S.tiny_chain(0),
    "small": lambda: S.small_solvated(),
    "ragged": lambda: S.small_solvated(n_solute=37, n_water=420, seed=8, cv_min_sep=3),
}


def oracle_total_force(s, p, pos, a):
    """-grad U + F^bias with the ratchet amplitude a (Eq. VR)."""
    F, e = O.forces(s, p, pos, use_list=False)
    if s.n_cv:
        _, g = O.cv(s, p, pos)
        F[: s.n_cv] += -0.5 * p.k_ratchet * a * g
    return F, e


# ---------------------------------------------------------------------------

def test_philox_raw_bitexact_and_normals():
    n = 2000
    for seed, step, stream in [(0, 1, 0), (123456789012345, 77, 0), (1000, 0, 1), (2 ** 40 + 3, 2 ** 33 + 5, 0)]:
        raw, nor = B.sim_philox_normals(seed, step, stream, n)
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for o in range(0, n, 97):
            ctr = [o, step & 0xFFFFFFFF, step >> 32, stream]
            assert np.array_equal(raw[o], O.philox4x32_10(ctr, key))
            assert np.abs(nor[o] - O.normal3(seed, o, step, stream)).max() < 2e-6


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_pairlist_bitexact(name):
    s, p = SYSTEMS[name]()
    with B.TrialBatch(s, p, [1]) as b:
        for n_steps in (0, 30, 7):
            b.step(n_steps)
            pos = B.sim_list_positions(b.h, 0)  # the positions the current list was built from
            gpu = {tuple(x) for x in B.sim_pairlist(b.h, 0).tolist()}
            ref = {tuple(x) for x in O.pairlist(s, pos.astype(np.float32), p.r_cut + p.skin).tolist()}
            assert len(gpu) == len(B.sim_pairlist(b.h, 0))  # no duplicates
            assert gpu == ref
            # every listed pair sits in one entry (a j-atom against the 8
            # atoms of its i-cluster), and no entry is empty
            n_ent = B.sim_diagnostics(b.h)["list_entries"]
            assert 0 < n_ent <= len(gpu) <= 8 * n_ent


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_forces_and_energies_parity(name):
    s, p = SYSTEMS[name]()
    with B.TrialBatch(s, p, [1]) as b:
        for n_steps in (0, 30, 5):
            b.step(n_steps)
            pos, vel, cv = b.get_state(0)
            e, F = b.energy_forces(0)
            Fr, er = oracle_total_force(s, p, pos, cv[2])
            assert rel_rms(F, Fr) < 1e-5
            scale = np.abs(er).sum() + 1.0
            assert np.abs(e[:4] - er).max() < 1e-5 * scale
            ekin = 0.5 * (s.mass[:, None] * vel ** 2).sum()
            assert e[4] == pytest.approx(ekin, rel=1e-6)
            assert e[5] == pytest.approx(0.25 * p.k_ratchet * cv[2] ** 2, rel=1e-12, abs=1e-300)
            z, _ = O.cv(s, p, pos)
            assert cv[0] == pytest.approx(z, rel=1e-10, abs=1e-10)


@pytest.mark.parametrize("name", ["tiny", "small"])
def test_bonded_forces_alone(name):
    """Bonds and angles only (no charges, no Lennard-Jones, no bias): the
    grouped bonded kernel against the oracle atom by atom on thermalised
    molecules (at the generated start every bond and angle sits at its rest
    value and the forces are rounding noise), and exact action-reaction (the
    fixed-point forces of every group sum to zero)."""
    s, p = SYSTEMS[name]()
    s = s.copy()
    s.charge = np.zeros_like(s.charge)
    s.epsilon = np.zeros_like(s.epsilon)
    p = S.Params(**{**p.__dict__, "k_ratchet": 0.0})
    with B.TrialBatch(s, p, [2], trial_seeds=[3, 4]) as b:
        for n_steps in (20, 20):
            b.step(n_steps)
            for t in range(2):
                pos, _, _ = b.get_state(t)
                _, F = b.energy_forces(t)
                Fr, _ = O.forces(s, p, pos, use_list=False)
                assert rel_rms(F, Fr) < 1e-5
                assert np.abs(F - Fr).max() < 1e-4 * np.abs(Fr).max()
                assert np.abs(F.sum(axis=0)).max() == 0.0


def test_many_lj_types_take_the_general_kernel():
    """More distinct Lennard-Jones types than the packed kernels' tables hold
    (16): the general pair kernel runs, with the same parity to the oracle,
    and graph replay and direct launches stay bit-identical; the one-kernel
    step (whose tables hold 16 types) is refused, and the step-form
    autotuner leaves it out."""
    s, p = S.small_solvated()
    s = s.copy()
    k = np.arange(s.n_solute) % 30
    n0 = len(s.sigma)
    s.sigma = np.concatenate([s.sigma, 0.30 + 0.002 * np.arange(30)])
    s.epsilon = np.concatenate([s.epsilon, 0.40 + 0.01 * np.arange(30)])
    s.lj_type = s.lj_type.copy()
    s.lj_type[: s.n_solute] = n0 + k
    results = []
    for flags in (0, B.SIM_NO_GRAPH):
        q = S.Params(**{**p.__dict__, "flags": flags})
        with B.TrialBatch(s, q, [2], trial_seeds=[21, 22]) as b:
            b.step(20)
            pos, vel, cv = b.get_state(1)
            e, F = b.energy_forces(1)
            Fr, er = oracle_total_force(s, q, pos, cv[2])
            assert rel_rms(F, Fr) < 1e-5
            results.append([b.get_state(t) for t in range(2)])
            with pytest.raises(B.SimError) as err:
                B.sim_set_step_mode(b.h, 1)
            assert err.value.code == B.SIM_EINVAL
    for x, y in zip(*results):
        assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])
    with B.TrialBatch(s, p, [2], trial_seeds=[21, 22]) as b:
        mode, ms = B.sim_autotune_step(b.h, 1, times=True)
        assert mode in (0, 2) and ms[1] < 0 and ms[0] > 0 and ms[2] > 0


@pytest.mark.parametrize("name", ["tiny", "small"])
def test_trajectory_parity_100_steps(name):
    s, p = SYSTEMS[name]()
    seed = 4242
    with B.TrialBatch(s, p, [1], trial_seeds=[seed]) as b:
        b.step(100)
        pos, vel, cv = b.get_state(0)
    r = O.run(s, p, seed, 100)
    assert r["status"] == 0
    d = min_image(pos - r["pos"], s.box)
    assert np.abs(d).max() < 1e-4
    assert np.abs(vel - r["vel"]).max() < 1e-2 * np.abs(r["vel"]).max()


@pytest.mark.parametrize("name", ["tiny", "small", "ragged"])
def test_functional_parity_on_shared_states(name):
    """The GPU's own frames are fed to the oracle: per-step z, a and the
    accumulated Phi must agree (Phi to 1e-6 relative)."""
    s, p = SYSTEMS[name]()
    n = 100
    with B.TrialBatch(s, p, [1], trial_seeds=[17]) as b:
        B.sim_record(b.h, n + 1)
        frames = [b.get_state(0)[0]]
        for _ in range(n):
            b.step(1)
            frames.append(b.get_state(0)[0])
        _, _, cv = b.get_state(0)
        rec = B.sim_get_record(b.h, 0, n + 1)
    Phi, z, a, phi = O.phi_frames(s, p, np.stack(frames))
    assert Phi > 0
    assert cv[3] == pytest.approx(Phi, rel=1e-6)
    assert np.allclose(rec[1:, 0], z[1:], rtol=1e-11, atol=1e-11)
    assert np.allclose(rec[1:, 2], a[1:], rtol=1e-6, atol=1e-9 * max(1.0, z.max()))
    assert np.allclose(rec[1:, 3], phi[1:], rtol=1e-5, atol=1e-12 * max(1.0, phi.max()))
    biased = rec[1:, 2] > 0
    assert np.allclose(rec[1:, 3][biased], (0.5 * p.k_ratchet) ** 2 * rec[1:, 2][biased] ** 2 * rec[1:, 4][biased],
                       rtol=1e-12)


def test_batch_invariance_and_determinism():
    s1, p = S.tiny_chain(0)
    s2, _ = S.small_solvated()
    seeds = [5, 6, 7, 8]
    with B.TrialBatch([s1, s2], p, [3, 1], trial_seeds=seeds) as b:
        b.step(47)
        batch = [b.get_state(t) for t in range(4)]
    with B.TrialBatch(s1, p, [1], trial_seeds=[6]) as b:
        b.step(47)
        alone = b.get_state(0)
    assert np.array_equal(batch[1][0], alone[0]) and np.array_equal(batch[1][1], alone[1])
    assert batch[1][2][3] == alone[2][3]
    with B.TrialBatch(s2, p, [1], trial_seeds=[8]) as b:
        b.step(47)
        alone2 = b.get_state(0)
    assert np.array_equal(batch[3][0], alone2[0]) and batch[3][2][3] == alone2[2][3]
    # graphs vs direct launches, and run-to-run: bit-identical
    p_ng = S.Params(**{**p.__dict__, "flags": B.SIM_NO_GRAPH})
    with B.TrialBatch([s1, s2], p_ng, [3, 1], trial_seeds=seeds) as b:
        b.step(47)
        again = [b.get_state(t) for t in range(4)]
    for x, y in zip(batch, again):
        assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1]) and x[2][3] == y[2][3]
    # splitting a run into calls only changes the rounding of the merged half kicks
    with B.TrialBatch([s1, s2], p, [3, 1], trial_seeds=seeds) as b:
        b.step(20)
        b.step(27)
        split = [b.get_state(t) for t in range(4)]
    for x, y in zip(batch, split):
        assert np.abs(min_image(x[0] - y[0], 3.0)).max() < 1e-4


def test_energy_conservation_without_friction():
    s, p = S.tiny_chain(0)
    p.gamma, p.k_ratchet = 0.0, 0.0
    es = []
    with B.TrialBatch(s, p, [1], trial_seeds=[3]) as b:
        for _ in range(21):
            e, _ = b.energy_forces(0, want_forces=False)
            es.append(e[:5])
            b.step(50)
    es = np.array(es)
    etot, ekin = es.sum(1), es[:, 4]
    assert np.std(etot) < 0.02 * np.std(ekin)
    assert abs(etot[-1] - etot[0]) / (1000 * p.dt) / s.n_atoms < 1e-3


def test_selection_and_no_cv_system():
    s, p = S.tiny_chain(0)
    with B.TrialBatch(s, p, [6], trial_seeds=list(range(100, 106))) as b:
        b.step(60)
        phi, am = b.bias_functional()
        assert am == int(np.argmin(phi)) and np.all(phi >= 0) and phi.max() > 0
        zs = np.array([b.get_state(t)[2][0] for t in range(6)])
        zmax = float(np.median(zs))
        _, am2 = b.bias_functional(zmax)
        ok = np.where(zs <= zmax)[0]
        assert am2 == int(ok[np.argmin(phi[ok])])
        _, am3 = b.bias_functional(0.0)  # no trial has reached z = 0
        assert am3 == -1
    s0 = s.copy()
    s0.n_cv = 0
    s0.native_pos = np.zeros((0, 3))
    with B.TrialBatch(s0, p, [2]) as b:
        b.step(25)
        phi, _ = b.bias_functional()
        assert np.all(phi == 0.0) and b.get_state(0)[2][0] == 0.0


def test_recorded_functional_bookkeeping_and_restart():
    s, p = S.small_solvated()
    with B.TrialBatch(s, p, [2], trial_seeds=[1, 2]) as b:
        B.sim_record(b.h, 64)
        b.step(40)
        rec = B.sim_get_record(b.h, 1, 64)[1:41]
        pos, vel, cv = b.get_state(1)
        assert cv[3] == pytest.approx(p.dt * rec[:, 3].sum(), rel=1e-12)
        z, zm, a = rec[:, 0], rec[:, 1], rec[:, 2]
        assert np.all(np.diff(zm) <= 0) and np.all(zm <= z + 1e-15)
        # restart trial 1 from its own state with the functional carried over
        b.set_state(1, pos, vel, cv_state=[cv[1], cv[3]])
        _, _, cv2 = b.get_state(1)
        assert cv2[3] == cv[3] and cv2[1] == pytest.approx(cv[1], rel=1e-12)
        assert cv2[0] == pytest.approx(cv[0], rel=1e-12)


def _pick_variant(b, variant):
    """Fixes the pair-kernel launch shape: a variant number, or "tuned" for
    whatever the autotuner picks on this batch (as the benchmark does)."""
    if variant == "tuned":
        return B.sim_autotune(b.h, 3, None)[0]
    B.sim_set_variants(b.h, variant, 0)
    return variant


# 0: the general kernel; 8: the persistent packed kernel (FP32x2 arithmetic,
# i-clusters handed out by a counter over a resident grid), the one the
# benchmark's autotuner picks for the 64-trial batch
@pytest.mark.slow
@pytest.mark.parametrize("variant", [0, 8, "tuned"])
def test_full_size_batch_sampled(variant):
    """64 trials of the 11 040-atom system in one batch (the benchmarked
    configuration and launch shape): sampled trials checked element by
    element after a chunk of graph-replayed steps."""
    s, p, seeds = S.batched_64(1)
    with B.TrialBatch(s, p, [64], trial_seeds=seeds) as b:
        _pick_variant(b, variant)
        b.step(10)
        diag = B.sim_diagnostics(b.h)
        assert diag["max_list_entries"] < diag["list_capacity"]
        for t in (0, 37, 63):
            pos, vel, cv = b.get_state(t)
            e, F = b.energy_forces(t)
            Fr, er = oracle_total_force(s, p, pos, cv[2])
            assert rel_rms(F, Fr) < 1e-5
            z, _ = O.cv(s, p, pos)
            assert cv[0] == pytest.approx(z, rel=1e-11)
        pos = B.sim_list_positions(b.h, 63)
        gpu = {tuple(x) for x in B.sim_pairlist(b.h, 63).tolist()}
        ref = {tuple(x) for x in O.pairlist(s, pos.astype(np.float32), p.r_cut + p.skin).tolist()}
        assert gpu == ref


def test_potential_autograd_backward_is_minus_force():
    """U(X, Y) as a torch.autograd.Function: forward = FP64 energy total of the
    kernels, backward = -F; checked against the FP64 oracle's -grad U."""
    import torch
    from paper_1405_6104_gb300.autograd import Evaluator, potential_energy
    s, p = S.small_solvated()
    ev = Evaluator(s, p)
    try:
        x = torch.tensor(s.pos, dtype=torch.float64, requires_grad=True)
        U = potential_energy(x, ev)
        L = 3.0 * U + 0.5 * (x ** 2).sum()
        L.backward()
        Fr, er = O.forces(s, p, s.pos)
        assert float(U.detach()) == pytest.approx(er.sum(), rel=1e-5, abs=1e-5 * np.abs(er).sum())
        g = x.grad.numpy()
        assert rel_rms(g, -3.0 * Fr + s.pos) < 1e-5
        assert rel_rms((g - s.pos) / 3.0, -Fr) < 1e-5
        # a second evaluation at displaced positions reuses the handle
        y = torch.tensor(s.pos + 0.001, dtype=torch.float64, requires_grad=True)
        potential_energy(y, ev).backward()
        Fr2, _ = O.forces(s, p, (s.pos + 0.001).astype(np.float32).astype(np.float64))
        assert rel_rms(y.grad.numpy(), -Fr2) < 1e-5
    finally:
        ev.close()


def test_potential_autograd_on_device_tensors():
    """U(X, Y) on CUDA tensors: a batch of three configurations evaluated in
    one call through device pointers (no host round trip); energies and
    gradients against the FP64 oracle for each configuration; a second
    evaluation within the list buffer reuses the lists."""
    import torch
    from paper_1405_6104_gb300.autograd import Evaluator, potential_energy
    s, p = S.small_solvated()
    rng = np.random.default_rng(4)
    confs = np.stack([s.pos + 0.01 * rng.normal(size=s.pos.shape) for _ in range(3)])
    confs = confs.astype(np.float32).astype(np.float64)
    ev = Evaluator(s, p, n_conf=3)
    try:
        dev = torch.device("cuda", 0)
        x = torch.tensor(confs, device=dev, requires_grad=True)
        U = potential_energy(x, ev)
        assert U.shape == (3,) and U.is_cuda
        w = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64, device=dev)
        (w * U).sum().backward()
        g = x.grad.cpu().numpy()
        for k in range(3):
            Fr, er = O.forces(s, p, confs[k])
            assert float(U[k]) == pytest.approx(er.sum(), rel=1e-5, abs=1e-5 * np.abs(er).sum())
            assert rel_rms(g[k], -float(w[k]) * Fr) < 1e-5
        rb0 = B.sim_diagnostics(ev.batch.h)["trial_rebuilds"]
        y = torch.tensor((confs + 1e-3).astype(np.float32).astype(np.float64), device=dev, requires_grad=True)
        potential_energy(y, ev).sum().backward()
        torch.cuda.synchronize()
        assert B.sim_diagnostics(ev.batch.h)["trial_rebuilds"] == rb0  # within the buffer: lists kept
        Fr, _ = O.forces(s, p, (confs[1] + 1e-3).astype(np.float32).astype(np.float64))
        assert rel_rms(y.grad.cpu().numpy()[1], -Fr) < 1e-5
        # a configuration far from the lists' positions: rebuilt, still exact
        z = torch.tensor(np.roll(confs, 1, axis=0), device=dev, requires_grad=True)
        potential_energy(z, ev).sum().backward()
        Fr, _ = O.forces(s, p, confs[0])
        assert rel_rms(z.grad.cpu().numpy()[1], -Fr) < 1e-5
    finally:
        ev.close()


def test_autotuner_variants_are_bit_identical(tmp_path):
    """Every launch shape the autotuner can pick computes the same result."""
    s, p = S.small_solvated()
    results = []
    for pv in range(9):  # every pair-kernel variant
        for cv in (0, 2):
            cache = tmp_path / f"tune_{pv}_{cv}.txt"
            with B.TrialBatch(s, p, [2], trial_seeds=[4, 5]) as b:
                key_probe = tmp_path / "probe.txt"
                B.sim_autotune(b.h, 1, str(key_probe))  # learn the size-class key
                key = key_probe.read_text().split()[0]
                cache.write_text(f"{key} {pv} {cv}\n")
                assert B.sim_autotune(b.h, 1, str(cache)) == (pv, cv)
                b.step(30)
                results.append([b.get_state(t) for t in range(2)])
    for r in results[1:]:
        for x, y in zip(results[0], r):
            assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1]) and x[2][3] == y[2][3]


def test_in_graph_pair_timing():
    """Event-record nodes around the pair kernel inside the chunk graph time
    every replayed launch and leave the trajectory bit-identical."""
    s, p = S.small_solvated()
    results = []
    for mode in (0, 2):
        with B.TrialBatch(s, p, [2], trial_seeds=[4, 5]) as b:
            B.sim_set_timing(b.h, mode)
            b.step(3 * p.nstlist)  # three chunk replays in one call
            b.step(3)  # direct steps
            b.step(p.nstlist - 3 + p.nstlist)  # one replay, then direct steps
            kt = B.sim_kernel_times(b.h)
            if mode == 2:
                ms, n = kt["pair_in_graph"]
                assert n == 4 * p.nstlist and ms > 0.0
            else:
                assert "pair_in_graph" not in kt
            results.append([b.get_state(t) for t in range(2)])
    for x, y in zip(*results):
        assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])


def test_set_state_rejects_non_finite_input_and_keeps_the_state():
    s, p = S.small_solvated()
    with B.TrialBatch(s, p, [2], trial_seeds=[4, 5]) as b:
        b.step(10)
        before = [b.get_state(t) for t in range(2)]
        pos, vel, _ = b.get_state(1)
        pos = pos.copy()
        pos[7, 1] = np.nan
        with pytest.raises(B.SimError) as e:
            b.set_state(1, pos, vel)
        assert e.value.code == B.SIM_EINVAL and "non-finite" in str(e.value)
        after = [b.get_state(t) for t in range(2)]
        for x, y in zip(before, after):
            assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])
        b.step(10)  # and the handle stays usable


def test_strict_skin_violation_is_reported():
    """Fixed-interval lists with SIM_STRICT_SKIN: an atom moving more than
    skin/2 between list rebuilds ends the call with SIM_ESKIN (a 0.002 nm
    skin is crossed within a list interval)."""
    s, p = S.small_solvated()
    p.skin = 0.002
    p.flags = B.SIM_STRICT_SKIN | B.SIM_FIXED_INTERVAL
    with B.TrialBatch(s, p, [1], trial_seeds=[9]) as b:
        with pytest.raises(B.SimError) as e:
            for _ in range(5):
                b.step(10)
        assert e.value.code == B.SIM_ESKIN


def test_list_overflow_is_reported(monkeypatch):
    """A cluster list capacity forced below what the system needs: the list
    build's own bounds checks drop the excess entries, flag the overflow, and
    sim_create returns SIM_ELIST_OVERFLOW (nothing is written out of bounds)."""
    s, p = S.small_solvated()
    monkeypatch.setenv("VPATH_LIST_CAP", "16")
    with pytest.raises(B.SimError) as e:
        B.TrialBatch(s, p, [1])
    assert e.value.code == B.SIM_ELIST_OVERFLOW
    monkeypatch.delenv("VPATH_LIST_CAP")
    with B.TrialBatch(s, p, [1]) as b:  # the default capacity holds it
        b.step(10)


def test_blow_up_is_reported_as_non_finite():
    """A time step far beyond the stable one makes the run blow up; the
    update kernel flags forces beyond the fixed-point range and atoms that
    cross the box in one step (lists are rebuilt and positions wrapped every
    step in such a run, so it would otherwise stay finite) and the call
    returns SIM_ENONFINITE."""
    s, p = S.small_solvated()
    p.dt = 0.05
    with B.TrialBatch(s, p, [1], trial_seeds=[9]) as b:
        with pytest.raises(B.SimError) as e:
            for _ in range(50):
                b.step(10)
        assert e.value.code == B.SIM_ENONFINITE


@pytest.mark.slow
@pytest.mark.parametrize("variant", [8, "tuned"])
def test_benchmarked_system_functional_parity(variant):
    """The 11 040-atom system (540-atom reaction coordinate, 127 260 contact
    pairs, k_R of the paper): 100 graph-replayed steps with the per-step
    record and the frame recorder on; the GPU's frames are fed to the oracle,
    which must reproduce z at every step and the accumulated Phi to 1e-6
    relative (Eq. VMDcondition; a = z - z_m is a small difference of large
    sums here)."""
    s, p = S.plain_single(1)
    n = 100
    with B.TrialBatch(s, p, [1], trial_seeds=[1000]) as b:
        _pick_variant(b, variant)
        x0, _, cv0 = b.get_state(0)
        B.sim_record(b.h, n + 1)
        B.sim_record_frames(b.h, 0, n + 1)
        b.step(n)
        _, _, cv = b.get_state(0)
        rec = B.sim_get_record(b.h, 0, n + 1)
        fr = B.sim_get_frames(b.h, n + 1, s.n_cv)
    fr[0] = x0[: s.n_cv]
    Phi, z, a, phi = O.phi_frames(s, p, fr)
    assert Phi > 0 and np.count_nonzero(a[1:]) > 10
    assert cv[3] - cv0[3] == pytest.approx(Phi, rel=1e-6)
    assert np.allclose(rec[1:, 0], z[1:], rtol=1e-10, atol=0.0)
    assert np.allclose(rec[1:, 2], a[1:], rtol=1e-6, atol=1e-9 * max(1.0, z.max()))
    assert np.allclose(rec[1:, 3], phi[1:], rtol=1e-5, atol=1e-12 * max(1.0, phi.max()))


@pytest.mark.slow
@pytest.mark.parametrize("variant", [8])
def test_benchmarked_system_trajectory_100_steps(variant):
    """The 11 040-atom system, 100 steps in ten graph replays on the
    benchmarked pair kernel, against the FP64 oracle's own 100-step run with
    the shared Philox noise: positions to 1e-4 nm.  Both start from the
    relaxed state the benchmark times (the generated start, with its random
    water orientations, is too hot for a 100-step comparison: a few
    overlapping atoms amplify rounding differences)."""
    s, p = relaxed_plain_single()
    seed = 1000
    with B.TrialBatch(s, p, [1], trial_seeds=[seed]) as b:
        _pick_variant(b, variant)
        b.step(100)
        pos, vel, cv = b.get_state(0)
    r = O.run(s, p, seed, 100, pos=s.pos, vel=s.vel)
    assert r["status"] == 0
    d = min_image(pos - r["pos"], s.box)
    assert np.abs(d).max() < 1e-4
    assert np.abs(vel - r["vel"]).max() < 1e-2 * np.abs(r["vel"]).max()


_RELAXED = {}


def relaxed_plain_single(steps: int = 2000):
    """The 11 040-atom system after `steps` steps of strong friction without
    bias on the GPU (as the benchmark prepares it), with the FP32 positions
    and velocities of that state as the start."""
    if steps not in _RELAXED:
        s, p = S.plain_single(1)
        pe = S.Params(**{**p.__dict__, "gamma": 20.0, "k_ratchet": 0.0})
        with B.TrialBatch(s, pe, [1], trial_seeds=[7]) as b:
            b.step(steps)
            pos, vel, _ = b.get_state(0)
        s = s.copy()
        s.pos, s.vel = pos, vel
        _RELAXED[steps] = (s, p)
    s, p = _RELAXED[steps]
    return s.copy(), S.Params(**p.__dict__)


@pytest.mark.slow
@pytest.mark.parametrize("start", ["generated", "relaxed"])
def test_no_pair_within_the_cut_off_is_missing(start):
    """The cut-off model of U (Eq. Lang) at every step: on the GPU's own
    frames of the 11 040-atom system, every non-excluded pair whose FP32
    distance is below r_cut (the oracle's brute-force list rule with
    r_list = r_cut) is in the list the forces of that step were computed
    with, over 25 single steps.  The generated start is hot enough that
    displacements trigger rebuilds before the 10-step interval is up; with
    fixed 10-step intervals the same run moves atoms farther than skin/2."""
    s, p = S.plain_single(1) if start == "generated" else relaxed_plain_single()
    with B.TrialBatch(s, p, [1], trial_seeds=[1000]) as b:
        B.sim_set_variants(b.h, 8, 0)
        for _ in range(25):
            b.step(1)
            pos, _, _ = b.get_state(0)
            listed = {tuple(x) for x in B.sim_pairlist(b.h, 0).tolist()}
            within = O.pairlist(s, pos.astype(np.float32), p.r_cut)
            missing = [tuple(x) for x in within.tolist() if tuple(x) not in listed]
            assert not missing, f"{len(missing)} pairs inside r_cut are not listed, e.g. {missing[:3]}"
        diag = B.sim_diagnostics(b.h)
        assert diag["skin_violations"] == 0
        assert diag["trial_rebuilds"] >= 3
        if start == "generated":
            assert diag["displacement_rebuilds"] >= 1
    q = S.Params(**{**p.__dict__, "flags": B.SIM_FIXED_INTERVAL})
    with B.TrialBatch(s, q, [1], trial_seeds=[1000]) as b:
        b.step(20)
        if start == "generated":
            assert B.sim_diagnostics(b.h)["skin_violations"] > 0
