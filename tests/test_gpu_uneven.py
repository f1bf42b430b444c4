"""The uneven batch: 32 solvated heteropolymers of 5 000 to 60 000 atoms
(boxes of 4 to 8.2 nm) advanced together in one handle, one trial each.
Sampled systems are checked element by element against the FP64 oracle
(forces 1e-5 relative RMS, z 1e-10 relative, neighbour lists bit-exact) and
a trial of the batch against the same system run alone (bit-identical)."""
import numpy as np
import pytest

import oracle as O
from paper_1405_6104_gb300 import binding as B
from paper_1405_6104_gb300 import systems as S

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def uneven():
    from paper_1405_6104_gb300 import build
    build.build()
    B.load()
    systems, p = S.uneven_32(2)
    return systems, p


def rel_rms(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def total_force(s, p, pos, a):
    F, e = O.forces(s, p, pos, use_list=False)
    if s.n_cv:
        _, g = O.cv(s, p, pos)
        F[: s.n_cv] += -0.5 * p.k_ratchet * a * g
    return F, e


def test_uneven_batch_sampled_parity_and_invariance(uneven):
    systems, p = uneven
    sizes = np.array([s.n_atoms for s in systems])
    order = np.argsort(sizes)
    smallest, median, largest = int(order[0]), int(order[len(order) // 2]), int(order[-1])
    seeds = [2000 + k for k in range(len(systems))]
    with B.TrialBatch(systems, p, [1] * len(systems), trial_seeds=seeds) as b:
        assert b.n_trials == len(systems)
        b.step(20)
        diag = B.sim_diagnostics(b.h)
        assert diag["max_list_entries"] < diag["list_capacity"]
        phi, best = b.bias_functional()
        assert np.all(np.isfinite(phi)) and np.all(phi >= 0.0)
        assert best == int(np.argmin(phi))
        states = {}
        for k in (smallest, median, largest):
            s = systems[k]
            pos, vel, cv = b.get_state(k)
            states[k] = (pos, vel, cv)
            e, F = b.energy_forces(k)
            Fr, er = total_force(s, p, pos, cv[2])
            assert rel_rms(F, Fr) < 1e-5, (k, s.n_atoms)
            z, _ = O.cv(s, p, pos)
            assert cv[0] == pytest.approx(z, rel=1e-10, abs=1e-10)
        for k in (smallest, median):
            s = systems[k]
            pos = B.sim_list_positions(b.h, k)  # the positions the current list was built from
            gpu = {tuple(x) for x in B.sim_pairlist(b.h, k).tolist()}
            ref = {tuple(x) for x in O.pairlist(s, pos.astype(np.float32), p.r_cut + p.skin).tolist()}
            assert gpu == ref, (k, s.n_atoms)
    # the smallest system alone, same trial seed: bit-identical trajectory
    s = systems[smallest]
    with B.TrialBatch(s, p, [1], trial_seeds=[seeds[smallest]]) as b:
        b.step(20)
        pos, vel, cv = b.get_state(0)
    assert np.array_equal(pos, states[smallest][0]) and np.array_equal(vel, states[smallest][1])
    assert cv[3] == states[smallest][2][3]


def test_per_class_launches_are_bit_identical(uneven):
    """The size classes of the uneven batch: one pair launch per class, each
    with its own variant (the autotuner's per-class picks, and a fixed mix),
    gives the same trajectories, bit for bit, as one launch over the whole
    batch with variant 0."""
    systems, p = uneven
    sub = [systems[k] for k in np.argsort([s.n_atoms for s in systems])[::6]]  # six systems across the sizes
    seeds = [3000 + k for k in range(len(sub))]
    results = []
    for mode in ("single", "tuned", "mix"):
        with B.TrialBatch(sub, p, [1] * len(sub), trial_seeds=seeds) as b:
            classes = B.sim_tune_classes(b.h)
            assert len(classes) >= 3 and sum(c["trials"] for c in classes) == len(sub)
            if mode == "tuned":
                B.sim_autotune(b.h, 1, None)
            elif mode == "mix":
                B.sim_set_class_variants(b.h, [(0, 8, 3, 6, 1)[k % 5] for k in range(len(classes))])
                assert all(c["own_launch"] for c in B.sim_tune_classes(b.h))
            b.step(15)
            results.append([b.get_state(k) for k in range(len(sub))])
    for other in results[1:]:
        for x, y in zip(results[0], other):
            assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1]) and x[2][3] == y[2][3]
