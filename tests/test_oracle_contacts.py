"""Pins of the contact-order oracle (Sec. "Results": matrix M of the order
of native-contact formation and path similarity s(k, k')) to the contact
function C(r) (pinned separately), to worked formation sequences, and to
closed-form values of s."""
import numpy as np
import pytest

import oracle as O


def r_half(r0=0.75):
    """C(r) = 1/2 by bisection on the oracle's contact function."""
    lo, hi = 0.5 * r0, 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if O.contact(mid, r0)[0] > 0.5:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def two_atom_frames(dists):
    return np.array([[[0.1, 0.2, 0.3], [0.1 + d, 0.2, 0.3]] for d in dists])


def test_formed_means_contact_value_above_one_half():
    r0 = 0.75
    rh = r_half(r0)
    assert 0.80 < rh < 0.83
    pairs = np.array([[0, 1]], np.int32)
    for d, want in [(rh * (1 - 1e-9), 0), (rh * (1 + 1e-9), -1), (0.3, 0), (r0, 0), (1.5, -1)]:
        t = O.contact_times(two_atom_frames([d]), [0], 10.0, r0, pairs)
        assert t[0] == want, d


def test_native_contacts_by_brute_force():
    rng = np.random.default_rng(4)
    nat = rng.uniform(0, 1.6, size=(60, 3))
    got = O.native_contacts(nat, 60, 0.75, 3)
    want = [(i, j) for i in range(60) for j in range(i + 4, 60)
            if O.contact(np.linalg.norm(nat[j] - nat[i]), 0.75)[0] > 0.5]
    assert [tuple(x) for x in got.tolist()] == want


def test_formation_time_worked_sequence():
    # four contacts between atom 0 and atoms 1..4 over six frames (steps 0, 10, ..., 50):
    # c0 forms at frame 2, breaks at 4, re-forms at 5 -> 50; c1 formed throughout -> 0;
    # c2 never -> -1; c3 formed until frame 4, broken at the last frame -> -1
    near, far = 0.5, 1.2
    seq = {1: [far, far, near, near, far, near], 2: [near] * 6, 3: [far] * 6, 4: [near] * 5 + [far]}
    # atom 0 at the origin, partner a on its own direction (partners stay far from each other)
    dirs = {1: (1, 0, 0), 2: (0, 1, 0), 3: (0, 0, 1), 4: (-1, 0, 0)}
    frames = np.zeros((6, 5, 3))
    for f in range(6):
        for a, ds in seq.items():
            frames[f, a] = ds[f] * np.array(dirs[a], float)
    pairs = np.array([[0, 1], [0, 2], [0, 3], [0, 4]], np.int32)
    t = O.contact_times(frames, np.arange(0, 60, 10), 20.0, 0.75, pairs)
    assert t.tolist() == [50, 0, -1, -1]


def test_minimum_image_decides_contacts():
    pairs = np.array([[0, 1]], np.int32)
    fr = np.array([[[0.1, 1.0, 1.0], [2.9, 1.0, 1.0]]])  # 0.2 apart through the face of a 3.0 box
    assert O.contact_times(fr, [7], 3.0, 0.75, pairs)[0] == 7


def test_similarity_closed_forms():
    rng = np.random.default_rng(1)
    t = rng.permutation(200).astype(np.int64)
    assert O.path_similarity(t, t) == 1.0
    assert O.path_similarity(t, 1000 - t) == 0.0  # every pair in the opposite order
    u = rng.permutation(200).astype(np.int64)
    assert O.path_similarity(t, u) == O.path_similarity(u, t)
    allnot = -np.ones(50, np.int64)
    assert O.path_similarity(allnot, allnot) == 1.0  # all ties: M = 1/2 everywhere
    # independent orders without ties agree on half the ordered pairs
    vals = [O.path_similarity(rng.permutation(120), rng.permutation(120)) for _ in range(40)]
    assert np.mean(vals) == pytest.approx(0.5, abs=0.02)
    # three equally likely order relations (formation in three tied stages):
    # agreement 3 x (1/3)^2 = 1/3 -- the random reference the paper's SM
    # reports "sharply peaked around 0.3"
    vals = [O.path_similarity(rng.integers(0, 3, 150), rng.integers(0, 3, 150)) for _ in range(40)]
    assert np.mean(vals) == pytest.approx(1.0 / 3.0, abs=0.02)


def test_one_swap_changes_two_ordered_pairs():
    t = np.arange(10, dtype=np.int64)
    u = t.copy()
    u[[3, 4]] = u[[4, 3]]
    assert O.path_similarity(t, u) == pytest.approx(1.0 - 2.0 / 90.0, rel=1e-15)
