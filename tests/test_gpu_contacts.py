"""Order of native-contact formation and path similarity (Sec. "Results")
on the GPU against the FP64 oracle: native contact lists and formation
times bit-exact (integers decided in FP64 on the same FP32 positions, the
GPU's own recorded frames), similarities exact (integer counts over the
same denominator)."""
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


@pytest.mark.parametrize("every", [1, 3])
def test_formation_times_match_the_oracle_on_gpu_frames(every):
    s, p = S.small_solvated()
    p.k_ratchet = 50.0  # a strong pull so that contacts form and break within the run
    n = 60
    with B.TrialBatch(s, p, [2], trial_seeds=[31, 32]) as b:
        pairs = B.sim_native_contacts(b.h, 0)
        ref = O.native_contacts(s.native_pos, s.n_cv, p.cv_r0, p.cv_min_sep)
        assert np.array_equal(pairs, ref) and len(pairs) > 100
        with pytest.raises(B.SimError):
            B.sim_contact_times(b.h, 0, len(pairs))
        B.sim_contact_tracking(b.h, every)
        B.sim_record_frames(b.h, 0, n + 1)
        b.step(n)
        t_gpu = B.sim_contact_times(b.h, 0, len(pairs))
        fr = B.sim_get_frames(b.h, n + 1, s.n_cv)
        B.sim_record_frames(b.h, 0, 0)
        steps = np.array([k for k in range(1, n + 1) if k % every == 0])
        t_ref = O.contact_times(fr[steps], steps, s.box, p.cv_r0, pairs)
        assert np.array_equal(t_gpu, t_ref)
        assert (t_gpu >= 0).any() and (t_gpu < 0).any()
        # restarting the tracker resets every time
        B.sim_contact_tracking(b.h, 0)
        b.step(5)
        assert np.array_equal(B.sim_contact_times(b.h, 0, len(pairs)), -np.ones(len(pairs), np.int64))


def test_similarity_matches_the_oracle():
    rng = np.random.default_rng(7)
    n_c = 700
    T = np.stack([rng.integers(-1, 40, n_c) for _ in range(6)]).astype(np.int64)
    T[5] = T[0]
    T[4] = np.where(T[0] >= 0, 1000 - T[0], -1)
    pairs = [(a, b) for a in range(6) for b in range(6)]
    s_gpu = B.path_similarity(T, pairs)
    for (a, b), v in zip(pairs, s_gpu):
        assert v == O.path_similarity(T[a], T[b]), (a, b)
    assert s_gpu[pairs.index((0, 5))] == 1.0
    assert np.array_equal(B.path_similarity(T[:, :1], [(0, 1)]), [1.0])  # one contact: no ordered pair


def test_similarity_both_counting_paths_match_the_oracle():
    """Path pairs with few distinct times (joint-histogram count) and with
    many (all ordered contact pairs), in one call, exact against the oracle;
    times of any size (only their order in a path matters), ties, and
    negative values of any kind as 'not formed'."""
    rng = np.random.default_rng(11)
    n_c = 900
    few = [rng.integers(-1, 30, n_c) for _ in range(3)]                      # <= 31 distinct each
    many = [rng.permutation(n_c) * 7919 + (1 << 40) for _ in range(2)]      # all distinct, beyond 2^31
    many.append(np.where(rng.random(n_c) < 0.2, -5, rng.integers(0, 10 ** 12, n_c)))
    T = np.stack(few + many).astype(np.int64)
    pairs = [(a, b) for a in range(len(T)) for b in range(len(T)) if a != b]
    s_gpu = B.path_similarity(T, pairs)
    for (a, b), v in zip(pairs, s_gpu):
        assert v == O.path_similarity(np.where(T[a] < 0, -1, T[a]), np.where(T[b] < 0, -1, T[b])), (a, b)


def test_similarity_of_trials_at_full_size():
    """The 11 040-atom system (23 160 native contacts): formation times of a
    few trials and their pairwise similarities, GPU against the oracle."""
    s, p = S.plain_single(1)
    with B.TrialBatch(s, p, [3], trial_seeds=[41, 42, 43]) as b:
        B.sim_contact_tracking(b.h, 5)
        b.step(50)
        pairs = B.sim_native_contacts(b.h, 0)
        assert len(pairs) == len(O.native_contacts(s.native_pos, s.n_cv, p.cv_r0, p.cv_min_sep))
        T = np.stack([B.sim_contact_times(b.h, t, len(pairs)) for t in range(3)])
    s_gpu = B.path_similarity(T, [(0, 1), (0, 2), (1, 2)])
    for (a, c), v in zip([(0, 1), (0, 2), (1, 2)], s_gpu):
        assert v == O.path_similarity(T[a], T[c])
