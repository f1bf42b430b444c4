"""Refinement of a path by descent on the functional (the adjoint of
Eq. VMDcondition with respect to the frames) on the GPU against the FP64
oracle's restatement of the same loop: initial Phi to 1e-6, the first
iterations' Phi to 1e-3 (the GPU gradient carries a 1e-4 relative error, so
the backtracking may pick slightly different steps later), monotone
decrease, fixed end frames, and the refined path re-scored by the oracle."""
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


def gpu_path(s, p, seed, n):
    b = B.TrialBatch(s, p, [1], trial_seeds=[seed])
    B.sim_record_frames(b.h, 0, n + 1)
    frames0 = b.get_state(0)[0][: s.n_cv]
    b.step(n)
    fr = B.sim_get_frames(b.h, n + 1, s.n_cv)
    fr[0] = frames0
    return b, fr


@pytest.mark.parametrize("name", ["tiny", "small"])
def test_refinement_matches_the_oracle(name):
    s, p = S.tiny_chain(0) if name == "tiny" else S.small_solvated()
    b, F = gpu_path(s, p, 91, 40)
    try:
        n_iter, step = 12, 1e-3
        X, hist, acc = B.phi_frames_refine(b.h, 0, F, n_iter, step)
        Xo, hist_o, acc_o = O.refine_frames(s, p, F, n_iter, step)
    finally:
        b.close()
    assert hist[0] > 0.0 and acc > 0
    assert hist[0] == pytest.approx(hist_o[0], rel=1e-6)
    assert np.all(np.diff(hist) <= 0.0) and hist[-1] < hist[0]
    assert np.array_equal(X[0], F[0]) and np.array_equal(X[-1], F[-1])
    np.testing.assert_allclose(hist[1:4], hist_o[1:4], rtol=1e-3)
    # the refined path re-scored by the oracle
    assert O.phi_frames(s, p, X)[0] == pytest.approx(hist[-1], rel=1e-6)
    assert hist[-1] == pytest.approx(hist_o[-1], rel=0.1)


@pytest.mark.parametrize("name", ["tiny", "small"])
def test_refinement_iterations_on_shared_paths(name):
    """Iteration by iteration from the same path (the GPU's path after the
    previous iteration, on both sides): each iteration's Phi and moved frames
    agree with the oracle's restatement, the Phi history to 1e-5 relative
    (the GPU gradient carries a 1e-4 relative error, which moves the trial
    point by that fraction of one step)."""
    s, p = S.tiny_chain(0) if name == "tiny" else S.small_solvated()
    b, X = gpu_path(s, p, 91, 40)
    try:
        step = 1e-3
        for it in range(8):
            Xg, hg, ag = B.phi_frames_refine(b.h, 0, X, 1, step)
            Xo, ho, ao = O.refine_frames(s, p, X, 1, step)
            assert hg[0] == pytest.approx(ho[0], rel=1e-6), it
            assert ag == ao, it
            if not ag:
                break
            assert hg[1] == pytest.approx(ho[1], rel=1e-5), it
            # the step (eta g) agrees to the gradient's 1e-4; then one FP32 rounding
            assert np.abs(Xg - Xo).max() <= 1e-3 * np.abs(Xo - X).max() + 5e-7, it
            X = Xg
        assert it >= 3
    finally:
        b.close()
