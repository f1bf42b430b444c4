"""Pins of the oracle's path refinement (descent on the functional of
Eq. VMDcondition over the inner frames): monotone decrease, fixed ends,
first-order agreement with the gradient, and the zero case of a path whose
reaction coordinate never rises (Phi = 0, nothing to refine)."""
import numpy as np
import pytest

import oracle as O
from paper_1405_6104_gb300 import systems as S


def _path():
    s, p = S.tiny_chain(0)
    r = O.run(s, p, 77, 40, record_every=1)
    return s, p, r["frames"][:, : s.n_cv, :]


def test_refinement_decreases_phi_and_keeps_the_ends():
    s, p, F = _path()
    X, hist, acc = O.refine_frames(s, p, F, 15, 1e-3)
    assert hist[0] > 0 and acc > 0
    assert np.all(np.diff(hist) <= 0.0)
    assert hist[-1] < 0.5 * hist[0]
    assert np.array_equal(X[0], F[0]) and np.array_equal(X[-1], F[-1])
    assert O.phi_frames(s, p, X)[0] == pytest.approx(hist[-1], rel=1e-12)


def test_first_step_follows_the_gradient():
    # Phi(X - eta g) = Phi(X) - eta |g|^2 + O(eta^2) for the free frames
    s, p, F = _path()
    phi, G = O.phi_frames_grad(s, p, F)
    G[0] = G[-1] = 0.0
    gg = float((G * G).sum())
    for eta in (1e-6, 1e-7):
        d = O.phi_frames(s, p, F - eta * G)[0] - phi
        assert d == pytest.approx(-eta * gg, rel=2e-2)


def test_monotone_path_has_nothing_to_refine():
    s, p, F = _path()
    z = [O.cv(s, p, f)[0] for f in F]
    # a path through the frames sorted by decreasing z never lets z rise: Phi = 0
    order = np.argsort(z)[::-1]
    Fm = F[order]
    X, hist, acc = O.refine_frames(s, p, Fm, 5, 1e-3)
    assert hist[0] == 0.0 and acc == 0 and np.array_equal(X, Fm)


def test_refined_frames_are_fp32_values():
    """The moved coordinates are FP32 values (the precision of the frames the
    path is recorded in), the end frames the input's."""
    s, p, F = _path()
    F = F.astype(np.float32).astype(np.float64)
    X, hist, acc = O.refine_frames(s, p, F, 6, 1e-3)
    assert acc > 0
    assert np.array_equal(X.astype(np.float32).astype(np.float64), X)
    assert not np.array_equal(X[1:-1], F[1:-1])
