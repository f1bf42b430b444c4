"""The two-dimensional toy model on the GPU (SM, "Illustrative Application in
a Toy Model") against the FP64 oracle, and against what the section reports.

Parity: the kernel runs FP64 in the operation order of the equations, so a
trial follows the oracle's trial step for step; the only difference is the
last bit of the Box-Muller transcendentals (CUDA's log/sincos against the
host's), which the dynamics amplify slowly.  Paths are compared to 1e-8 over
the first 3000 steps; the functional and first passage of any GPU path are
recomputed by the oracle from that path (1e-12).  The section's findings
that the model must reproduce: plain Langevin rarely crosses the ring within
90 000 steps and then through the gate near (1.5, 0); the fraction of rMD
trials reaching the product within 30 000 steps grows with K_R and saturates
for large K_R; the optimum rMD path (least Phi) crosses at the gate."""
import dataclasses

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


def ring_crossing_angle(path, r_ring=1.2):
    """Polar angle where the path last comes inside r_ring before its end."""
    r = np.hypot(path[:, 0], path[:, 1])
    ok = np.isfinite(r)
    r, P = r[ok], path[ok]
    outside = np.where(r > r_ring)[0]
    j = outside[-1]
    return float(np.arctan2(P[j, 1], P[j, 0]))


@pytest.mark.parametrize("bias", [S.TOY_RATCHET, S.TOY_STEERED, S.TOY_NONE])
def test_paths_match_the_oracle(bias):
    tp = dataclasses.replace(S.Toy2dParams(), bias=bias)
    ks = np.array([0.5, 2.0, 8.0, 30.0] * 3)
    seeds = np.arange(100, 100 + len(ks), dtype=np.uint64)
    n = 3000
    passage, phi, state, path = B.toy2d_run(tp, ks, seeds, n, path_every=1)
    for t in range(len(ks)):
        pr, phr, str_, pathr = O.toy2d_run(tp, ks[t], int(seeds[t]), n, want_path=True)
        m = len(pathr)
        assert np.abs(path[t, :m] - pathr).max() < 1e-8, t
        assert np.all(np.isnan(path[t, m:]))
        assert passage[t] == pr
        assert phi[t] == pytest.approx(phr, rel=1e-9, abs=1e-12)
        assert np.abs(state[t] - str_).max() < 1e-7
        # the functional of the GPU's own path, recomputed by the oracle
        Phi_o, pas_o = O.toy2d_phi_path(tp, ks[t], path[t, :m])
        assert pas_o == passage[t]
        assert phi[t] == pytest.approx(Phi_o, rel=1e-12, abs=1e-15)


def test_full_size_rmd_batch_sampled_and_batch_invariant():
    """2000 trials x 30 000 steps at K_R = 8 (the section's trial count and
    length); sampled trials re-run alone with their paths recorded give the
    same results bit for bit, and the oracle recomputes their functional."""
    tp, ks, seeds = S.toy2d_rmd_batch(2000, [8.0])
    n = 30000
    passage, phi, state, _ = B.toy2d_run(tp, ks, seeds, n)
    sample = [0, 777, 1999]
    p1, f1, s1, path = B.toy2d_run(tp, ks[sample], seeds[sample], n, path_every=1)
    assert np.array_equal(p1, passage[sample]) and np.array_equal(f1, phi[sample])
    assert np.array_equal(s1, state[sample])
    for j, t in enumerate(sample):
        m = (p1[j] + 1) if p1[j] >= 0 else n + 1
        Phi_o, pas_o = O.toy2d_phi_path(tp, ks[t], path[j, :m])
        assert pas_o == p1[j] and f1[j] == pytest.approx(Phi_o, rel=1e-12, abs=1e-15)
        # the oracle's own trial agrees over its first 3000 steps
        _, _, _, pathr = O.toy2d_run(tp, ks[t], int(seeds[t]), 3000, want_path=True)
        assert np.abs(path[j, : len(pathr)] - pathr).max() < 1e-8


def test_rmd_reach_fraction_grows_and_saturates():
    """The section: for K_R below about 4 the fraction of the 2000 rMD trials
    that reach the product within 30 000 steps varies strongly with K_R; for
    larger K_R almost all of them do."""
    kvals = [0.3, 1.0, 4.0, 16.0, 40.0]
    tp, ks, seeds = S.toy2d_rmd_batch(2000, kvals)
    passage, phi, _, _ = B.toy2d_run(tp, ks, seeds, 30000, want_state=False)
    frac = [(passage[ks == k] >= 0).mean() for k in kvals]
    assert frac[0] < 0.15 and frac[1] < 0.3 and frac[2] > frac[1] + 0.05
    assert frac[3] > 0.95 and frac[4] > 0.95
    assert np.all(phi >= 0.0)


def test_plain_langevin_crosses_rarely_and_through_the_gate():
    """The section: of 20 000 plain Langevin trajectories of 90 000 steps from
    (0, 5), only a few reach the product, all through the gate near (1.5, 0)."""
    tp, ks, seeds = S.toy2d_plain_batch(20000)
    passage, phi, _, _ = B.toy2d_run(tp, ks, seeds, 90000, want_state=False)
    reached = np.where(passage >= 0)[0]
    assert 0 < len(reached) < 0.15 * len(seeds)
    assert np.all(phi == 0.0)
    sel = reached[:60]
    p1, _, _, path = B.toy2d_run(tp, ks[sel], seeds[sel], 90000, path_every=5, want_state=False)
    assert np.array_equal(p1, passage[sel])
    angles = np.array([ring_crossing_angle(path[j]) for j in range(len(sel))])
    assert np.mean(np.abs(angles) < np.pi / 4) > 0.9


def test_optimum_rmd_path_crosses_at_the_gate():
    """The section: after selection by the variational condition the optimum
    path crosses the ring at the gate, for every K_R scanned, although the
    biasing coordinate z ignores the gate."""
    kvals = [4.0, 8.0, 16.0]
    tp, ks, seeds = S.toy2d_rmd_batch(2000, kvals)
    passage, phi, _, _ = B.toy2d_run(tp, ks, seeds, 30000, want_state=False)
    for k in kvals:
        idx = np.where((ks == k) & (passage >= 0))[0]
        best = idx[np.argmin(phi[idx])]
        _, _, _, path = B.toy2d_run(tp, ks[[best]], seeds[[best]], 30000, path_every=1, want_state=False)
        assert abs(ring_crossing_angle(path[0])) < np.pi / 4, k
