"""Adjoint of the bias functional with respect to the path frames (GPU)
against the FP64 oracle gradient and central finite differences, and the
segment-checkpointed trajectory adjoint (frames recomputed from checkpoints
must be bit-identical to the forward frames)."""
import numpy as np
import pytest

import oracle as O
from paper_1405_6104_gb300 import binding as B
from paper_1405_6104_gb300 import systems as S
from paper_1405_6104_gb300.adjoint import trajectory_adjoint

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1405_6104_gb300 import build
    build.build()
    B.load()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def biased_path(s, n=24, seed=3):
    nat, X0 = s.native_pos, s.pos[: s.n_cv]
    ts = np.concatenate([np.linspace(0.1, 0.6, n // 2), np.linspace(0.55, 1.0, n - n // 2)])
    rng = np.random.default_rng(seed)
    fr = np.stack([nat + t * (X0 - nat) + 0.01 * rng.normal(size=nat.shape) for t in ts])
    return fr.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("which", ["tiny", "small"])
def test_frames_adjoint_matches_oracle_gradient(which):
    s, p = S.tiny_chain(0) if which == "tiny" else S.small_solvated()
    fr = biased_path(s)
    with B.TrialBatch(s, p, [1]) as b:
        phi, z, G = B.phi_frames_adjoint(b.h, 0, fr)
    Phi_ref, G_ref = O.phi_frames_grad(s, p, fr)
    _, z_ref, _, _ = O.phi_frames(s, p, fr)
    assert Phi_ref > 0
    assert phi == pytest.approx(Phi_ref, rel=1e-6)
    assert np.allclose(z, z_ref, rtol=1e-11, atol=1e-11)
    assert rel(G, G_ref) < 1e-4


def test_frames_adjoint_central_differences():
    """200 random coordinates, fourth-order central differences with
    h = 1e-4 nm of Phi from the FP64 oracle (the functional is stiff enough
    that the two-point formula's O(h^2) error reaches 1e-4 at this h);
    coordinates where the stencil flips a ratchet branch or the running
    minimum are skipped."""
    s, p = S.small_solvated()
    fr = biased_path(s, n=16)
    with B.TrialBatch(s, p, [1]) as b:
        _, _, G = B.phi_frames_adjoint(b.h, 0, fr)
    _, z, a, _ = O.phi_frames(s, p, fr)
    rng = np.random.default_rng(11)
    h = 1e-4
    scale = np.abs(G).max()
    checked = 0
    for _ in range(200):
        f, i, k = rng.integers(len(fr)), rng.integers(s.n_cv), rng.integers(3)
        vals, ok = [], True
        for m in (2, 1, -1, -2):
            X = fr.copy()
            X[f, i, k] += m * h
            P, zz, aa, _ = O.phi_frames(s, p, X)
            ok &= np.array_equal(aa > 0, a > 0) and np.array_equal(np.minimum.accumulate(zz) == zz,
                                                                    np.minimum.accumulate(z) == z)
            vals.append(P)
        if not ok:
            continue
        fd = (-vals[0] + 8 * vals[1] - 8 * vals[2] + vals[3]) / (12 * h)
        assert abs(G[f, i, k] - fd) <= 1e-4 * max(abs(fd), 1e-3 * scale), (f, i, k, G[f, i, k], fd)
        checked += 1
    assert checked >= 150


def test_checkpointed_trajectory_adjoint():
    s, p = S.small_solvated()
    with B.TrialBatch(s, p, [2], trial_seeds=[31, 32]) as b:
        phi, G, info = trajectory_adjoint(b, 1, 100, every=50, keep_frames=True)
        end_state = b.get_state(1)
    fwd, rep = info["forward_frames"], info["replayed_frames"]
    assert np.array_equal(fwd, rep), "frames recomputed from checkpoints differ from the forward frames"
    assert phi == pytest.approx(info["phi_handle"], rel=1e-10, abs=1e-300)
    assert phi > 0
    # the whole path at once gives the same gradient (z and Q there come from
    # the adjoint's own kernels, rounded differently from the step kernels)
    with B.TrialBatch(s, p, [1]) as b1:
        phi1, _, G1 = B.phi_frames_adjoint(b1.h, 0, fwd)
    assert phi1 == pytest.approx(phi, rel=1e-7)
    assert rel(G, G1) < 1e-6
    # and so does the FP64 oracle
    Phi_ref, G_ref = O.phi_frames_grad(s, p, fwd)
    assert phi == pytest.approx(Phi_ref, rel=1e-6)
    assert rel(G, G_ref) < 1e-4
    assert np.isfinite(end_state[0]).all()


def test_batched_and_sequential_replays_agree():
    """Segments replayed side by side (groups of 4 of 10 segments, the last
    group padded) and one after another give bit-identical frames and
    gradients; both leave the batch in its forward end state."""
    s, p = S.small_solvated()
    out = {}
    for mode in ("batched", "sequential"):
        with B.TrialBatch(s, p, [3], trial_seeds=[41, 42, 43]) as b:
            phi, G, info = trajectory_adjoint(b, 2, 100, every=10, keep_frames=True, replay=mode, group=4)
            out[mode] = (phi, G, info, b.get_state(2), B.sim_step_count(b.h))
    pb, Gb, ib, eb, nb = out["batched"]
    ps, Gs, is_, es, ns = out["sequential"]
    assert np.array_equal(ib["forward_frames"], ib["replayed_frames"])
    assert np.array_equal(ib["replayed_frames"], is_["replayed_frames"])
    assert np.array_equal(Gb, Gs) and pb == ps
    assert np.array_equal(eb[0], es[0]) and np.array_equal(eb[1], es[1]) and nb == ns


@pytest.mark.slow
def test_adjoint_30k_system_500_frames():
    """30 000 atoms (1800-atom solute), 500 frames, checkpoints every 50
    steps: replayed frames bit-identical; the whole gradient (all 501
    frames, segment by segment from the recorded coefficients) against the
    FP64 oracle's gradient of Phi along the same frames, a 21-frame prefix
    on its own as well; central differences of the GPU functional."""
    s, p = S.adjoint_30k(3)
    p.k_ratchet = 5.0
    with B.TrialBatch(s, p, [1], trial_seeds=[3]) as b:
        phi, G, info = trajectory_adjoint(b, 0, 500, every=50, keep_frames=True)
        fwd, rep = info["forward_frames"], info["replayed_frames"]
        assert np.array_equal(fwd, rep)
        assert phi == pytest.approx(info["phi_handle"], rel=1e-10, abs=1e-300)
        Phi_all, G_all = O.phi_frames_grad(s, p, fwd)
        assert phi == pytest.approx(Phi_all, rel=1e-6)
        assert rel(G, G_all) < 1e-4
        pre = fwd[:21]
        phi_p, _, Gp = B.phi_frames_adjoint(b.h, 0, pre)
        Phi_ref, G_ref = O.phi_frames_grad(s, p, pre)
        assert phi_p == pytest.approx(Phi_ref, rel=1e-6)
        assert rel(Gp, G_ref) < 1e-4
        # fourth-order central differences of the GPU functional on 200
        # coordinates of the full path, h = 2^-13 nm (~1.2e-4 nm, exact in FP32
        # at these coordinates so the stencil offsets are exact)
        rng = np.random.default_rng(5)
        h = 2.0 ** -13
        _, z, _ = B.phi_frames_adjoint(b.h, 0, fwd)[:3]
        scale = np.abs(G).max()
        checked = 0
        nz = np.nonzero(np.abs(G).reshape(len(fwd), -1).max(1) > 0)[0]
        first_min = lambda zz: np.minimum.accumulate(zz) == zz
        for _ in range(200):
            f = int(rng.choice(nz)) if len(nz) else int(rng.integers(len(fwd)))
            i, k = rng.integers(s.n_cv), rng.integers(3)
            vals, ok = [], True
            for m in (2, 1, -1, -2):
                X = fwd.copy()
                X[f, i, k] = X[f, i, k] + m * h
                assert np.float32(X[f, i, k]) == X[f, i, k]
                P, zz, _ = B.phi_frames_adjoint(b.h, 0, X)[:3]
                ok &= np.array_equal(first_min(zz), first_min(z))
                vals.append(P)
            if not ok:
                continue
            fd = (-vals[0] + 8 * vals[1] - 8 * vals[2] + vals[3]) / (12 * h)
            if abs(fd) < 1e-6 * scale:
                continue
            assert abs(G[f, i, k] - fd) <= 1e-4 * max(abs(fd), 1e-3 * scale), (f, i, k, G[f, i, k], fd)
            checked += 1
        assert checked >= 50
