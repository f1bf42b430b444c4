"""The allocation-free reaction-coordinate entry point (cv_eval_noalloc) gives
the same z and gradient as the batched path, on two calls in a row.

It exists for callers that must not allocate device memory (their memory
belongs to another allocator or a fixed budget, or they cannot accept the
synchronisation of cudaMalloc); its scratch is a fixed static device array
shared by all calls, so the second call also checks that a call leaves
nothing behind that the next one would pick up.  This file is collected last
on purpose."""
import numpy as np
import pytest

from paper_1405_6104_gb300 import binding as B
from paper_1405_6104_gb300 import systems as S

pytestmark = pytest.mark.gpu


def rel_rms(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("which", ["tiny", "small"])
def test_no_alloc_matches_batched_path_on_two_calls(which):
    import torch
    from paper_1405_6104_gb300 import build
    build.build()
    s, p = S.tiny_chain(0) if which == "tiny" else S.small_solvated()
    p.k_ratchet = 8.0
    p0 = S.Params(**{**p.__dict__, "k_ratchet": 0.0})
    with B.TrialBatch(s, p, [1], trial_seeds=[21]) as b:
        b.step(15)
        pos, vel, cv = b.get_state(0)
        # ratchet amplitude a = 0.5: the batched path's force then carries -(k_R/2) a grad z
        b.set_state(0, pos, vel, cv_state=[cv[0] - 0.5, 0.0])
        pos, vel, cv = b.get_state(0)
        _, F = b.energy_forces(0)
    with B.TrialBatch(s, p0, [1], trial_seeds=[21]) as b0:
        b0.set_state(0, pos, vel)
        _, F0 = b0.energy_forces(0)
    n = s.n_cv
    dev = torch.device("cuda", 0)
    d_pos = torch.tensor(pos[:n].astype(np.float32).reshape(-1), device=dev)
    d_nat = torch.tensor(np.asarray(s.native_pos, np.float64).reshape(-1), device=dev)
    for call in range(2):
        d_z = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        d_g = torch.full((3 * n,), float("nan"), dtype=torch.float64, device=dev)
        rc, msg = B.cv_eval_noalloc(d_pos.data_ptr(), d_nat.data_ptr(), n, s.box, p, d_z.data_ptr(),
                                    d_g.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert rc == B.SIM_OK, msg
        z = float(d_z.item())
        g = d_g.cpu().numpy().reshape(n, 3)
        assert z == pytest.approx(cv[0], rel=1e-10, abs=1e-10), f"call {call}"
        expected = F0.copy()
        expected[:n] += -0.5 * p.k_ratchet * cv[2] * g
        assert rel_rms(F, expected) < 1e-5, f"call {call}"


def test_no_alloc_rejects_sizes_beyond_its_scratch():
    s, p = S.tiny_chain(0)
    rc, msg = B.cv_eval_noalloc(1, 1, 2049, s.box, p, 1, 1)
    assert rc == B.SIM_EINVAL and "2048" in msg


def _synthetic_reaction_coordinate(n, seed):
    """n reaction-coordinate atoms packed at about 60 atoms/nm^3 in an 8 nm
    box (many pairs inside the contact cut-off) and a native structure 0.1 nm
    away from them."""
    rng = np.random.default_rng(seed)
    side = (n / 60.0) ** (1.0 / 3.0)
    pos = (2.0 + side * rng.random((n, 3))).astype(np.float32).astype(np.float64)
    nat = pos + 0.1 * rng.normal(size=(n, 3))
    return pos, nat


@pytest.mark.parametrize("sizes", [(2048, 1000, 2048)])
def test_no_alloc_at_its_limit_and_ragged_against_the_oracle(sizes):
    """The fixed scratch at its limit (2048 atoms: the whole 64 x 64 tile
    grid) and a ragged size (1000 atoms: 32 tile rows, the last one partial),
    larger call first, each against the FP64 oracle: nothing a larger call
    leaves in the shared array reaches a smaller one."""
    import types

    import torch

    import oracle as O
    from paper_1405_6104_gb300 import build
    build.build()
    B.load()
    p = S.Params(cv_min_sep=3)
    dev = torch.device("cuda", 0)
    box = 8.0
    for call, n in enumerate(sizes):
        pos, nat = _synthetic_reaction_coordinate(n, seed=100 + n)
        ref = types.SimpleNamespace(n_cv=n, native_pos=nat, box=box)
        z_ref, g_ref = O.cv(ref, p, pos)
        d_pos = torch.tensor(pos.astype(np.float32).reshape(-1), device=dev)
        d_nat = torch.tensor(nat.reshape(-1), device=dev)
        d_z = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        d_g = torch.full((3 * n,), float("nan"), dtype=torch.float64, device=dev)
        rc, msg = B.cv_eval_noalloc(d_pos.data_ptr(), d_nat.data_ptr(), n, box, p, d_z.data_ptr(), d_g.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert rc == B.SIM_OK, msg
        assert z_ref > 0
        assert float(d_z.item()) == pytest.approx(z_ref, rel=1e-10), f"call {call}, n_cv {n}"
        assert rel_rms(d_g.cpu().numpy().reshape(n, 3), g_ref) < 1e-5, f"call {call}, n_cv {n}"


def test_no_alloc_rejects_bad_contact_parameters():
    s, p = S.tiny_chain(0)
    for bad in ({"cv_min_sep": -1}, {"cv_r_switch": 0.0}, {"cv_r_cut": 0.9, "cv_r_switch": 1.0}):
        q = S.Params(**{**p.__dict__, **bad})
        rc, msg = B.cv_eval_noalloc(1, 1, 12, s.box, q, 1, 1)
        assert rc == B.SIM_EINVAL and "invalid" in msg, bad
