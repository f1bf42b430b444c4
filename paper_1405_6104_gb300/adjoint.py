"""Adjoint of the bias functional along a simulated trial path, with segment
checkpointing of the frames.

The variational condition of Eq. VMDcondition is a functional derivative of
Phi with respect to the path; ``trajectory_adjoint`` returns dPhi/dX_n for
every frame X_n (the reaction-coordinate atoms at steps step0 .. step0 + N)
of one trial, computed entirely by the library's kernels:

1. forward: the batch advances N steps in calls of ``every`` steps; before
   each call the full state of every trial (positions, velocities, z_m, Phi,
   step counter) is kept as a checkpoint, and the per-step record holds z_n
   and Q_n of the trial;
2. the coefficients A_n, B_n of dPhi/dX_n = A_n grad z + B_n H_z w follow
   from the record (``phi_adjoint_coefficients``);
3. reverse: segment by segment, from the last one back, the checkpoint is
   restored and the segment re-run with the frame recorder on (bit-identical
   to the forward run: same list schedule, same call boundaries, counter-based
   noise), and ``phi_frames_adjoint`` turns the segment's frames into
   gradients.

Only ``every`` + 1 frames and the checkpoints are held at a time.
"""
from __future__ import annotations

import numpy as np

from . import binding as B


def _capture(batch):
    h = batch.h
    states = [B.sim_get_state(h, t) for t in range(batch.n_trials)]
    return B.sim_step_count(h), states


def _restore(batch, ck):
    step, states = ck
    pos = np.concatenate([s[0] for s in states])
    vel = np.concatenate([s[1] for s in states])
    cv = np.array([[s[2][1], s[2][3]] for s in states])
    # the step counter first: the restore's own force evaluation records its
    # frame under the current step number
    B.sim_set_step_count(batch.h, step)
    B.sim_set_state(batch.h, -1, pos, vel, cv)


def trajectory_adjoint(batch, trial: int, n_steps: int, every: int = 50, keep_frames: bool = False):
    """Runs the batch n_steps forward and returns (Phi over the path, dPhi/dX
    of shape (n_steps + 1, n_cv, 3), info).  The batch ends in its forward
    end state.  info holds the forward and replayed frames when keep_frames."""
    h = batch.h
    nst = batch.params.nstlist
    step0 = B.sim_step_count(h)
    if every % nst or n_steps % every or step0 % nst:
        raise ValueError("every must be a multiple of nstlist, n_steps of every, and the start a list step")
    n_cv = batch.systems[_system_of(batch, trial)].n_cv
    nseg = n_steps // every
    cap = n_steps + 1
    B.sim_record(h, cap)
    B.sim_record_frames(h, trial, cap if keep_frames else 0)
    z0 = B.sim_get_state(h, trial)[2][0]
    phi_start = B.sim_get_state(h, trial)[2][3]
    ckpts = [_capture(batch)]
    for _ in range(nseg):
        batch.step(every)
        ckpts.append(_capture(batch))
    phi_end = ckpts[-1][1][trial][2][3]
    rec = B.sim_get_record(h, trial, cap)
    idx = [(step0 + k) % cap for k in range(1, n_steps + 1)]
    z = np.concatenate([[z0], rec[idx, 0]])
    Q = np.concatenate([[0.0], rec[idx, 4]])
    coef, phi = B.phi_adjoint_coefficients(h, z, Q)
    info = {"phi_handle": phi_end - phi_start, "z": z}
    if keep_frames:
        fr = B.sim_get_frames(h, cap, n_cv)
        fwd = fr[[(step0 + k) % cap for k in range(n_steps + 1)]]
        fwd[0] = ckpts[0][1][trial][0][:n_cv]  # the start state was computed before recording began
        info["forward_frames"] = fwd
    # reverse sweep over the segments
    grad = np.zeros((n_steps + 1, n_cv, 3))
    replay = np.zeros((n_steps + 1, n_cv, 3)) if keep_frames else None
    B.sim_record_frames(h, trial, every + 1)
    for s in reversed(range(nseg)):
        _restore(batch, ckpts[s])
        batch.step(every)
        seg_step0 = ckpts[s][0]
        fr = B.sim_get_frames(h, every + 1, n_cv)
        order = [(seg_step0 + k) % (every + 1) for k in range(every + 1)]
        lo = 0 if s == 0 else 1
        frames = fr[order[lo:]]
        g0 = s * every + lo
        rows = slice(g0, s * every + every + 1)
        _, _, G = B.phi_frames_adjoint(h, trial, frames, coef=coef[rows])
        grad[rows] = G
        if keep_frames:
            replay[rows] = frames
    B.sim_record_frames(h, trial, 0)
    _restore(batch, ckpts[-1])
    if keep_frames:
        info["replayed_frames"] = replay
    return phi, grad, info


def _system_of(batch, trial: int) -> int:
    t = trial
    for s, n in enumerate(batch.trials_per_system):
        if t < n:
            return s
        t -= n
    raise IndexError(trial)
