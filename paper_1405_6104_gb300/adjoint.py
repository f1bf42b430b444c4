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
3. replay: each segment is re-run from its checkpoint with the frame
   recorder on, bit-identical to the forward run (the forward run rebuilds
   every list at each checkpoint, as the restore there does; same call
   boundaries, counter-based noise, list rebuilds decided per trial from its
   own state).  By default the segments are
   replayed side by side as the trials of a second batch of the trial's
   system ("batched": every trial carries the original seed and its
   segment's start step as noise offset, so it draws the original noise;
   trials of a batch do not influence each other), up to ``group`` segments
   per call; "sequential" restores and re-runs them one after another on the
   original batch;
4. ``phi_frames_adjoint`` turns each segment's frames into gradients.

Only the frames of the segments being replayed and the checkpoints are held.
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


def _replay_batch(batch, trial: int, size: int):
    """A batch of `size` trials of `trial`'s system with its seed, kept on
    the batch object for later calls."""
    cache = batch.__dict__.setdefault("_replay_batches", {})
    key = (trial, size)
    if key not in cache:
        sys_ = batch.systems[_system_of(batch, trial)]
        seed = B.sim_trial_seed(batch.h, trial)
        rb = B.TrialBatch(sys_, batch.params, [size], trial_seeds=[seed] * size)
        B.sim_autotune(rb.h, 3, None)  # launch shapes for this batch size (all give the same results)
        B.sim_autotune_step(rb.h, 2)    # and the step form (both give the same results)
        cache[key] = rb
    return cache[key]


def _replay_group(batch, trial, ckpts, segs, every, n_cv, group):
    """Frames (len(segs), every + 1, n_cv, 3) of the segments `segs`, replayed
    side by side from their checkpoints."""
    rb = _replay_batch(batch, trial, group)
    h = rb.h
    B.sim_record_frames(h, -1, every + 1)
    B.sim_set_step_count(h, 0)
    # padding trials (a short last group) replay the group's first segment
    src = list(segs) + [segs[0]] * (group - len(segs))
    # the forward trial's own noise offset carries over (a forward batch may
    # itself be a replay batch)
    off0 = B.sim_noise_offset(batch.h, trial)
    for k, sg in enumerate(src):
        B.sim_set_noise_offset(h, k, off0 + ckpts[sg][0])
    states = [ckpts[sg][1][trial] for sg in src]
    pos = np.concatenate([st[0] for st in states])
    vel = np.concatenate([st[1] for st in states])
    cv = np.array([[st[2][1], st[2][3]] for st in states])
    B.sim_set_state(h, -1, pos, vel, cv)
    rb.step(every)
    fr = B.sim_get_frames(h, every + 1, n_cv, group)
    B.sim_record_frames(h, -1, 0)
    return fr[: len(segs)]


def trajectory_adjoint(batch, trial: int, n_steps: int, every: int = 50, keep_frames: bool = False,
                       replay: str = "batched", group: int = 16):
    """Runs the batch n_steps forward and returns (Phi over the path, dPhi/dX
    of shape (n_steps + 1, n_cv, 3), info).  The batch ends in its forward
    end state.  info holds the forward and replayed frames when keep_frames.
    replay: "batched" (segments side by side, up to `group` per call, on a
    second batch kept with this one) or "sequential"."""
    if replay not in ("batched", "sequential"):
        raise ValueError("replay must be 'batched' or 'sequential'")
    h = batch.h
    step0 = B.sim_step_count(h)
    if every < 1 or n_steps % every:
        raise ValueError("n_steps must be a multiple of every >= 1")
    n_cv = batch.systems[_system_of(batch, trial)].n_cv
    nseg = n_steps // every
    cap = n_steps + 1
    B.sim_record(h, cap)
    B.sim_record_frames(h, trial, cap if keep_frames else 0)
    # every checkpoint holds freshly built lists, like the state a restore
    # there produces
    B.sim_rebuild(h)
    z0 = B.sim_get_state(h, trial)[2][0]
    phi_start = B.sim_get_state(h, trial)[2][3]
    ckpts = [_capture(batch)]
    for _ in range(nseg):
        batch.step(every)
        B.sim_rebuild(h)
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
    grad = np.zeros((n_steps + 1, n_cv, 3))
    replayed = np.zeros((n_steps + 1, n_cv, 3)) if keep_frames else None

    def consume(s, seg_frames):
        # seg_frames[k]: the frame of step ckpt_s + k, k = 0 .. every
        lo = 0 if s == 0 else 1
        frames = seg_frames[lo:]
        rows = slice(s * every + lo, s * every + every + 1)
        _, _, G = B.phi_frames_adjoint(h, trial, frames, coef=coef[rows])
        grad[rows] = G
        if keep_frames:
            replayed[rows] = frames

    if replay == "batched":
        g = max(1, min(group, nseg))
        for s0 in range(0, nseg, g):
            segs = list(range(s0, min(s0 + g, nseg)))
            fr = _replay_group(batch, trial, ckpts, segs, every, n_cv, g)
            for k, s in enumerate(segs):
                consume(s, fr[k])
    else:
        B.sim_record_frames(h, trial, every + 1)
        for s in reversed(range(nseg)):
            _restore(batch, ckpts[s])
            batch.step(every)
            seg_step0 = ckpts[s][0]
            fr = B.sim_get_frames(h, every + 1, n_cv)
            consume(s, fr[[(seg_step0 + k) % (every + 1) for k in range(every + 1)]])
        B.sim_record_frames(h, trial, 0)
        _restore(batch, ckpts[-1])
    if keep_frames:
        info["replayed_frames"] = replayed
    return phi, grad, info


def _system_of(batch, trial: int) -> int:
    t = trial
    for s, n in enumerate(batch.trials_per_system):
        if t < n:
            return s
        t -= n
    raise IndexError(trial)
