"""The one-kernel step (every phase of every trial in one cooperative kernel,
grid barriers between phases), and the kernel-per-phase step whose rebuild
kernels sit in conditional graph nodes, against the kernel-per-phase step:
the same device code per phase, so the states must agree bit for bit, with
list rebuilds, on single trials and on a mixed batch; a grid barrier whose poll
bound runs out ends the call with SIM_ETIMEOUT and leaves the GPU usable;
the step-form autotuner restores the state it started from."""
import numpy as np
import pytest

from paper_1405_6104_gb300 import binding as B
from paper_1405_6104_gb300 import systems as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1405_6104_gb300 import build
    build.build()
    B.load()


def _run(systems, p, tps, seeds, mode, calls):
    with B.TrialBatch(systems, p, tps, trial_seeds=seeds) as b:
        B.sim_set_step_mode(b.h, mode)
        for n in calls:
            b.step(n)
        diag = B.sim_diagnostics(b.h)
        return [b.get_state(t) for t in range(b.n_trials)], diag


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("which", ["small", "mixed", "benchmarked"])
def test_step_forms_are_bit_identical(which, mode):
    if which == "small":
        s, p = S.small_solvated()
        args = ([s], p, [1], [9])
    elif which == "mixed":
        s1, p = S.tiny_chain(0)
        s2, _ = S.small_solvated()
        args = ([s1, s2], p, [2, 2], [5, 6, 7, 8])
    else:
        s, p = S.plain_single(1)
        args = ([s], p, [1], [1000])
    calls = (20, 7, 13)  # graph chunks, direct steps, both
    ref, d0 = _run(*args, 0, calls)
    got, d1 = _run(*args, mode, calls)
    for x, y in zip(ref, got):
        assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])
        assert x[2][3] == y[2][3] and x[2][1] == y[2][1]
    assert d0["trial_rebuilds"] == d1["trial_rebuilds"] and d0["trial_rebuilds"] > len(ref)


def test_one_kernel_step_barrier_timeout_is_reported(monkeypatch):
    """A poll bound of zero: every grid barrier that a block reaches before
    the last one gives up at once; the kernel records the timeout and ends,
    the call returns SIM_ETIMEOUT, and a new batch runs normally."""
    s, p = S.small_solvated()
    monkeypatch.setenv("VPATH_SPIN_LIMIT", "0")
    with B.TrialBatch(s, p, [1], trial_seeds=[9]) as b:
        B.sim_set_step_mode(b.h, 1)
        with pytest.raises(B.SimError) as e:
            b.step(10)
        assert e.value.code == B.SIM_ETIMEOUT
    monkeypatch.delenv("VPATH_SPIN_LIMIT")
    ref, _ = _run([s], p, [1], [9], 0, (10,))
    got, _ = _run([s], p, [1], [9], 1, (10,))
    assert np.array_equal(ref[0][0], got[0][0])


def test_step_form_autotuner_restores_the_state():
    s, p = S.small_solvated()
    with B.TrialBatch(s, p, [2], trial_seeds=[3, 4]) as b:
        b.step(10)
        before = [b.get_state(t) for t in range(2)]
        step0 = B.sim_step_count(b.h)
        mode = B.sim_autotune_step(b.h, 2)
        assert mode in (0, 1, 2) and B.sim_step_mode(b.h) == mode
        assert B.sim_step_count(b.h) == step0
        for t in range(2):
            pos, vel, cv = b.get_state(t)
            assert np.array_equal(pos, before[t][0]) and np.array_equal(vel, before[t][1])
            assert cv[1] == before[t][2][1] and cv[3] == before[t][2][3]
        b.step(10)  # and it steps on in the picked form
