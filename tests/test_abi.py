"""The C-ABI library loads and exports every symbol that include/*.h
declares; host-side validation rejects bad input before touching a GPU.
CPU only (no compute calls)."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

from paper_1405_6104_gb300 import binding as B
from paper_1405_6104_gb300 import build as BUILD
from paper_1405_6104_gb300 import systems as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    BUILD.build()
    return B.load()


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            if m.group(1) not in ("if", "defined"):
                names.append(m.group(1))
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "sim_create" in names and "sim_step_batch" in names and "bias_functional" in names
    assert "energy_forces" in names
    for n in names:
        assert hasattr(lib, n), n
        assert n in B._SIGS, f"binding lacks {n}"


def test_null_handles_are_rejected(lib):
    assert lib.sim_step_batch(None, 1) == B.SIM_EINVAL
    assert lib.energy_forces(None, 0, None, None) == B.SIM_EINVAL
    assert lib.sim_num_trials(None) == 0
    assert lib.sim_last_error(None) == b"null handle"
    lib.sim_destroy(None)


def _expect_einval(systems, params, trials=(1,)):
    with pytest.raises(B.SimError) as e:
        B.sim_create(systems, params, trials)
    assert e.value.code == B.SIM_EINVAL
    return str(e.value)


def test_invalid_systems_are_rejected_on_the_host(lib):
    s, p = S.tiny_chain(0)
    bad = s.copy()
    bad.box = 2.0  # < 2 (r_cut + skin)
    assert "box" in _expect_einval([bad], p)
    bad = s.copy()
    bad.bonds = np.array([[0, 999]], np.int32)
    bad.bond_r0 = np.array([0.38])
    bad.bond_k = np.array([1e5])
    assert "bond" in _expect_einval([bad], p)
    bad = s.copy()
    bad.mass = bad.mass.copy()
    bad.mass[3] = 0.0
    assert "mass" in _expect_einval([bad], p)
    bad = s.copy()
    bad.pos = bad.pos.copy()
    bad.pos[5, 1] = np.nan
    assert "non-finite" in _expect_einval([bad], p)
    p2 = S.Params(**{**p.__dict__, "nstlist": 0})
    assert "params" in _expect_einval([s], p2)
    _expect_einval([s], p, trials=(0,))
    assert "65535" in _expect_einval([s, s], p, trials=(40000, 40000))


def test_toy2d_host_validation(lib):
    import dataclasses
    tp = S.Toy2dParams()
    k, seeds = np.ones(3), np.arange(3, dtype=np.uint64)
    for bad in (dict(bias=7), dict(s_power=3), dict(dt=0.0), dict(mass=-1.0), dict(gamma=0.0), dict(kT=-0.1)):
        with pytest.raises(B.SimError) as e:
            B.toy2d_run(dataclasses.replace(tp, **bad), k, seeds, 10)
        assert e.value.code == B.SIM_EINVAL, bad
    with pytest.raises(B.SimError) as e:
        B.toy2d_run(tp, k, seeds, -1)
    assert e.value.code == B.SIM_EINVAL
    # no trials: nothing to do, no device touched
    passage, phi, state, path = B.toy2d_run(tp, np.zeros(0), np.zeros(0, np.uint64), 10)
    assert len(passage) == 0 and len(phi) == 0
