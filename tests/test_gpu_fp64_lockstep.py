"""The CUDA path (float32) against the FP64 oracle in lockstep, with near-tie
flags and resynchronisation (fp64_lockstep.py).

Off flagged steps the integer state and every decision of the GPU must equal
the FP64 oracle's; a step whose decisions differ must be explained by a
near-tie of the oracle (a position within 5e-3 m of the arrival line or of the
jam spacing, or a choice / merge top-2 gap below 1e-4), after which the
oracle's state is copied into the GPU (sim_set_state) and the run goes on.
Floats against FP64: positions within 1e-4 of their link's length, speeds and
travel times within 1e-4 relative on unflagged bins.  The GPU flags exactly the
steps the oracle's float build flags (the two are bitwise equal).
"""
import json

import numpy as np
import pytest

import fp64_lockstep as LK
from oracle.oracle import OracleSim
from paper_2603_25068_b300 import scenario as S

pytestmark = pytest.mark.gpu

RTOL = 1e-4


@pytest.fixture(scope="module")
def Simulator():
    import torch
    assert torch.cuda.is_available()
    from paper_2603_25068_b300.sim import Simulator
    return Simulator


def _run(Simulator, sc, executor):
    g = Simulator(sc)
    g.set_executor(executor)
    rep = LK.run(g, OracleSim(sc, "fp64"), sc.T)
    g.close()
    err = rep["max_rel_err"]
    assert err["positions"] < RTOL and err["speed"] < RTOL and err["travel_time"] < RTOL, err
    ref = LK.run(OracleSim(sc, "fp32"), OracleSim(sc, "fp64"), sc.T)
    assert [t for t, _ in rep["flags"]] == [t for t, _ in ref["flags"]]
    summary = dict(case=sc.name, executor=executor, steps=sc.T, flagged_steps=[t for t, _ in rep["flags"]],
                   near_ties=sorted({r[0] for _, rs in rep["flags"] for r in rs}),
                   bins_compared=rep["bins_compared"], max_rel_err=err)
    print("fp64 lockstep:", json.dumps(summary))
    return rep


@pytest.mark.parametrize("executor", ["persistent", "step"])
def test_tiny_grid_against_fp64(Simulator, executor):
    rep = _run(Simulator, S.tiny_grid().copy(obs_every=30), executor)
    assert rep["n_flags"] <= 20 and rep["bins_compared"] >= 3


def test_city_small_against_fp64(Simulator):
    rep = _run(Simulator, S.city_small(), "persistent")
    assert rep["n_flags"] <= 5


def test_random_grids_against_fp64(Simulator):
    for seed in (1, 2, 3):
        sc = S.random_small(seed=seed, side=3, n_vehicles=150, T=150).copy(obs_every=40)
        _run(Simulator, sc, "persistent")
