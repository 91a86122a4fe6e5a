"""The FP64 lockstep protocol with near-tie flags (fp64_lockstep.py), run on the
CPU with the oracle's float build as the float side.

The float build takes every decision in float32 with the kernel's operation
order (the GPU path is bitwise equal to it, test_gpu_forward.py), so the
near-ties flagged here are the ones the GPU meets (test_gpu_fp64_lockstep.py).
The protocol is also checked to reject float sides that are wrong: mistakes
planted in the float side's inputs must surface as unexplained mismatches or
as errors above tolerance.
"""
import numpy as np
import pytest

import fp64_lockstep as LK
from oracle.oracle import OracleSim
from paper_2603_25068_b300 import scenario as S

POS_RTOL = 1e-4      # positions, relative to their link's length
OUT_RTOL = 1e-4      # speeds and travel times per bin


def _check(rep):
    assert rep["identical_steps"] + rep["n_flags"] == rep["steps"]
    for t, reasons in rep["flags"]:
        assert reasons, f"step {t} flagged without a near-tie"
        for kind, _, _, margin in reasons:
            tol = LK.DELTA_POS if kind in ("arrival", "vacancy") else LK.DELTA_G
            assert abs(margin) < tol
    err = rep["max_rel_err"]
    assert err["positions"] < POS_RTOL, err
    assert err["speed"] < OUT_RTOL and err["travel_time"] < OUT_RTOL, err


def test_tiny_grid_float_build_against_fp64():
    sc = S.tiny_grid().copy(obs_every=30)
    rep = LK.run(OracleSim(sc, "fp32"), OracleSim(sc, "fp64"), sc.T)
    _check(rep)
    # the flagged decisions are vacancy tests of full one-lane links: with
    # kappa = 0.2 f32 the jam spacing is 5 m in float32 and 5 - 7.5e-8 m in
    # double, so 40 queued vehicles leave the rearmost at exactly 5 m (not
    # vacant) in float32 and 3e-6 m beyond it (vacant) in double
    kinds = {r[0] for _, reasons in rep["flags"] for r in reasons}
    assert kinds <= {"vacancy", "merge", "choice", "arrival"}
    assert rep["n_flags"] <= 20
    assert rep["bins_compared"] >= 3


def test_city_small_float_build_against_fp64():
    sc = S.city_small()
    rep = LK.run(OracleSim(sc, "fp32"), OracleSim(sc, "fp64"), sc.T)
    _check(rep)
    assert rep["n_flags"] <= 5
    assert rep["bins_compared"] >= 1


@pytest.mark.parametrize("plant", ["w", "alpha_origin", "eps_arr", "kappa"])
def test_protocol_rejects_a_wrong_float_side(plant):
    """A float side with a planted mistake (one input perturbed) fails: its
    decisions differ away from near-ties, or its positions drift beyond the
    tolerance."""
    sc = S.tiny_grid().copy(obs_every=30)
    bad = dict(w=lambda: sc.copy(w=(sc.w + np.float32(1e-3)).astype(np.float32)),
               alpha_origin=lambda: sc.copy(alpha_origin=2.6),
               eps_arr=lambda: sc.copy(eps_arr=6.0),      # leaders at 194.6 m of 200 m arrive early
               kappa=lambda: sc.copy(kappa=(sc.kappa * np.float32(1.001)).astype(np.float32)))[plant]()
    with pytest.raises(AssertionError):
        _check(LK.run(OracleSim(bad, "fp32"), OracleSim(sc, "fp64"), sc.T))


def test_state_import_continues_like_the_original_run():
    """The oracle's state import (the resync step of the protocol) continues a
    run exactly: importing a run's own state at step t changes nothing."""
    sc = S.random_small(seed=2, side=3, n_vehicles=150, T=150).copy(obs_every=40)
    a, b = OracleSim(sc, "fp64"), OracleSim(sc, "fp64")
    a.reset(sc.T)
    b.reset(sc.T)
    a.step(57)
    b.step(57)
    b.set_state(a.state(), 57)
    a.step(sc.T - 57)
    b.step(sc.T - 57)
    for k, v in a.state().items():
        np.testing.assert_array_equal(v, b.state()[k], err_msg=k)
    # bins that start after the import are whole
    np.testing.assert_array_equal(a.outputs()["counts"][2:], b.outputs()["counts"][2:])
    # an inconsistent state is refused
    st = a.state()
    st["veh_rank"] = np.where(st["veh_link"] >= 0, 0, -1).astype(np.int32)
    if np.bincount(st["veh_link"][st["veh_link"] >= 0]).max() > 1:
        with pytest.raises(RuntimeError):
            b.set_state(st, sc.T)
