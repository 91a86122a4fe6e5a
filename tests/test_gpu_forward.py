"""Parity of the CUDA forward step against the CPU oracle.

The GPU path computes in float32.  The oracle's float build takes every
floating-point decision in that precision with the same operation order, so the
comparison is exact: integer state (link, queue order, credit, exits, origin
queues, candidates, targets, merge winners) must be identical and positions
must be bitwise equal.  Speeds are float sums in a different order: 1e-4
relative.  The double-precision oracle is compared for the error statement.
"""
import numpy as np
import pytest

from oracle.oracle import OracleSim
from paper_2603_25068_b300 import scenario as S

pytestmark = pytest.mark.gpu

RTOL = 1e-4      # float outputs summed in a different order


@pytest.fixture(scope="module")
def Simulator():
    import torch
    assert torch.cuda.is_available()
    from paper_2603_25068_b300.sim import Simulator
    return Simulator


def assert_state_equal(gs, os_, where=""):
    for k in ("veh_link", "veh_rank", "link_credit", "link_exits", "fifo_off"):
        np.testing.assert_array_equal(gs[k], os_[k], err_msg=f"{k} {where}")
    on = gs["veh_link"] >= 0
    np.testing.assert_array_equal(gs["veh_entry"][on], os_["veh_entry"][on], err_msg=f"entry {where}")
    np.testing.assert_array_equal(gs["veh_pos"], os_["veh_pos"], err_msg=f"positions {where}")


def assert_outputs_equal(g, o, T):
    np.testing.assert_array_equal(g["counts"], o["counts"])
    for k in ("n_waiting", "n_on", "n_arrived"):
        np.testing.assert_array_equal(g[k], o[k][:T + 1], err_msg=k)
    np.testing.assert_allclose(g["travel_time"], o["travel_time"], rtol=1e-6, atol=0)
    np.testing.assert_allclose(g["speed"], o["speed"], rtol=RTOL, atol=1e-5)


def lockstep(Simulator, sc, T, check_every=1, stage=2048):
    g = Simulator(sc)
    from paper_2603_25068_b300.autotune import set_stage
    set_stage(g, stage)
    o = OracleSim(sc, "fp32")
    g.reset(T)
    o.reset(T)
    for t in range(T):
        g.step(1)
        o.step(1)
        if (t + 1) % check_every == 0 or t + 1 == T:
            gr, orr = g.records(), o.records()
            for k in ("link_cand", "link_target", "node_cand", "node_target", "link_in"):
                np.testing.assert_array_equal(gr[k], orr[k], err_msg=f"{k} step {t}")
            assert_state_equal(g.state(), o.state(), f"after step {t}")
    assert_outputs_equal(g.outputs(), o.outputs(), T)


def test_lockstep_tiny_grid(Simulator):
    sc = S.tiny_grid()
    lockstep(Simulator, sc, sc.T)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_lockstep_dense_small(Simulator, seed):
    sc = S.random_small(seed=seed, side=3, n_vehicles=150, T=150)
    lockstep(Simulator, sc.copy(obs_every=40), 150)


@pytest.mark.parametrize("dn", [5.0, 30.0])
def test_lockstep_platoons(Simulator, dn):
    # agents of dn vehicles: step dn seconds, jam spacing dn / kappa, a transfer
    # takes dn of outflow credit
    sc = S.with_platoons(S.random_small(seed=2, side=3, n_vehicles=150, T=int(150 * dn)), dn)
    lockstep(Simulator, sc, sc.T)


def test_lockstep_wide_choice_set(Simulator):
    # the hub has 11 out-links: slots beyond those evaluated in parallel by the
    # persistent executor's choice warps are evaluated at the decision
    sc = S.hub()
    assert np.bincount(sc.tail).max() == 11
    lockstep(Simulator, sc, sc.T)


@pytest.mark.parametrize("stage", [256, 2048])
def test_lockstep_long_queues(Simulator, stage):
    # queues longer than a block's thread count, links larger than the stage
    # (a block of their own) and ring-buffer wrap-around of the slot arena
    sc = S.line_network(n_links=2, length=1500.0, u=13.9, kappa=0.2, q=0.5, N=700, T=900)
    lockstep(Simulator, sc.copy(obs_every=70), 900, check_every=9, stage=stage)


@pytest.mark.parametrize("stage", [256, 1024, 4096, 8192])
def test_rollout_graph_matches_oracle_city_small(Simulator, stage):
    sc = S.city_small()
    g = Simulator(sc)
    from paper_2603_25068_b300.autotune import set_stage
    set_stage(g, stage)
    out = g.rollout()
    o = OracleSim(sc, "fp32")
    ref = o.rollout()
    assert_outputs_equal(out, ref, sc.T)
    assert_state_equal(g.state(), o.state(), "end of rollout")
    # a second rollout replays the captured graph and gives the same result
    out2 = g.rollout()
    for k in out:
        np.testing.assert_array_equal(out[k], out2[k])


def test_edge_cases(Simulator):
    # no vehicles
    sc = S.tiny_grid(n_vehicles=1, T=5)
    sc = sc.copy(N=0, origin=sc.origin[:0], dest_zone=sc.dest_zone[:0], dep_step=sc.dep_step[:0],
                 od=sc.od[:0])
    out = Simulator(sc).rollout()
    assert out["counts"].sum() == 0 and np.all(out["n_waiting"] == 0)
    # a single step; horizon not a multiple of the bin
    sc = S.random_small(seed=4, n_vehicles=30, T=1)
    g, o = Simulator(sc), OracleSim(sc, "fp32")
    assert_outputs_equal(g.rollout(), o.rollout(), 1)
    sc = S.random_small(seed=4, n_vehicles=30, T=97).copy(obs_every=25)
    g, o = Simulator(sc), OracleSim(sc, "fp32")
    assert_outputs_equal(g.rollout(), o.rollout(), 97)
    # a vehicle whose origin lies in its destination zone leaves at once
    sc = S.line_network(n_links=2, N=3, T=20)
    sc = sc.copy(dest_zone=np.array([2, 0, 2], np.int32))
    g, o = Simulator(sc), OracleSim(sc, "fp32")
    assert_outputs_equal(g.rollout(), o.rollout(), 20)


def test_invalid_inputs_rejected(Simulator):
    from paper_2603_25068_b300.native import SimError, SIM_EINVAL
    sc = S.tiny_grid(n_vehicles=10, T=5)
    with pytest.raises(SimError) as e:
        Simulator(sc.copy(cost=np.zeros(sc.L, np.float32)))
    assert e.value.code == SIM_EINVAL
    with pytest.raises(SimError):
        Simulator(sc.copy(origin=np.full(sc.N, sc.V, np.int32)))
    g = Simulator(sc)
    with pytest.raises(SimError):
        g.step(1)                     # no reset
    g.reset(3)
    with pytest.raises(SimError):
        g.step(4)                     # beyond the horizon


def test_fp32_against_fp64_error_statement(Simulator):
    """Error of the float32 path against the double oracle on the tiny grid,
    up to the first decision that differs (trajectories are chaotic after it)."""
    sc = S.tiny_grid()
    g = Simulator(sc)
    o = OracleSim(sc, "fp64")
    g.reset(sc.T)
    o.reset(sc.T)
    worst = 0.0
    steps_equal = 0
    for t in range(sc.T):
        g.step(1)
        o.step(1)
        gs, os_ = g.state(), o.state()
        if not (np.array_equal(gs["veh_link"], os_["veh_link"]) and np.array_equal(gs["veh_rank"], os_["veh_rank"])):
            break
        on = gs["veh_link"] >= 0
        if on.any():
            err = np.abs(gs["veh_pos"][on] - os_["veh_pos"][on]) / np.maximum(1.0, np.abs(os_["veh_pos"][on]))
            worst = max(worst, float(err.max()))
        steps_equal = t + 1
    assert steps_equal >= 100
    assert worst < 1e-4, worst


def test_handles_with_different_launch_shapes_coexist(Simulator):
    """A handle created after another with a smaller shared-memory stage must not
    break the first one (the kernel attribute is shared by all handles)."""
    big = S.line_network(n_links=2, length=3000.0, kappa=0.8, N=50, T=60)
    small = S.tiny_grid(n_vehicles=50, T=60)
    g1 = Simulator(big)
    g2 = Simulator(small)
    o1 = g1.rollout()
    o2 = g2.rollout()
    r1 = OracleSim(big, "fp32").rollout()
    r2 = OracleSim(small, "fp32").rollout()
    assert_outputs_equal(o1, r1, 60)
    assert_outputs_equal(o2, r2, 60)
