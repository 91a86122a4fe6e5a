"""The persistent executor (one cooperative launch per run, queues resident in
shared memory, one grid barrier per step) against the two-kernel executor and
against the oracle.

Both executors evaluate every floating-point operation of the step in the same
order, so every output and every piece of state must be bitwise identical; the
oracle's float build takes the same decisions, so lockstep comparison against
it is exact as well.
"""
import numpy as np
import pytest

from oracle.oracle import OracleSim
from paper_2603_25068_b300 import scenario as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Simulator():
    import torch
    assert torch.cuda.is_available()
    from paper_2603_25068_b300.sim import Simulator
    return Simulator


STATE_KEYS = ("veh_link", "veh_rank", "veh_entry", "veh_pos", "link_credit", "link_exits", "fifo_off")
OUT_KEYS = ("counts", "speed", "travel_time", "n_waiting", "n_on", "n_arrived")
REC_KEYS = ("link_cand", "link_target", "node_cand", "node_target", "link_in")


def run(Simulator, sc, T, executor, chunks=None):
    g = Simulator(sc)
    g.set_executor(executor)
    if chunks is None:
        out = g.rollout(T)
    else:
        g.reset(T)
        for c in chunks:
            g.step(c)
        out = g.outputs()
    res = dict(out=out, state=g.state(), rec=g.records(), executor=g.executor)
    g.close()
    return res


def assert_same(a, b):
    for k in OUT_KEYS:
        np.testing.assert_array_equal(a["out"][k], b["out"][k], err_msg=k)
    for k in STATE_KEYS:
        np.testing.assert_array_equal(a["state"][k], b["state"][k], err_msg=k)
    for k in REC_KEYS:
        np.testing.assert_array_equal(a["rec"][k], b["rec"][k], err_msg=k)


SCENARIOS = {
    "tiny_grid": lambda: S.tiny_grid(),
    "dense_small": lambda: S.random_small(seed=2, side=3, n_vehicles=150, T=150).copy(obs_every=40),
    "city_small": lambda: S.city_small(),
    "line": lambda: S.line_network(n_links=2, length=1500.0, u=13.9, kappa=0.2, q=0.5, N=700, T=900).copy(obs_every=70),
    "hub": lambda: S.hub(),          # an 11-way choice set: wider than the parallel slots
}


def test_executor_selection(Simulator):
    from paper_2603_25068_b300.native import SimError
    sc = S.city_small()
    g = Simulator(sc)
    assert g.executor == "persistent"
    g.set_executor("step")
    assert g.executor == "step"
    g.set_executor("auto")
    assert g.executor == "persistent"
    g.close()
    g = Simulator(sc, ckpt_every=30)          # records the reverse-pass tape: persistent too
    assert g.executor == "persistent"
    g.set_executor("step")
    assert g.executor == "step"
    g.close()
    from paper_2603_25068_b300.native import check
    g2 = Simulator(sc)
    with pytest.raises(SimError):
        check(g2.lib.sim_set_executor(g2.h, 7), g2.h)          # unknown executor
    g2.close()


@pytest.mark.parametrize("name", ["dense_small", "city_small"])
def test_checkpointed_rollout_and_gradient_match_step_executor(Simulator, name):
    # the checkpointed forward (one launch per segment) and the recording
    # recomputation of the reverse pass, persistent vs two-kernel executor
    sc = SCENARIOS[name]()
    res = {}
    for ex in ("step", "persistent"):
        g = Simulator(sc, ckpt_every=17, route_cap=64)
        g.set_executor(ex)
        out = g.rollout(sc.T)
        rng = np.random.default_rng(3)
        yb = rng.normal(size=out["counts"].shape).astype(np.float32)
        res[ex] = (out, g.backward(yb))
        g.close()
    (oa, ga), (ob, gb) = res["step"], res["persistent"]
    for k in OUT_KEYS:
        np.testing.assert_array_equal(oa[k], ob[k], err_msg=k)
    for k in ga:
        scale = np.max(np.abs(ga[k])) + 1e-30
        assert np.max(np.abs(ga[k].astype(np.float64) - gb[k])) <= 1e-6 * scale, k


@pytest.mark.parametrize("name", sorted(SCENARIOS))
def test_persistent_matches_step_executor(Simulator, name):
    sc = SCENARIOS[name]()
    a = run(Simulator, sc, sc.T, "step")
    b = run(Simulator, sc, sc.T, "persistent")
    assert (a["executor"], b["executor"]) == ("step", "persistent")
    assert_same(a, b)


@pytest.mark.parametrize("name", ["tiny_grid", "city_small"])
def test_runs_split_into_launches(Simulator, name):
    # sim_step in uneven pieces (each piece one launch, the first step of each
    # reading the vacancy flags written by the previous launch), also with the
    # executors alternating, equals one whole-run launch
    sc = SCENARIOS[name]()
    T = sc.T
    whole = run(Simulator, sc, T, "persistent")
    pieces = [1, 7, 33, 2, 60]
    pieces.append(T - sum(pieces))
    split = run(Simulator, sc, T, "persistent", chunks=pieces)
    assert_same(whole, split)
    g = Simulator(sc)
    g.reset(T)
    for i, c in enumerate(pieces):
        g.set_executor("persistent" if i % 2 == 0 else "step")
        g.step(c)
    mixed = dict(out=g.outputs(), state=g.state(), rec=g.records())
    g.close()
    assert_same(whole, mixed)


def test_lockstep_against_oracle_in_multi_step_launches(Simulator):
    # launches of 10 steps: steps after the first of a launch derive the
    # vacancy of other CTAs' links from their records and the merge words
    sc = S.random_small(seed=3, side=3, n_vehicles=150, T=150).copy(obs_every=40)
    g = Simulator(sc)
    g.set_executor("persistent")
    o = OracleSim(sc, "fp32")
    g.reset(150)
    o.reset(150)
    for _ in range(15):
        g.step(10)
        o.step(10)
        gs, os_ = g.state(), o.state()
        for k in ("veh_link", "veh_rank", "link_credit", "link_exits", "fifo_off", "veh_pos"):
            np.testing.assert_array_equal(gs[k], os_[k], err_msg=k)
    go, oo = g.outputs(), o.outputs()
    np.testing.assert_array_equal(go["counts"], oo["counts"])
    np.testing.assert_array_equal(go["n_on"], oo["n_on"])
    g.close()


def test_queue_longer_than_a_chunk(Simulator):
    # more than 4096 vehicles queued on one link: the car-following update of
    # one CTA runs in several chunks whose boundary headway is carried over
    sc = S.line_network(n_links=2, length=12000.0, u=13.9, kappa=0.5, q=0.02, N=5200, T=5600)
    g = Simulator(sc)
    g.set_executor("persistent")
    o = OracleSim(sc, "fp32")
    g.reset(sc.T)
    o.reset(sc.T)
    peak = 0
    for _ in range(sc.T // 700):
        g.step(700)
        o.step(700)
        gs, os_ = g.state(), o.state()
        peak = max(peak, int(np.max(np.bincount(gs["veh_link"][gs["veh_link"] >= 0], minlength=sc.L))))
        for k in ("veh_link", "veh_rank", "link_credit", "link_exits", "veh_pos"):
            np.testing.assert_array_equal(gs[k], os_[k], err_msg=k)
    assert peak > 4096
    np.testing.assert_array_equal(g.outputs()["counts"], o.outputs()["counts"])
    g.close()


def test_city_full_size_executors_agree(Simulator):
    # 36,000 links and 1,000,000 vehicles, first 900 steps: every output and
    # every piece of state identical between the executors
    sc = S.city().copy(T=900)
    a = run(Simulator, sc, 900, "step")
    b = run(Simulator, sc, 900, "persistent")
    assert_same(a, b)
    assert a["out"]["n_on"][-1] > 100_000


def test_bounded_barrier_wait_reports_timeout_and_recovers(Simulator):
    # the wait runs out (arrivals that never come), no fault: SIM_ETIMEOUT,
    # then the same handle and the device work normally after a reset
    import time
    from paper_2603_25068_b300.native import SimError, SIM_ETIMEOUT, check
    sc = S.tiny_grid()
    ref = run(Simulator, sc, sc.T, "persistent")
    g = Simulator(sc)
    check(g.lib.sim_test_barrier_timeout(g.h, 1), g.h)
    t0 = time.perf_counter()
    with pytest.raises(SimError) as e:
        g.rollout(sc.T)
    assert e.value.code == SIM_ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    out = g.rollout(sc.T)                      # reset by the rollout: a normal run again
    for k in OUT_KEYS:
        np.testing.assert_array_equal(out[k], ref["out"][k], err_msg=k)
    g.close()


def test_partition_weights_leave_results_unchanged(Simulator):
    # which CTA owns which links must not change any result: equal-capacity
    # groups, random weights and one heavy link give bit-identical runs
    from paper_2603_25068_b300.native import SimError
    sc = S.city_small()
    base = run(Simulator, sc, sc.T, "persistent")
    g = Simulator(sc)
    b0 = g.persist_groups()
    assert b0[0] == 0 and b0[-1] == sc.L and np.all(np.diff(b0) >= 0)
    rng = np.random.default_rng(4)
    w_heavy = np.ones(sc.L)
    w_heavy[sc.L // 2] = 500.0
    seen = {tuple(b0)}
    for w in (rng.uniform(0.0, 10.0, sc.L), rng.lognormal(0.0, 2.0, sc.L), w_heavy):
        g.set_partition_weights(w)
        b = g.persist_groups()
        assert b[0] == 0 and b[-1] == sc.L and np.all(np.diff(b) >= 0)
        seen.add(tuple(b))
        out = g.rollout(sc.T)
        res = dict(out=out, state=g.state(), rec=g.records())
        assert_same(base, res)
    assert len(seen) > 1, "the weights never moved a group bound"
    for bad in (np.full(sc.L, -1.0), np.zeros(sc.L), np.full(sc.L, np.nan)):
        with pytest.raises(SimError):
            g.set_partition_weights(bad)
    with pytest.raises(ValueError):
        g.set_partition_weights(np.ones(sc.L + 1))
    g.set_partition_weights(None)
    np.testing.assert_array_equal(g.persist_groups(), b0)
    g.close()
