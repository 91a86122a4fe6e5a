"""Batched execution: every member of a batch gives bitwise the same outputs and
state as when it runs alone, whatever its size, horizon or start step, with
either batch executor (one cooperative launch per advance, or one launch per
phase and step).  The batch kernels carry their own node-model and transfer
code, so each member is also compared with the oracle directly: state and
counts bitwise against its float build, speeds and travel times to 1e-4 and
1e-6 relative, gradients against its reverse mode (gradcheck.py)."""
import numpy as np
import pytest

from gradcheck import compare_grads
from oracle.oracle import OracleSim
from paper_2603_25068_b300 import scenario as S


def _oracle_equal(sc, T, out, st):
    o = OracleSim(sc, "fp32")
    ref = o.rollout(T)
    np.testing.assert_array_equal(out["counts"], ref["counts"], err_msg=sc.name)
    for k in ("n_waiting", "n_on", "n_arrived"):
        if k in out:
            np.testing.assert_array_equal(out[k], ref[k][:T + 1], err_msg=k)
    np.testing.assert_allclose(out["travel_time"], ref["travel_time"], rtol=1e-6, atol=0)
    np.testing.assert_allclose(out["speed"], ref["speed"], rtol=1e-4, atol=1e-5)
    ost = o.state()
    for k in ("veh_link", "veh_rank", "link_credit", "link_exits", "fifo_off", "veh_pos"):
        np.testing.assert_array_equal(st[k], ost[k], err_msg=f"{sc.name} {k}")

pytestmark = pytest.mark.gpu


def _solo(sc, T):
    from paper_2603_25068_b300.sim import Simulator
    g = Simulator(sc)
    out = g.rollout(T)
    return out, g.state()


def _same(a, b):
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


EXECUTORS = ["persistent", "step"]


def _batch(sims, executor):
    from paper_2603_25068_b300.batch import Batch
    b = Batch(sims)
    b.set_executor(executor)
    assert b.executor == executor
    return b


@pytest.mark.parametrize("executor", EXECUTORS)
def test_batch_rollout_equals_solo(executor):
    from paper_2603_25068_b300.batch import Batch
    from paper_2603_25068_b300.sim import Simulator
    scs = S.batched_scenarios(n=5, n_min=2000, n_max=15000, n_perturbed=100, T=400,
                              n_nodes=400, n_links=1200, n_vehicles=20000, n_origin_zones=8, n_dest_zones=12)
    sims = [Simulator(sc) for sc in scs]
    with _batch(sims, executor) as b:
        outs = b.rollout(400)
        states = [s.state() for s in sims]
    for sc, o, st in zip(scs, outs, states):
        ref, rst = _solo(sc, 400)
        _same(o, ref)
        _same(st, rst)


@pytest.mark.parametrize("executor", EXECUTORS)
def test_continuous_batching_staggered_members_equal_solo(executor):
    """Members with different networks, horizons and start steps."""
    from paper_2603_25068_b300.batch import Batch
    from paper_2603_25068_b300.sim import Simulator
    scs = [S.tiny_grid(T=250), S.city_small(T=300), S.random_small(seed=2, n_vehicles=120, T=170).copy(obs_every=40),
           S.city_small(seed=12, n_vehicles=8000, T=200)]
    Ts = [250, 300, 170, 200]
    sims = [Simulator(sc) for sc in scs]
    with _batch(sims, executor) as b:
        b.start(0, Ts[0])
        b.advance(37)
        b.start(1, Ts[1])
        b.advance(10)
        b.start(2, Ts[2])
        fin = b.advance(100)
        b.start(3, Ts[3])
        for _ in range(40):
            fin = b.advance(13)
            if fin.all():
                break
        assert fin.all()
        outs = [s.outputs() for s in sims]
        states = [s.state() for s in sims]
    for sc, T, o, st in zip(scs, Ts, outs, states):
        ref, rst = _solo(sc, T)
        _same(o, ref)
        _same(st, rst)
        _oracle_equal(sc, T, o, st)


@pytest.mark.parametrize("executor", EXECUTORS)
def test_batched_member_reverse_pass_equals_solo(executor):
    from paper_2603_25068_b300.batch import Batch
    from paper_2603_25068_b300.sim import Simulator
    scs = [S.random_small(seed=s, side=3, n_vehicles=160, T=90).copy(obs_every=30) for s in (1, 2, 3)]
    rng = np.random.default_rng(0)
    ybar = [rng.normal(size=(3, sc.L)).astype(np.float32) for sc in scs]
    sims = [Simulator(sc, ckpt_every=13) for sc in scs]
    with _batch(sims, executor) as b:
        b.rollout(90)
        gb = [s.backward(y) for s, y in zip(sims, ybar)]
    for sc, y, g in zip(scs, ybar, gb):
        solo = Simulator(sc, ckpt_every=13)
        solo.rollout()
        gs = solo.backward(y)
        for k in g:
            np.testing.assert_array_equal(g[k], gs[k], err_msg=k)
        o = OracleSim(sc, "fp32", keep_history=True)
        o.rollout()
        compare_grads(g, o.backward(y.astype(np.float64)))


@pytest.mark.parametrize("executor", EXECUTORS)
def test_staggered_checkpointed_members_reverse_pass_equals_solo(executor):
    """Members recording checkpoints join at different steps and advance in
    uneven pieces, so checkpoint steps fall anywhere inside a launch."""
    from paper_2603_25068_b300.sim import Simulator
    scs = [S.random_small(seed=s, side=3, n_vehicles=140, T=70 + 11 * s).copy(obs_every=20) for s in (4, 5, 6)]
    Ts = [sc.T for sc in scs]
    rng = np.random.default_rng(1)
    sims = [Simulator(sc, ckpt_every=9) for sc in scs]
    with _batch(sims, executor) as b:
        b.start(0, Ts[0])
        b.advance(5)
        b.start(1, Ts[1])
        b.advance(17)
        b.start(2, Ts[2])
        for n in (3, 31, 8, 64, 64):
            fin = b.advance(n)
        assert fin.all()
        outs = [s.outputs() for s in sims]             # before the reverse passes consume the runs
        ybar = [rng.normal(size=o["counts"].shape).astype(np.float32) for o in outs]
        gb = [s.backward(y) for s, y in zip(sims, ybar)]
    for sc, T, y, g, o in zip(scs, Ts, ybar, gb, outs):
        solo = Simulator(sc, ckpt_every=9)
        ref = solo.rollout(T)
        _same(o, ref)
        gs = solo.backward(y)
        for k in g:
            np.testing.assert_array_equal(g[k], gs[k], err_msg=k)


def test_persistent_batch_barrier_timeout_is_reported_and_recoverable():
    """The bounded grid-barrier wait of the persistent batch runs out (a test
    hook makes every barrier wait for arrivals that never come); the advance
    reports SIM_ETIMEOUT, and restarted members run correctly afterwards."""
    from paper_2603_25068_b300 import native as nat
    from paper_2603_25068_b300.sim import Simulator
    scs = [S.tiny_grid(T=60), S.random_small(seed=3, n_vehicles=100, T=60)]
    sims = [Simulator(sc) for sc in scs]
    with _batch(sims, "persistent") as b:
        for k in range(2):
            b.start(k, 60)
        nat.check(b.lib.sim_batch_test_barrier_timeout(b.h, 1), None)
        with pytest.raises(nat.SimError) as ei:
            b.advance(10)
        assert ei.value.code == nat.SIM_ETIMEOUT
        outs = b.rollout(60)                   # restarts every member
    for sc, o in zip(scs, outs):
        ref, _ = _solo(sc, 60)
        _same(o, ref)
