"""sim_set_state: continuing a run from a given state, as the lockstep protocol
does after a flagged near-tie (copy the oracle's state into the GPU and go on).
The continuation must equal the oracle's own continuation bit for bit."""
import numpy as np
import pytest

from oracle.oracle import OracleSim
from paper_2603_25068_b300 import scenario as S

pytestmark = pytest.mark.gpu

KEYS = ("veh_link", "veh_rank", "veh_pos", "link_credit", "link_exits", "fifo_off")


@pytest.fixture(scope="module")
def Simulator():
    import torch
    assert torch.cuda.is_available()
    from paper_2603_25068_b300.sim import Simulator
    return Simulator


def assert_state(a, b):
    for k in KEYS:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    on = a["veh_link"] >= 0
    np.testing.assert_array_equal(a["veh_entry"][on], b["veh_entry"][on])


@pytest.mark.parametrize("executor", ["persistent", "step"])
@pytest.mark.parametrize("t0", [40, 97])
def test_oracle_state_continues_in_lockstep(Simulator, executor, t0):
    sc = S.random_small(seed=2, side=3, n_vehicles=150, T=150).copy(obs_every=40)
    o = OracleSim(sc, "fp32")
    o.reset(sc.T)
    o.step(t0)
    g = Simulator(sc)
    g.set_executor(executor)
    g.reset(sc.T)
    g.set_state(o.state(), t0)
    assert g.t == t0
    for _ in range(3):                         # a few uneven pieces
        n = min(23, sc.T - g.t)
        g.step(n)
        o.step(n)
        assert_state(g.state(), o.state())
    g.step(sc.T - g.t)
    o.step(sc.T - o.t)
    assert_state(g.state(), o.state())
    # bins that start at or after t0 are whole in the continuation
    first = -(-t0 // sc.obs_every)
    np.testing.assert_array_equal(g.outputs()["counts"][first:], o.outputs()["counts"][first:])
    g.close()


def test_gpu_state_roundtrip(Simulator):
    sc = S.city_small()
    a = Simulator(sc)
    a.reset(sc.T)
    a.step(137)
    st = a.state()
    b = Simulator(sc)
    b.reset(sc.T)
    b.set_state(st, 137)
    assert_state(b.state(), st)
    a.step(sc.T - 137)
    b.step(sc.T - 137)
    assert_state(a.state(), b.state())
    a.close()
    b.close()


def test_set_state_rejects_inconsistent_states(Simulator):
    from paper_2603_25068_b300.native import SimError
    sc = S.tiny_grid()
    g = Simulator(sc)
    g.reset(sc.T)
    g.step(60)
    st = g.state()
    on = np.nonzero(st["veh_link"] >= 0)[0]
    assert len(on) >= 2
    bad = {k: v.copy() for k, v in st.items()}
    bad["veh_pos"][on[0]] = 1e6                                     # outside its link
    with pytest.raises(SimError):
        g.set_state(bad, 60)
    bad = {k: v.copy() for k, v in st.items()}
    same = on[st["veh_link"][on] == st["veh_link"][on[0]]]
    if len(same) >= 2:                                              # two vehicles with one rank
        bad["veh_rank"][same[1]] = bad["veh_rank"][same[0]]
        with pytest.raises(SimError):
            g.set_state(bad, 60)
    bad = {k: v.copy() for k, v in st.items()}
    bad["veh_link"][on[0]] = -1                                     # waiting, but its queue released it
    with pytest.raises(SimError):
        g.set_state(bad, 60)
    with pytest.raises(SimError):
        g.set_state(st, sc.T + 1)                                   # outside the horizon
    g.set_state(st, 60)                                             # the state itself is accepted
    g.close()


def test_release_cached_memory_and_recompute_mode_validation(Simulator):
    """Cached pool memory can be returned to the driver between runs (live
    simulators keep theirs); unknown recompute modes are refused."""
    from paper_2603_25068_b300 import native as nat
    sc = S.tiny_grid(T=60)
    a = Simulator(sc)
    ref = a.rollout(60)
    lib = nat.lib()
    nat.check(lib.sim_release_cached_memory(0), None)
    assert lib.sim_release_cached_memory(-1) == nat.SIM_EINVAL
    again = a.rollout(60)                          # the live simulator's memory is untouched
    for k in ("counts", "speed", "travel_time"):
        np.testing.assert_array_equal(again[k], ref[k])
    assert lib.sim_set_recompute(a.h, 7) == nat.SIM_EINVAL
    a.close()
    b = Simulator(sc)                              # allocations after a release
    np.testing.assert_array_equal(b.rollout(60)["counts"], ref["counts"])
    b.close()
