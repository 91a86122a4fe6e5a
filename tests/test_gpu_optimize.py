"""The calibration and control loops (Methods, Optimization) on the GPU
against the oracle's loop: the same loss, the same gradient and the same AdamW
step from the same parameters; and the loops' bookkeeping (best parameters,
early stop)."""
import numpy as np
import pytest

from oracle.optim import AdamW, LR, WEIGHT_DECAY, calibration_loss, control_loss
from oracle.oracle import OracleSim
from paper_2603_25068_b300 import scenario as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available()
    from paper_2603_25068_b300 import optimize
    from paper_2603_25068_b300.sim import Simulator
    return Simulator, optimize


def _calibration_problem():
    sc = S.random_small(seed=2, side=3, n_vehicles=150, T=150).copy(obs_every=30)
    truth = sc.copy(u=(sc.u * 0.8).astype(np.float32), beta=(sc.beta + 0.5).astype(np.float32))
    sensors = np.arange(0, sc.L, 2)
    observed = OracleSim(truth, "fp32").rollout()["counts"][:, sensors].astype(np.float64)
    return sc, observed, sensors


def _control_problem():
    # the busiest link of a small grid; its candidates compete at merges, which
    # is where the choice adjoint reaches the utilities beta / c
    sc = S.random_small(seed=2, side=3, n_vehicles=150, T=150).copy(obs_every=30)
    counts = OracleSim(sc, "fp32").rollout()["counts"]
    return sc, int(np.argmax(counts.sum(0))), counts


def _step_matches(theta0, got, want, grad):
    # AdamW's first step is lr (g / (|g| + eps) + wd theta): components whose
    # gradient is not tiny must agree; the others moved by at most one step
    big = np.abs(grad) > 1e-4 * max(np.abs(grad).max(), 1e-30)
    np.testing.assert_allclose(got[big], want[big], rtol=0, atol=1e-5)
    bound = LR * (1.0 + WEIGHT_DECAY * np.abs(theta0)) + 1e-6 * (1.0 + np.abs(theta0))   # float32 rounding
    assert np.all(np.abs(got - theta0) <= bound)


def test_one_calibration_iteration_matches_oracle_loop(env):
    Simulator, optimize = env
    sc, observed, sensors = _calibration_problem()
    names = ("w", "u", "beta", "od_lambda")
    sim = Simulator(sc, ckpt_every=30, route_cap=64)
    p = optimize.initial_params(sim)
    theta0 = {k: p[k].detach().cpu().numpy().astype(np.float64) for k in names}
    res = optimize.calibrate(sim, observed, sensors, names=names, params=p, max_iter=1)
    o = OracleSim(sc, "fp32", keep_history=True)
    loss, ybar = calibration_loss(o.rollout()["counts"], observed, sensors)
    assert res["losses"][0] == pytest.approx(loss, rel=1e-6)
    g = o.backward(ybar)
    for k in names:
        want = AdamW().step(theta0[k], g[k])
        _step_matches(theta0[k], p[k].detach().cpu().numpy().astype(np.float64), want, g[k])
    sim.close()


def test_one_control_iteration_matches_oracle_loop(env):
    Simulator, optimize = env
    sc, target, counts = _control_problem()
    sim = Simulator(sc, ckpt_every=30, route_cap=64)
    p = optimize.initial_params(sim)
    c0 = p["cost"].detach().cpu().numpy().astype(np.float64)
    baseline = float(counts[:, target].sum())
    res = optimize.control(sim, target, baseline=baseline, params=p, max_iter=1)
    loss, ybar = control_loss(counts, target, 0.5 * baseline)
    assert res["losses"][0] == pytest.approx(loss, rel=1e-6)
    o = OracleSim(sc, "fp32", keep_history=True)
    o.rollout()
    g = o.backward(ybar)
    assert g["cost"][target] < 0         # a dearer target link draws fewer vehicles
    _step_matches(c0, p["cost"].detach().cpu().numpy().astype(np.float64), AdamW().step(c0, g["cost"]), g["cost"])
    sim.close()


def test_calibration_loop_improves_and_keeps_the_best(env):
    import torch
    from paper_2603_25068_b300.autograd import rollout_counts
    Simulator, optimize = env
    sc, observed, sensors = _calibration_problem()
    sim = Simulator(sc, ckpt_every=30, route_cap=64)
    res = optimize.calibrate(sim, observed, sensors, names=("w", "u", "beta"), max_iter=30, patience=8)
    assert res["best_loss"] < res["losses"][0]
    assert res["best_loss"] == min(res["losses"]) and res["losses"][res["best_iter"]] == res["best_loss"]
    n = res["iterations"]
    assert n == 30 or n - 1 - res["best_iter"] == 8          # stopped by the patience rule
    p = optimize.initial_params(sim)
    for k, v in res["params"].items():
        p[k] = torch.tensor(v, device=p[k].device)
    counts = rollout_counts(sim, p["u"], p["kappa"], p["alpha"], p["beta"], p["cost"], p["w"], p["alpha_origin"],
                            p["od_lambda"])
    sens = torch.as_tensor(sensors, device=counts.device)
    obs = torch.as_tensor(observed, dtype=torch.float32, device=counts.device)
    assert float(((counts[:, sens] - obs) ** 2).mean()) == pytest.approx(res["best_loss"], rel=1e-6)
    sim.close()


def test_control_loop_lowers_the_target_count(env):
    Simulator, optimize = env
    sc, target, counts = _control_problem()
    sim = Simulator(sc, ckpt_every=30, route_cap=64)
    res = optimize.control(sim, target, max_iter=30, patience=10)
    assert res["baseline"] == counts[:, target].sum()
    assert res["best_loss"] < res["losses"][0]
    sim.close()
