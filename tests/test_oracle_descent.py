"""The reverse pass's gradient against the expected loss it stands for.

The simulation draws Gumbel noise, so the loss of one run is piecewise
constant in the parameters; its expectation over the noise is smooth.  Along
the descent direction d of the surrogate gradient (averaged over seeds), a
central finite difference of the mean loss over the same seeds (common random
numbers) must fall as the surrogate predicts (Methods, Optimization: the
gradient steers the calibration).  Oracle only (fp64), a small paper-mode
problem."""
import numpy as np
import pytest

from oracle.optim import calibration_loss
from oracle.oracle import OracleSim
from paper_2603_25068_b300 import scenario as S

K = 24                       # seeds


@pytest.fixture(scope="module")
def problem():
    model, truth = S.paper_mode(n_vehicles=4000, T=600, dep_window=600)
    obs = S.noisy_counts(OracleSim(truth, "fp64").rollout()["counts"][:, model.sensors], np.random.default_rng(1))
    return model, obs


def _loss(sc, obs, grad):
    o = OracleSim(sc, "fp64", keep_history=grad)
    L, yb = calibration_loss(o.rollout()["counts"], obs, sc.sensors)
    return L, (o.backward(yb) if grad else None)


def _check(problem, name):
    model, obs = problem
    gbar = np.mean([_loss(model.copy(seed=100 + s), obs, True)[1][name] for s in range(K)], axis=0)
    d = -gbar / np.abs(gbar).max()
    lo, hi = S.PAPER_RANGES[name]
    eps = 0.02 * (hi - lo)
    p = getattr(model, name).astype(np.float64)
    fd = np.array([(_loss(model.copy(seed=100 + s, **{name: (p + eps * d).astype(np.float32)}), obs, False)[0]
                    - _loss(model.copy(seed=100 + s, **{name: (p - eps * d).astype(np.float32)}), obs, False)[0])
                   / (2 * eps) for s in range(K)])
    pred = float(gbar @ d)
    return pred, fd.mean(), fd.std() / np.sqrt(K)


@pytest.mark.parametrize("name", ["u", "kappa"])
def test_surrogate_gradient_descends_the_expected_loss(problem, name):
    pred, fd, se = _check(problem, name)
    assert pred < 0
    assert fd < -2.0 * se, (name, pred, fd, se)        # the loss falls along the surrogate's descent direction


@pytest.mark.xfail(strict=True, reason="the paper's straight-through merge surrogate (Eq. transfer carries "
                                       "the sentinel M into the merge adjoint) gives an alpha gradient that "
                                       "does not descend the expected loss on this problem (measured: "
                                       "+4.3 +- 1.1 along its descent direction)")
def test_merge_priority_gradient_descends_the_expected_loss(problem):
    pred, fd, se = _check(problem, "alpha")
    assert fd < -2.0 * se, (pred, fd, se)


# ---------------------------------------------------------------- calibration parameters
@pytest.fixture(scope="module")
def calibration_problem():
    """A small instance shaped like the calibration workload: a city-family
    network with the 16-feature route-choice utility and per-OD demand
    parameters, 1-minute bins on 150 sensor links, observations from a hidden
    route-choice draw w* = w + N(0, 0.5^2) with the same vehicles."""
    model = S.city(seed=21, n_nodes=150, n_links=450, n_vehicles=4000, T=600, n_origin_zones=6, n_dest_zones=8,
                   dep_window=300.0, name="calibration_small")
    rng = np.random.default_rng(2)
    truth = model.copy(w=(model.w + rng.normal(0.0, 0.5, size=model.F)).astype(np.float32))
    sens = np.sort(rng.choice(model.L, size=150, replace=False)).astype(np.int32)
    model, truth = model.copy(sensors=sens, obs_every=60), truth.copy(sensors=sens, obs_every=60)
    obs = OracleSim(truth, "fp64").rollout()["counts"][:, sens]
    return model, obs


def _check_free(problem, name, eps):
    model, obs = problem
    gbar = np.mean([_loss(model.copy(seed=100 + s), obs, True)[1][name] for s in range(K)], axis=0)
    d = -gbar / np.abs(gbar).max()
    p = getattr(model, name).astype(np.float64)
    fd = np.array([(_loss(model.copy(seed=100 + s, **{name: (p + eps * d).astype(np.float32)}), obs, False)[0]
                    - _loss(model.copy(seed=100 + s, **{name: (p - eps * d).astype(np.float32)}), obs, False)[0])
                   / (2 * eps) for s in range(K)])
    return float(gbar @ d), fd.mean(), fd.std() / np.sqrt(K)


def test_demand_parameters_do_not_enter_the_forward(calibration_problem):
    """The demand gradient is that of the straight-through demand weight
    1 + (lambda - sg lambda)/lambda (a reading: the paper does not
    differentiate demand): the simulated vehicles are the scenario's, so the
    loss itself does not change along any lambda direction while the
    surrogate predicts a descent."""
    model, _ = calibration_problem
    pred, fd, se = _check_free(calibration_problem, "od_lambda", 0.05 * float(np.abs(model.od_lambda).max()))
    assert pred < 0
    assert fd == 0.0 and se == 0.0


@pytest.mark.xfail(strict=True, reason="the route-choice gradient reaches w through the merge adjoint of the "
                                       "paper's straight-through surrogate (sentinel M in Eq. transfer), like "
                                       "alpha; on this problem the loss rises along its descent direction "
                                       "(measured: predicted -1.7e3, finite difference +36.5 +- 3.5)")
def test_route_choice_gradient_descends_the_expected_loss(calibration_problem):
    pred, fd, se = _check_free(calibration_problem, "w", 0.05)
    assert fd < -2.0 * se, (pred, fd, se)
