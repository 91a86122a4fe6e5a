"""Paper-mode parameterisation end to end (Methods, experimental setting):
per-link u, kappa, beta, alpha on a Sioux-Falls-shaped synthetic network,
noisy observations on 80 % of the links; gradients and one calibration step
against the oracle."""
import numpy as np
import pytest

from oracle.optim import AdamW, LR, WEIGHT_DECAY, calibration_loss
from oracle.oracle import OracleSim
from paper_2603_25068_b300 import scenario as S

pytestmark = pytest.mark.gpu
LINK = ("u", "kappa", "beta", "alpha")


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available()
    from paper_2603_25068_b300 import optimize
    from paper_2603_25068_b300.sim import Simulator
    return Simulator, optimize


def _problem():
    # the paper's shape at a size the oracle runs in seconds
    model, truth = S.paper_mode(n_vehicles=4000, T=600, dep_window=600)
    observed = S.noisy_counts(OracleSim(truth, "fp32").rollout()["counts"][:, model.sensors],
                              np.random.default_rng(1))
    return model, observed


def test_paper_mode_gradients_match_oracle(env):
    Simulator, _ = env
    model, observed = _problem()
    g = Simulator(model, ckpt_every=60, route_cap=64)
    out = g.rollout()
    o = OracleSim(model, "fp32", keep_history=True)
    oc = o.rollout()["counts"]
    np.testing.assert_array_equal(out["counts"], oc)
    _, ybar = calibration_loss(oc, observed, model.sensors)
    gg = g.backward(ybar.astype(np.float32))
    go = o.backward(ybar)
    # 1e-4 of each parameter's largest gradient (the FP32 tolerance of the
    # path): the destination term puts the choice keys near -80, where the
    # float32 keys carry ~1e-5 relative error into the softmax weights, and the
    # choice adjoint sums terms that cancel (measured: 7e-5 on two beta entries)
    for k in LINK + ("alpha_origin", "cost"):
        scale = max(np.abs(go[k]).max(), 1e-6)
        np.testing.assert_allclose(gg[k], go[k], rtol=0, atol=1e-4 * scale, err_msg=k)
    for k in LINK:
        assert np.count_nonzero(go[k]) > model.L // 4, k        # the four parameters all get gradients
    g.close()


def test_paper_mode_calibration_step_matches_oracle(env):
    # the optimiser works on z = (theta - lo) / (hi - lo): dL/dz = (hi - lo) dL/dtheta
    Simulator, optimize = env
    model, observed = _problem()
    sim = Simulator(model, ckpt_every=60, route_cap=64)
    res = optimize.calibrate_ranges(sim, observed, model.sensors, S.PAPER_RANGES, max_iter=1)
    o = OracleSim(model, "fp32", keep_history=True)
    loss, ybar = calibration_loss(o.rollout()["counts"], observed, model.sensors)
    assert res["losses"][0] == pytest.approx(loss, rel=1e-6)
    go = o.backward(ybar)
    for k in LINK:
        lo, hi = S.PAPER_RANGES[k]
        z0 = (getattr(model, k).astype(np.float64) - lo) / (hi - lo)
        gz = go[k] * (hi - lo)
        want = np.clip(AdamW().step(z0, gz), 0.0, 1.0)
        got = (res["last_params"][k].astype(np.float64) - lo) / (hi - lo)
        big = np.abs(gz) > 1e-4 * max(np.abs(gz).max(), 1e-30)
        np.testing.assert_allclose(got[big], want[big], rtol=0, atol=2e-5, err_msg=k)
        assert np.all(np.abs(got - z0) <= LR * (1.0 + WEIGHT_DECAY) + 1e-5), k
    sim.close()
