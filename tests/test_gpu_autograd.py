"""torch.autograd.Function over the C ABI: forward value and gradients equal the
library's rollout and reverse pass, and a few optimiser steps of the paper's
calibration loop (AdamW, lr 0.1, weight decay 1e-5) run end to end on device."""
import numpy as np
import pytest

from paper_2603_25068_b300 import scenario as S

pytestmark = pytest.mark.gpu


def _params(sc, dev):
    import torch
    t = lambda a: torch.tensor(np.asarray(a, np.float32), device=dev, requires_grad=True)
    return dict(u=t(sc.u), kappa=t(sc.kappa), alpha=t(sc.alpha), beta=t(sc.beta), cost=t(sc.cost), w=t(sc.w),
                alpha_origin=torch.tensor(float(sc.alpha_origin), device=dev, requires_grad=True),
                od_lambda=t(sc.od_lambda))


def test_autograd_matches_library():
    import torch
    from paper_2603_25068_b300.autograd import PARAMS, rollout_counts
    from paper_2603_25068_b300.sim import Simulator
    dev = torch.device("cuda", 0)
    sc = S.random_small(seed=2, side=3, n_vehicles=160, T=90).copy(obs_every=30)
    sim = Simulator(sc, ckpt_every=30)
    p = _params(sc, dev)
    counts = rollout_counts(sim, **p)
    ref = Simulator(sc).rollout()["counts"]
    np.testing.assert_array_equal(counts.detach().cpu().numpy(), ref)
    g_out = torch.randn_like(counts)
    counts.backward(g_out)
    sim2 = Simulator(sc, ckpt_every=30)
    sim2.rollout()
    g = sim2.backward(g_out.cpu().numpy())
    for k in PARAMS:
        np.testing.assert_allclose(p[k].grad.detach().cpu().numpy().reshape(-1), g[k].reshape(-1),
                                   rtol=1e-5, atol=1e-6 * max(1.0, np.abs(g[k]).max()), err_msg=k)


def test_calibration_loop_runs_on_device():
    import torch
    from paper_2603_25068_b300.autograd import rollout_counts
    from paper_2603_25068_b300.sim import Simulator
    dev = torch.device("cuda", 0)
    model, truth = S.calibration(n_sensors=400, n_nodes=300, n_links=900, n_vehicles=15000, T=600,
                                 n_origin_zones=6, n_dest_zones=10)
    sens = torch.tensor(model.sensors, device=dev, dtype=torch.long)
    y_obs = torch.tensor(Simulator(truth).rollout()["counts"], device=dev, dtype=torch.float32)[:, sens]
    sim = Simulator(model, ckpt_every=60, route_cap=128)
    w = torch.tensor(model.w, device=dev, requires_grad=True)
    lam = torch.tensor(model.od_lambda, device=dev, requires_grad=True)
    fixed = {k: torch.tensor(np.asarray(getattr(model, k), np.float32), device=dev)
             for k in ("u", "kappa", "alpha", "beta", "cost")}
    opt = torch.optim.AdamW([w, lam], lr=1e-1, weight_decay=1e-5)
    losses = []
    for _ in range(3):
        opt.zero_grad()
        counts = rollout_counts(sim, fixed["u"], fixed["kappa"], fixed["alpha"], fixed["beta"], fixed["cost"],
                                w, model.alpha_origin, lam)
        loss = ((counts[:, sens] - y_obs) ** 2).mean()
        loss.backward()
        assert torch.isfinite(w.grad).all() and torch.isfinite(lam.grad).all()
        assert w.grad.abs().sum() > 0
        opt.step()
        with torch.no_grad():
            lam.clamp_(min=1e-3)
        losses.append(float(loss))
    assert all(np.isfinite(losses))


def test_device_parameters_equal_host_parameters_and_are_validated():
    """sim_set_params_device (parameters in device memory, no host round trip)
    gives the rollout of sim_set_params with the same values; an invalid
    device parameter is reported by the next synchronous call."""
    import torch
    from paper_2603_25068_b300.native import SimError, SIM_EINVAL
    from paper_2603_25068_b300.sim import Simulator
    dev = torch.device("cuda", 0)
    sc = S.random_small(seed=3, side=3, n_vehicles=160, T=90).copy(obs_every=30)
    rng = np.random.default_rng(4)
    new = dict(u=(sc.u * rng.uniform(0.8, 1.2, sc.L)).astype(np.float32),
               kappa=(sc.kappa * rng.uniform(0.9, 1.0, sc.L)).astype(np.float32),
               alpha=rng.uniform(0.5, 4.0, sc.L).astype(np.float32), beta=rng.uniform(0, 2, sc.L).astype(np.float32),
               cost=rng.uniform(0.5, 2.0, sc.L).astype(np.float32), w=(sc.w + 0.3).astype(np.float32))
    host = Simulator(sc)
    host.set_params(alpha_origin=1.7, **new)
    ref = host.rollout()
    devsim = Simulator(sc)
    t = {k: torch.tensor(v, device=dev) for k, v in new.items()}
    devsim.set_params_device(t["u"], t["kappa"], t["alpha"], t["beta"], t["cost"], t["w"],
                             torch.tensor([1.7], device=dev))
    got = devsim.rollout()
    for k in ("counts", "speed", "travel_time", "n_arrived"):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
    bad = t["u"].clone()
    bad[3] = -1.0
    devsim.set_params_device(bad, t["kappa"], t["alpha"], t["beta"], t["cost"], t["w"], torch.tensor([1.7], device=dev))
    with pytest.raises(SimError) as e:
        devsim.rollout()
    assert e.value.code == SIM_EINVAL
    devsim.set_params_device(t["u"], t["kappa"], t["alpha"], t["beta"], t["cost"], t["w"],
                             torch.tensor([1.7], device=dev))
    np.testing.assert_array_equal(devsim.rollout()["counts"], ref["counts"])
    host.close()
    devsim.close()
