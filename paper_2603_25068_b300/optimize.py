"""Gradient-based calibration and control (Methods, Optimization).

Each iteration runs the forward simulation, the loss, the reverse pass
(`sim_backward` through `rollout_counts`) and an AdamW update with learning
rate 1e-1 and weight decay 1e-5 (other hyperparameters at their defaults).
The loop ends once the loss has not improved over the last 20 iterations,
and the parameters of the lowest loss are returned.

    res = calibrate(sim, observed, sensors)                # demand + route choice
    res = control(sim, target_link)                        # link costs, halve its count

Losses:
  * calibration: mean squared error of the simulated counts on the observed
    links (every bin);
  * control (Results, gradient-guided traffic control): squared error between
    the goal (a fraction, by default half, of the target link's cumulative
    count without control) and its simulated cumulative count.

The parameters live on the simulator's device as torch tensors; the
simulation and its reverse pass run in the library's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from .autograd import rollout_counts

LR, WEIGHT_DECAY, PATIENCE = 1e-1, 1e-5, 20
LINK_PARAMS = ("u", "kappa", "alpha", "beta", "cost")


def initial_params(sim):
    """The scenario's parameters as float32 tensors on the simulator's device."""
    dev = torch.device("cuda", sim.device)
    sc = sim.sc
    p = {k: torch.tensor(np.asarray(getattr(sc, k), np.float32), device=dev) for k in LINK_PARAMS + ("w",)}
    p["alpha_origin"] = torch.tensor(float(sc.alpha_origin), device=dev)
    p["od_lambda"] = torch.tensor(np.asarray(sc.od_lambda, np.float32), device=dev)
    return p


def run(sim, loss_fn, names, params=None, max_iter=200, patience=PATIENCE, lr=LR, weight_decay=WEIGHT_DECAY,
        project=None, T=None, transform=None):
    """The loop for the parameters in `names`.  loss_fn(counts) -> scalar
    tensor, counts [n_bins, L] float32 on the device.  project(params), if
    given, restores bounds after each update (in place, no gradient).
    transform(params), if given, maps the trained tensors to the simulator's
    parameters (differentiably) before each rollout.
    Returns a dict: best_loss, best_iter, iterations, losses (per iteration),
    params (host copies of the named simulator parameters at the best
    iteration) and last_params (the same after the last update)."""
    p = initial_params(sim) if params is None else params
    tf = transform if transform is not None else (lambda x: x)
    train = [p[k] for k in names]
    for t in train:
        t.requires_grad_(True)
    opt = torch.optim.AdamW(train, lr=lr, weight_decay=weight_decay)
    best, best_iter, best_params, losses = float("inf"), -1, None, []
    for it in range(max_iter):
        opt.zero_grad(set_to_none=True)
        q = tf(p)
        counts = rollout_counts(sim, q["u"], q["kappa"], q["alpha"], q["beta"], q["cost"], q["w"],
                                q["alpha_origin"], q["od_lambda"], T=T)
        loss = loss_fn(counts)
        loss.backward()
        lv = float(loss.detach())
        losses.append(lv)
        if lv < best:
            best, best_iter = lv, it
            best_params = {k: q[k].detach().cpu().numpy().copy() for k in names}
        if it - best_iter >= patience:
            break
        opt.step()
        if project is not None:
            with torch.no_grad():
                project(p)
    last = tf(p)
    return {"best_loss": best, "best_iter": best_iter, "iterations": len(losses), "losses": losses,
            "params": best_params, "last_params": {k: last[k].detach().cpu().numpy().copy() for k in names}}


def calibrate(sim, observed, sensors, names=("w", "od_lambda"), lambda_min=1e-3, **kw):
    """Calibration against observed counts [n_bins, len(sensors)] on the links
    `sensors`.  Demand parameters are kept >= lambda_min."""
    dev = torch.device("cuda", sim.device)
    obs = torch.as_tensor(np.asarray(observed), dtype=torch.float32, device=dev)
    sens = torch.as_tensor(np.asarray(sensors), dtype=torch.long, device=dev)

    def loss_fn(counts):
        return ((counts[:, sens] - obs) ** 2).mean()

    def project(p):
        if "od_lambda" in p:
            p["od_lambda"].clamp_(min=lambda_min)

    return run(sim, loss_fn, names, project=project, **kw)


def control(sim, target, goal_fraction=0.5, baseline=None, names=("cost",), cost_min=1e-2, **kw):
    """Link-cost control: bring the target link's cumulative count to
    goal_fraction of its count without control (`baseline`, simulated when not
    given).  Costs are kept >= cost_min.  The result also holds the goal and
    the baseline."""
    if baseline is None:
        baseline = float(sim.rollout(kw.get("T"))["counts"][:, target].sum())
    goal = goal_fraction * baseline

    def loss_fn(counts):
        return (counts[:, target].sum() - goal) ** 2

    def project(p):
        p["cost"].clamp_(min=cost_min)

    res = run(sim, loss_fn, names, project=project, **kw)
    res.update(goal=goal, baseline=baseline)
    return res


def range_simulator(model, ranges, **sim_kw):
    """A simulator for calibrating within `ranges`: its queue rings are sized
    for the largest jam density of the range (the ring capacity is fixed when
    the simulator is created), and it starts at the model's parameters."""
    from .sim import Simulator
    sized = model
    if "kappa" in ranges:
        sized = model.copy(kappa=np.full(model.L, max(float(ranges["kappa"][1]), float(np.max(model.kappa))),
                                         np.float32))
    sim = Simulator(sized, **sim_kw)
    sim.sc = model
    sim.set_params()
    return sim


def calibrate_ranges(sim, observed, sensors, ranges, **kw):
    """Calibration of per-link parameters within given ranges ({name: (lo,
    hi)}, e.g. the paper's u, kappa, beta, alpha ranges).  The optimiser works
    on z = (theta - lo) / (hi - lo), kept in [0, 1], so that the learning rate
    is a fraction of each range (a step of 0.1 moves a tenth of it); it starts
    from the simulator's current parameters.  The result's params are the
    simulator parameters theta."""
    p = initial_params(sim)
    lo = {k: float(r[0]) for k, r in ranges.items()}
    span = {k: float(r[1]) - float(r[0]) for k, r in ranges.items()}
    for k in ranges:
        p[k] = ((p[k] - lo[k]) / span[k]).clamp(0.0, 1.0)

    def transform(x):
        y = dict(x)
        for k in ranges:
            y[k] = lo[k] + span[k] * x[k]
        return y

    def project(x):
        for k in ranges:
            x[k].clamp_(0.0, 1.0)

    dev = torch.device("cuda", sim.device)
    obs = torch.as_tensor(np.asarray(observed), dtype=torch.float32, device=dev)
    sens = torch.as_tensor(np.asarray(sensors), dtype=torch.long, device=dev)

    def loss_fn(counts):
        return ((counts[:, sens] - obs) ** 2).mean()

    return run(sim, loss_fn, tuple(ranges), params=p, project=project, transform=transform, **kw)
