"""Pins of the oracle's reverse mode (no GPU).

* the trajectory-grafting toy of SI-C: closed-form gradient at the start and the
  gradient-descent result the paper prints (tests/golden/tg_toy.json);
* the dense literal formulation (SI-A Alg. S1, SI-B Alg. S2 on N x L tensors,
  torch autograd for jax.grad): same forward decisions, same gradients;
* central finite differences of the surrogate with every decision and every
  stop_gradient value frozen (the function the method differentiates)."""
import json
import os

import numpy as np
import pytest

from oracle import dense_ref
from oracle.oracle import OracleSim
from paper_2603_25068_b300 import scenario as S

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "tg_toy.json")))
KEYS = ("u", "kappa", "alpha", "alpha_origin", "beta", "cost", "w", "od_lambda")


def _toy_grad(u1, u2, no_tg, prec="fp64"):
    sc = S.tg_toy(u1, u2)
    o = OracleSim(sc, prec, keep_history=True)
    o.rollout()
    x = o.positions()
    link = o.state()["veh_link"][0]
    g = o.backward(np.zeros((1, sc.L)), xbarT=2 * x, no_tg=no_tg)
    return x[0], link, g["u"][:2]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tg_toy_closed_form_gradient(prec):
    cf = GOLD["closed_form_at_start"]
    x, link, g = _toy_grad(2.0, 1.0, False, prec)
    assert link == 1 and x == 2.0
    np.testing.assert_allclose(g, [cf["dloss_du1"], cf["dloss_du2"]], rtol=1e-12)
    _, _, g0 = _toy_grad(2.0, 1.0, True, prec)
    assert g0[0] == cf["dloss_du1_without_tg"] and g0[1] == cf["dloss_du2"]


@pytest.mark.parametrize("tg", [True, False])
def test_tg_toy_gradient_descent_reproduces_paper(tg):
    """SI-C: with TG the estimates approach the truth (1.5, ~0.9); without TG
    u1 stays at 2.0 and u2 collapses to 0."""
    u = np.array([2.0, 1.0])
    for _ in range(300):
        x, link, g = _toy_grad(u[0], u[1], not tg)
        u = np.maximum(u - 1e-2 * g, 1e-3)
    want = GOLD["printed_results"]["with_tg" if tg else "without_tg"]
    tol = GOLD["tolerance"]["u_abs"]
    assert abs(u[0] - want["u1"]) < tol and abs(u[1] - want["u2"]) < tol, u


CASES = [(1, 120, 80), (2, 160, 80), (7, 200, 100)]


@pytest.mark.parametrize("seed,nv,T", CASES)
def test_dense_formulation_matches_compact_oracle(seed, nv, T):
    sc = S.random_small(seed=seed, side=3, n_vehicles=nv, T=T).copy(obs_every=T // 3)
    rng = np.random.default_rng(seed)
    nb = (T + sc.obs_every - 1) // sc.obs_every
    ybar = rng.normal(size=(nb, sc.L))
    xbarT = rng.normal(size=sc.N)
    out, gd, _ = dense_ref.run(sc, ybar=ybar, xbarT=xbarT)
    o = OracleSim(sc, "fp64", keep_history=True)
    ref = o.rollout()
    np.testing.assert_array_equal(out["counts"], ref["counts"])
    st = o.state()
    np.testing.assert_array_equal(np.where(out["vlink"] == -1, -1, out["vlink"]), st["veh_link"])
    on = st["veh_link"] >= 0
    np.testing.assert_allclose(out["x_T"][on], st["veh_pos"][on], rtol=0, atol=1e-9)
    go = o.backward(ybar, xbarT=np.where(on, xbarT, 0.0))
    for k in KEYS:
        scale = max(1.0, np.abs(gd[k]).max())
        np.testing.assert_allclose(go[k], gd[k], rtol=0, atol=1e-10 * scale, err_msg=k)
    # the case exercises every parameter family
    for k in ("u", "kappa", "alpha", "beta", "cost", "w", "od_lambda"):
        assert np.count_nonzero(np.abs(gd[k]) > 1e-9) > 0, k


def test_finite_differences_of_frozen_surrogate():
    seed, nv, T = CASES[0]
    sc = S.random_small(seed=seed, side=3, n_vehicles=nv, T=T).copy(obs_every=T // 3)
    rng = np.random.default_rng(100)
    nb = (T + sc.obs_every - 1) // sc.obs_every
    ybar = rng.normal(size=(nb, sc.L))
    tape = dense_ref.Tape()
    dense_ref.run(sc, ybar=ybar, tape=tape)
    o = OracleSim(sc, "fp64", keep_history=True)
    o.rollout()
    go = o.backward(ybar)
    base = dict(u=sc.u, kappa=sc.kappa, alpha=sc.alpha, alpha_origin=np.array([np.float32(sc.alpha_origin)]),
                beta=sc.beta, cost=sc.cost, w=sc.w, od_lambda=sc.od_lambda)
    base = {k: np.asarray(v, np.float64).copy() for k, v in base.items()}

    def F(params):
        tape.rewind()
        return dense_ref.run(sc, ybar=ybar, tape=tape, params=params)[0]["loss"]

    def central(k, idx, h):
        p1 = {kk: v.copy() for kk, v in base.items()}
        p2 = {kk: v.copy() for kk, v in base.items()}
        p1[k][idx] += h
        p2[k][idx] -= h
        return (F(p1) - F(p2)) / (2 * h)

    checked = 0
    for k in KEYS:
        nz = np.nonzero(np.abs(go[k]) > 1e-6)[0]
        for idx in rng.permutation(nz)[:2]:
            h = 2e-6 * max(1.0, abs(base[k][idx]))
            # Richardson extrapolation of two central differences: error O(h^4)
            fd = (4.0 * central(k, idx, h / 2) - central(k, idx, h)) / 3.0
            assert abs(fd - go[k][idx]) <= 2e-6 * max(abs(go[k][idx]), 1e-3), (k, idx, fd, go[k][idx])
            checked += 1
    assert checked >= 12


def test_finite_differences_on_the_calibration_parameterisation():
    """The calibration workload's parameterisation (the 16-feature route-choice
    utility w, a demand parameter lambda per origin-destination pair, counts on
    sensor links) on a city-family network: Richardson-extrapolated central
    differences of the frozen surrogate (dense formulation, decisions and
    stop-gradient values replayed) against the compact oracle's reverse mode
    for 16 lambda (every one the loss reaches, up to 16) and all 16 w."""
    import torch
    sc = S.city(seed=31, n_nodes=40, n_links=120, n_vehicles=240, T=120, n_origin_zones=4, n_dest_zones=6,
                dep_window=60.0, name="calibration_tiny").copy(obs_every=40)
    assert sc.F == 16 and sc.n_od == 24
    rng = np.random.default_rng(100)
    nb = (sc.T + sc.obs_every - 1) // sc.obs_every
    sens = np.sort(rng.choice(sc.L, size=40, replace=False))
    ybar = np.zeros((nb, sc.L))
    ybar[:, sens] = rng.normal(size=(nb, len(sens)))
    tape = dense_ref.Tape()
    out, gd, _ = dense_ref.run(sc, ybar=ybar, tape=tape)
    o = OracleSim(sc, "fp64", keep_history=True)
    np.testing.assert_array_equal(o.rollout()["counts"], out["counts"])
    go = o.backward(ybar)
    base = dict(w=np.asarray(sc.w, np.float64).copy(), od_lambda=np.asarray(sc.od_lambda, np.float64).copy())

    def F(params):
        tape.rewind()
        with torch.no_grad():
            return dense_ref.run(sc, ybar=ybar, tape=tape, params=params)[0]["loss"]

    def central(k, idx, h):
        p1 = {kk: v.copy() for kk, v in base.items()}
        p2 = {kk: v.copy() for kk, v in base.items()}
        p1[k][idx] += h
        p2[k][idx] -= h
        return (F(p1) - F(p2)) / (2 * h)

    lam = rng.permutation(np.nonzero(np.abs(go["od_lambda"]) > 1e-9)[0])[:16]
    assert len(lam) >= 12
    checked = {"w": 0, "od_lambda": 0}
    for k, idxs in (("w", range(16)), ("od_lambda", lam)):
        for idx in idxs:
            h = 2e-6 * max(1.0, abs(base[k][idx]))
            # lambda enters through straight-through weights, linearly: one
            # central difference is exact; w through softmaxes: Richardson
            fd = central(k, idx, h) if k == "od_lambda" else (4.0 * central(k, idx, h / 2) - central(k, idx, h)) / 3.0
            assert abs(fd - go[k][idx]) <= 2e-6 * max(abs(go[k][idx]), 1e-3), (k, idx, fd, go[k][idx])
            checked[k] += 1
    assert checked == {"w": 16, "od_lambda": len(lam)}
