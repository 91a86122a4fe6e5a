"""Parity of the CUDA reverse pass (sim_backward) with the oracle's reverse mode.

Both differentiate the same frozen-decision surrogate through the same float32
forward (the oracle's float build takes every decision in the kernel's
precision), with double-precision accumulators on both sides; the GPU returns
float32 gradients.  Tolerance: 1e-5 of the largest gradient of each parameter
family (the M-scaled merge terms make absolute scales differ by ~1e5), and
1e-4 relative on the entries above 1 % of it (gradcheck.py)."""
import numpy as np
import pytest

from gradcheck import compare_grads
from oracle.oracle import OracleSim
from paper_2603_25068_b300 import scenario as S

pytestmark = pytest.mark.gpu

KEYS = ("u", "kappa", "alpha", "alpha_origin", "beta", "cost", "w", "od_lambda")


@pytest.fixture(scope="module")
def Simulator():
    import torch
    assert torch.cuda.is_available()
    from paper_2603_25068_b300.sim import Simulator
    return Simulator


def compare(Simulator, sc, K, seed=0, with_xT=True, rtol=1e-5, recompute="overlap"):
    rng = np.random.default_rng(seed)
    g = Simulator(sc, ckpt_every=K, route_cap=64)
    g.set_recompute(recompute)
    out = g.rollout()
    nb = out["counts"].shape[0]
    ybar = rng.normal(size=(nb, sc.L)).astype(np.float32)
    xT = rng.normal(size=sc.N).astype(np.float32) if with_xT else None
    st = g.state()
    gg = g.backward(ybar, xT)
    o = OracleSim(sc, "fp32", keep_history=True)
    ref = o.rollout()
    np.testing.assert_array_equal(out["counts"], ref["counts"])
    on = o.state()["veh_link"] >= 0
    go = o.backward(ybar.astype(np.float64), None if xT is None else np.where(on, xT, 0).astype(np.float64))
    compare_grads(gg, go, KEYS, abs_frac=rtol)
    return go


@pytest.mark.parametrize("recompute", ["overlap", "serial"])
@pytest.mark.parametrize("K", [300, 7])
def test_backward_tiny_grid(Simulator, K, recompute):
    sc = S.tiny_grid(T=150).copy(obs_every=50)
    compare(Simulator, sc, K, recompute=recompute)


@pytest.mark.parametrize("seed", [1, 2, 7])
def test_backward_dense_small(Simulator, seed):
    sc = S.random_small(seed=seed, side=3, n_vehicles=160, T=90).copy(obs_every=30)
    go = compare(Simulator, sc, 13, seed=seed)
    assert np.count_nonzero(go["alpha"]) > 0 and np.count_nonzero(go["beta"]) > 0


@pytest.mark.parametrize("recompute", ["overlap", "serial"])
def test_backward_city_small(Simulator, recompute):
    sc = S.city_small(T=240).copy(obs_every=60)
    compare(Simulator, sc, 60, seed=5, with_xT=False, recompute=recompute)


@pytest.mark.parametrize("recompute", ["overlap", "serial"])
def test_backward_platoons(Simulator, recompute):
    # agents of 5 vehicles (step 5 s); gradients against the oracle's reverse mode
    sc = S.with_platoons(S.random_small(seed=2, side=3, n_vehicles=150, T=750), 5.0)
    compare(Simulator, sc, 20, recompute=recompute)


def test_backward_tg_toy(Simulator):
    sc = S.tg_toy(2.0, 1.0)
    g = Simulator(sc, ckpt_every=4, route_cap=8)
    g.rollout()
    x = g.state()["veh_pos"]
    gg = g.backward(np.zeros((1, sc.L), np.float32), (2 * x).astype(np.float32))
    np.testing.assert_allclose(gg["u"][:2], [32.0, 8.0], rtol=1e-6)


def test_backward_needs_a_recorded_rollout(Simulator):
    from paper_2603_25068_b300.native import SimError, SIM_ESTATE
    sc = S.tiny_grid(n_vehicles=50, T=20)
    g = Simulator(sc)                                   # forward only
    g.rollout()
    with pytest.raises(SimError) as e:
        g.backward(np.zeros((1, sc.L), np.float32))
    assert e.value.code == SIM_ESTATE
    g = Simulator(sc, ckpt_every=5)
    g.reset(20)
    g.step(20)                                          # the step path records no tape
    with pytest.raises(SimError):
        g.backward(np.zeros((1, sc.L), np.float32))


def test_concurrent_reverse_passes_equal_sequential(Simulator):
    """Reverse passes of several simulators from several host threads (each
    handle on its own stream, each call with its own workspace) give the
    gradients of the same passes one after another, up to the order of the
    double-precision atomic additions."""
    import threading
    import torch
    scs = [S.random_small(seed=s, side=3, n_vehicles=150, T=80).copy(obs_every=20) for s in (11, 12, 13, 14)]
    rng = np.random.default_rng(3)
    sims = [Simulator(sc, ckpt_every=9, route_cap=64, stream=torch.cuda.Stream()) for sc in scs]
    ybar = []
    for s_ in sims:
        out = s_.rollout()
        ybar.append(rng.normal(size=out["counts"].shape).astype(np.float32))
    seq = [s_.backward(y) for s_, y in zip(sims, ybar)]
    for s_ in sims:
        s_.rollout()
    par = [None] * len(sims)

    def run(k):
        par[k] = sims[k].backward(ybar[k])
    ths = [threading.Thread(target=run, args=(k,)) for k in range(len(sims))]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    for a, b in zip(seq, par):
        assert b is not None
        for k in a:
            scale = max(1e-6, float(np.abs(a[k]).max()))
            np.testing.assert_allclose(b[k], a[k], rtol=0, atol=1e-6 * scale, err_msg=k)
    for s_ in sims:
        s_.close()


def test_tune_recompute_keeps_a_mode_and_the_gradient(Simulator):
    # the recompute-mode autotuner times both modes and keeps one; the
    # gradient after tuning is the gradient of either mode
    from paper_2603_25068_b300.autotune import RECOMPUTE_MODES, tune_recompute
    sc = S.city_small()
    g = Simulator(sc, ckpt_every=30, route_cap=64)
    out = g.rollout()
    ybar = np.random.default_rng(5).normal(size=out["counts"].shape).astype(np.float32)
    g.set_recompute("overlap")
    g.rollout()
    ref = g.backward(ybar)
    best, times = tune_recompute(g, ybar)
    assert best in RECOMPUTE_MODES and set(times) == set(RECOMPUTE_MODES)
    assert all(v > 0 for v in times.values())
    g.rollout()
    got = g.backward(ybar)
    for k in ref:
        scale = np.max(np.abs(ref[k])) + 1e-30
        assert np.max(np.abs(got[k].astype(np.float64) - ref[k])) <= 1e-6 * scale, k
    g.close()
