"""Pins of the oracle's optimisation loop (Methods, Optimization): AdamW with
decoupled weight decay and bias-corrected moments, the 20-iteration early stop,
and the calibration and control losses."""
import numpy as np
import pytest

from oracle.optim import AdamW, EarlyStop, calibration_loss, control_loss, LR, WEIGHT_DECAY, EPS


def test_first_step_is_signed_learning_rate_plus_decay():
    # bias correction makes the first moments exactly g and g^2
    rng = np.random.default_rng(0)
    theta, g = rng.normal(size=7), rng.normal(size=7)
    out = AdamW().step(theta, g)
    want = theta - LR * (g / (np.abs(g) + EPS) + WEIGHT_DECAY * theta)
    np.testing.assert_allclose(out, want, rtol=1e-12, atol=1e-15)


def test_constant_gradient_closed_form():
    # with a constant gradient every bias-corrected step is lr g / (|g| + eps)
    # plus the decay: theta_t = a^t theta_0 - b (1 - a^t) / (1 - a),
    # a = 1 - lr wd, b = lr g / (|g| + eps)
    theta0, g, n = np.array([3.0, -2.0, 0.5]), np.array([0.7, -1e-3, 4.0]), 50
    opt, th = AdamW(), theta0.copy()
    for _ in range(n):
        th = opt.step(th, g)
    a = 1.0 - LR * WEIGHT_DECAY
    b = LR * g / (np.abs(g) + EPS)
    want = a ** n * theta0 - b * (1.0 - a ** n) / (1.0 - a)
    np.testing.assert_allclose(th, want, rtol=1e-9)


def test_agrees_with_torch_adamw():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    theta0 = rng.normal(size=11)
    grads = rng.normal(size=(30, 11)) * np.linspace(1e-3, 10.0, 11)
    p = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
    opt_t = torch.optim.AdamW([p], lr=LR, weight_decay=WEIGHT_DECAY, betas=(0.9, 0.999), eps=EPS)
    opt_o, th = AdamW(), theta0.copy()
    for g in grads:
        p.grad = torch.tensor(g, dtype=torch.float64)
        opt_t.step()
        th = opt_o.step(th, g)
    np.testing.assert_allclose(th, p.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_early_stop_after_twenty_iterations_without_improvement():
    es = EarlyStop()
    seq = [5.0, 4.0, 3.0] + [3.0, 3.5, 10.0] * 10
    stopped_at = None
    for i, loss in enumerate(seq):
        es.update(loss)
        if es.stop:
            stopped_at = i
            break
    assert (es.best, es.best_iter) == (3.0, 2)
    assert stopped_at == 22                  # iterations 3 .. 22: twenty without a lower loss
    es = EarlyStop()
    for i, loss in enumerate([5.0] + [6.0] * 15 + [4.0] + [7.0] * 19):
        es.update(loss)
        assert not es.stop, i                # the improvement at 16 restarts the count
    es.update(7.0)
    assert es.stop and es.best_iter == 16


def test_losses_and_their_gradients():
    rng = np.random.default_rng(2)
    counts = rng.integers(0, 50, size=(6, 20)).astype(np.float64)
    sensors = np.array([1, 4, 7, 19])
    obs = rng.integers(0, 50, size=(6, 4)).astype(np.float64)
    loss, g = calibration_loss(counts, obs, sensors)
    assert loss == pytest.approx(np.mean((counts[:, sensors] - obs) ** 2))
    # finite differences (the loss is quadratic: central differences are exact)
    for (b, j) in [(0, 1), (5, 19), (3, 2)]:
        e = np.zeros_like(counts)
        e[b, j] = 0.5
        fd = (calibration_loss(counts + e, obs, sensors)[0] - calibration_loss(counts - e, obs, sensors)[0]) / 1.0
        assert g[b, j] == pytest.approx(fd, rel=1e-12, abs=1e-12)
    target, goal = 7, 0.5 * counts[:, 7].sum()
    loss, g = control_loss(counts, target, goal)
    assert loss == pytest.approx((counts[:, 7].sum() - goal) ** 2)
    assert np.all(g[:, target] == 2.0 * (counts[:, 7].sum() - goal))
    assert np.count_nonzero(g) == counts.shape[0]
