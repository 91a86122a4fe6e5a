"""The optimisation loop of the paper, written out plainly (Methods,
Optimization), in float64 numpy.

TEST INFRASTRUCTURE ONLY: imported by tests/ and by nothing on the product path.

Each iteration runs the forward simulation, the loss, its gradient and an
AdamW update.  AdamW is Loshchilov & Hutter's decoupled weight decay on top of
Adam (Kingma & Ba), with the paper's learning rate 1e-1 and weight decay 1e-5
and the default hyperparameters otherwise (beta1 0.9, beta2 0.999, eps 1e-8).
The loop stops once the loss has not improved for 20 iterations and keeps the
parameters of the lowest loss.

Losses (Methods, Optimization; Results, gradient-guided traffic control):
  * calibration: mean over the observed links (and bins) of the squared error
    between simulated and observed counts;
  * control: squared error between half the target link's cumulative count
    without control and its simulated cumulative count.
"""
from __future__ import annotations

import numpy as np

BETA1, BETA2, EPS = 0.9, 0.999, 1e-8
LR, WEIGHT_DECAY, PATIENCE = 1e-1, 1e-5, 20


class AdamW:
    """Adam moments with bias correction; the weight decay is applied to the
    parameter directly (decoupled), scaled by the learning rate."""

    def __init__(self, lr=LR, weight_decay=WEIGHT_DECAY, beta1=BETA1, beta2=BETA2, eps=EPS):
        self.lr, self.wd, self.b1, self.b2, self.eps = lr, weight_decay, beta1, beta2, eps
        self.m = self.v = None
        self.t = 0

    def step(self, theta, grad):
        theta = np.asarray(theta, np.float64)
        grad = np.asarray(grad, np.float64)
        if self.m is None:
            self.m = np.zeros_like(theta)
            self.v = np.zeros_like(theta)
        self.t += 1
        self.m = self.b1 * self.m + (1.0 - self.b1) * grad
        self.v = self.b2 * self.v + (1.0 - self.b2) * grad * grad
        m_hat = self.m / (1.0 - self.b1 ** self.t)
        v_hat = self.v / (1.0 - self.b2 ** self.t)
        return theta - self.lr * (m_hat / (np.sqrt(v_hat) + self.eps) + self.wd * theta)


class EarlyStop:
    """Tracks the lowest loss; ``stop`` once `patience` iterations in a row
    have not lowered it."""

    def __init__(self, patience=PATIENCE):
        self.patience = patience
        self.best = np.inf
        self.best_iter = -1
        self.iter = -1

    def update(self, loss) -> bool:
        self.iter += 1
        if loss < self.best:
            self.best, self.best_iter = float(loss), self.iter
            return True
        return False

    @property
    def stop(self) -> bool:
        return self.iter - self.best_iter >= self.patience


def calibration_loss(counts, observed, sensors):
    """Mean squared error over the observed links and bins, and its gradient
    with respect to the counts."""
    c = np.asarray(counts, np.float64)
    d = c[:, sensors] - np.asarray(observed, np.float64)
    g = np.zeros_like(c)
    g[:, sensors] = 2.0 * d / d.size
    return float(np.mean(d * d)), g


def control_loss(counts, target, goal):
    """Squared error between the goal and the target link's cumulative count
    over all bins, and its gradient with respect to the counts."""
    c = np.asarray(counts, np.float64)
    cum = c[:, target].sum()
    g = np.zeros_like(c)
    g[:, target] = 2.0 * (cum - goal)
    return float((cum - goal) ** 2), g
