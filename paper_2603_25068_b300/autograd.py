"""torch.autograd.Function over the C ABI: bin counts of a rollout as a
differentiable function of the simulator's parameters.

The forward value is the simulated (integer) count of each link and bin; the
backward is sim_backward, the reverse pass of the straight-through /
trajectory-grafting surrogate (SI-B, SI-C, SI-D).  PyTorch provides the tensors
and the stream only; both passes run in the library's CUDA kernels.

    counts = rollout_counts(sim, u, kappa, alpha, beta, cost, w, alpha_origin, od_lambda)
    loss = ((counts[:, sensors] - observed) ** 2).mean()
    loss.backward()
"""
from __future__ import annotations

import torch

PARAMS = ("u", "kappa", "alpha", "beta", "cost", "w", "alpha_origin", "od_lambda")


class RolloutCounts(torch.autograd.Function):
    # The simulator enqueues on its own stream: it waits for torch's current
    # stream before it reads or writes tensors torch produced or allocated, and
    # torch's stream waits for it before the outputs are used.
    @staticmethod
    def forward(ctx, sim, T, u, kappa, alpha, beta, cost, w, alpha_origin, od_lambda):
        dev = torch.device("cuda", sim.device)
        params = (u, kappa, alpha, beta, cost, w, alpha_origin)
        cur, s = torch.cuda.current_stream(dev), sim.torch_stream()
        if all(x.device == dev for x in params):
            # device tensors: copied on the simulator's stream, no host round trip
            prep = lambda x: x.detach().to(torch.float32).contiguous().reshape(-1)
            dp = [prep(x) for x in params]                       # made on torch's stream
            s.wait_stream(cur)
            sim.set_params_device(*dp)
        else:
            host = lambda x: x.detach().to("cpu", torch.float32).numpy()
            sim.set_params(u=host(u), kappa=host(kappa), alpha=host(alpha), beta=host(beta), cost=host(cost),
                           w=host(w), alpha_origin=float(alpha_origin.detach().reshape(-1)[0]))
            s.wait_stream(cur)
        out = sim.rollout(T, device=True)
        cur.wait_stream(s)
        ctx.sim = sim
        ctx.od_dtype = od_lambda.dtype
        return out["counts"].to(torch.float32)

    @staticmethod
    def backward(ctx, g_counts):
        sim = ctx.sim
        dev = torch.device("cuda", sim.device)
        yb = g_counts.to(device=dev, dtype=torch.float32).contiguous()      # before the wait: made on torch's stream
        cur, s = torch.cuda.current_stream(dev), sim.torch_stream()
        s.wait_stream(cur)
        g = sim.backward_device(yb)
        cur.wait_stream(s)
        return (None, None, g["u"], g["kappa"], g["alpha"], g["beta"], g["cost"], g["w"],
                g["alpha_origin"].reshape(()), g["od_lambda"])


def rollout_counts(sim, u, kappa, alpha, beta, cost, w, alpha_origin, od_lambda, T=None):
    """Counts [n_bins, L] (float32, on the simulator's device); differentiable in
    every parameter.  od_lambda enters through the demand weights only: the
    simulated vehicles stay those of the scenario."""
    T = sim.sc.T if T is None else T
    if not torch.is_tensor(alpha_origin):
        alpha_origin = torch.tensor(float(alpha_origin))
    return RolloutCounts.apply(sim, T, u, kappa, alpha, beta, cost, w, alpha_origin, od_lambda)
