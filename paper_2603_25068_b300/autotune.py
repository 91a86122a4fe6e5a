"""Launch-shape autotuner: times short rollouts for each candidate shape and
keeps the fastest.  For one simulator: the queue slots staged in shared memory
per link block of the node-model kernel.  For a batch: the executor (one
cooperative launch per advance with warp-per-32-links items, or one launch per
phase and step with link blocks).  Results never depend on the shape, only the
time does."""
from __future__ import annotations

from . import native as nat

STAGES = (2048, 4096, 6144)


def set_stage(sim, slots: int) -> None:
    nat.check(sim.lib.sim_set_stage(sim.h, int(slots)), sim.h)


def tune_stage(sim, T: int = 600, reps: int = 2, stages=STAGES):
    """Returns (best stage, {stage: ms per rollout of T steps})."""
    import torch
    stream = torch.cuda.current_stream()
    times = {}
    for g in stages:
        set_stage(sim, g)
        sim.rollout(T, device=True)                 # capture + warm
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        for _ in range(reps):
            sim.rollout(T, device=True)
        ev[1].record(stream)
        torch.cuda.synchronize()
        times[g] = ev[0].elapsed_time(ev[1]) / reps
    best = min(times, key=times.get)
    set_stage(sim, best)
    return best, times


BATCH_EXECUTORS = ("persistent", "step")


def tune_batch(batch, T: int = 120, reps: int = 1, executors=BATCH_EXECUTORS):
    """Times a batch rollout of T steps with each executor and keeps the
    fastest.  Returns (best executor, {executor: ms per rollout})."""
    import time

    import torch
    times = {}
    for e in executors:
        try:
            batch.set_executor(e)
        except nat.SimError:                      # unavailable on this device
            continue
        batch.rollout(T)                          # warm (and graph capture)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            batch.rollout(T)
        torch.cuda.synchronize()
        times[e] = (time.perf_counter() - t0) * 1e3 / reps
    best = min(times, key=times.get)
    batch.set_executor(best)
    return best, times


def link_occupancy(sim, T=None, samples: int = 12):
    """Mean number of vehicles on each link over a rollout of T steps, from
    the exported state at ``samples`` evenly spaced steps."""
    import numpy as np
    T = sim.sc.T if T is None else T
    sim.reset(T)
    occ = np.zeros(sim.sc.L, np.float64)
    every = max(1, T // samples)
    n = 0
    while sim.t + every <= T:
        sim.step(every)
        vl = sim.state(fields=("veh_link",))["veh_link"]
        occ += np.bincount(vl[vl >= 0], minlength=sim.sc.L)
        n += 1
    return occ / max(n, 1)


def balance_partition(sim, T=None, samples: int = 12, per_link: float = 20.0, occ=None):
    """Partition the persistent executor's links by measured load: weight of a
    link = its mean vehicle count over a rollout + ``per_link``.  Returns the
    weights set (None if the simulator has no persistent executor)."""
    if sim.persist_groups() is None:
        return None
    if occ is None:
        occ = link_occupancy(sim, T, samples)
    w = occ + float(per_link)
    sim.set_partition_weights(w)
    return w


RECOMPUTE_MODES = ("overlap", "serial")


def tune_recompute(sim, ybar, T=None, modes=RECOMPUTE_MODES):
    """Segment recomputation of the reverse pass: times one reverse pass of a
    fresh rollout per mode (after one untimed pass) and keeps the faster.
    Gradients do not depend on the mode.  Returns (best, {mode: ms})."""
    import time
    import torch
    sim.rollout(T)
    sim.backward(ybar)                               # workspaces and streams exist before timing
    times = {}
    for m in modes:
        sim.set_recompute(m)
        sim.rollout(T)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.backward(ybar)
        torch.cuda.synchronize()
        times[m] = 1e3 * (time.perf_counter() - t0)
    best = min(times, key=times.get)
    sim.set_recompute(best)
    return best, times
