"""Launch-shape autotuner: times short rollouts for each candidate shape of the
node-model kernel (queue slots staged in shared memory per link block) on the
simulator's own stream and keeps the fastest.  Results never depend on the
shape, only the time does."""
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
