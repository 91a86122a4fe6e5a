"""Batched simulation: many Simulator handles advanced together (sim_batch_* of
the C ABI), by one cooperative launch per advance (persistent executor) or one
launch per phase and step (step executor).  Members keep their own scenario, state,
step counter and horizon, so they can join at any step boundary (continuous
batching) and each member's result equals its solo result."""
from __future__ import annotations

import ctypes as C
from typing import Sequence

import numpy as np

from . import native as nat


class Batch:
    def __init__(self, sims: Sequence):
        self.sims = list(sims)
        self.lib = nat.lib()
        arr = (C.c_void_p * len(self.sims))(*[s.h.value for s in self.sims])
        h = C.c_void_p()
        rc = self.lib.sim_batch_create(C.cast(arr, C.POINTER(C.c_void_p)), len(self.sims), C.byref(h))
        if rc != nat.SIM_OK:
            raise nat.SimError(rc, self.lib.sim_batch_last_error(None).decode())
        self.h = h

    EXECUTORS = {"auto": 0, "step": 1, "persistent": 2}

    def set_executor(self, name: str):
        """"persistent", "step" or "auto"; results do not depend on it."""
        self._check(self.lib.sim_batch_set_executor(self.h, self.EXECUTORS[name]))

    @property
    def executor(self) -> str:
        return {1: "step", 2: "persistent"}[self.lib.sim_batch_get_executor(self.h)]

    def _check(self, rc):
        if rc != nat.SIM_OK:
            raise nat.SimError(rc, self.lib.sim_batch_last_error(self.h).decode())

    def start(self, k: int, T: int):
        self.sims[k].T = T
        self._check(self.lib.sim_batch_start(self.h, k, T))

    def advance(self, n_steps: int):
        """Advance running members; returns a bool array of finished members."""
        fin = np.zeros(len(self.sims), np.int32)
        self._check(self.lib.sim_batch_advance(self.h, n_steps, C.c_void_p(fin.ctypes.data)))
        return fin.astype(bool)

    def rollout(self, T: int):
        for s in self.sims:
            s.T = T
        self._check(self.lib.sim_batch_rollout(self.h, T))
        return [s.outputs() for s in self.sims]

    def close(self):
        if getattr(self, "h", None):
            self.lib.sim_batch_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
