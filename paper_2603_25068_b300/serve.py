"""Serving loop: continuous batching of simulation requests on one GPU.

Requests (nowcast rollouts, calibration-gradient rollouts, control-candidate
rollouts) arrive over time.  The engine
  * admits waiting requests shortest remaining work first (vehicle-steps,
    three times for a gradient request, as seconds of engine time, less the
    time the request has already waited: a large request is not passed over
    for longer than about its own run time), each as soon as an upper bound of its
    device memory fits in the HBM budget (replaced by sim_device_bytes of the
    handle once created, plus its reverse-pass needs) and fewer than
    max_in_flight + prefetch requests are admitted and unfinished (None:
    memory only); at most max_in_flight of them run at once, the others'
    simulators are built ahead so that host set-up overlaps the GPU work,
  * runs a request that is alone (max_in_flight 1, or nothing else running or
    ready) as one rollout of its own simulator, without a batch,
  * builds the simulator of an admitted request on a creation thread with a
    stream of its own, so that host set-up and uploads overlap the running
    batch instead of stalling it,
  * runs every admitted forward rollout in one batch (sim_batch_*), a new
    request joining at the next step boundary, finished ones leaving it,
  * runs the reverse pass of a finished gradient request between forward
    chunks on the engine's stream (reversers = 0, the default: the
    simulator's kernels each fill the GPU, so one device job at a time is
    the fastest order), or on worker threads with streams of their own
    (reversers > 0: reverse passes overlap one another and the forward work
    on the device),
  * records each request's latency from arrival to result.
Each request's result is the one it would get alone: batching changes neither
its random key nor its state.
"""
from __future__ import annotations

import dataclasses
import queue
import sys
import threading
import time
from typing import List, Optional

import numpy as np

from . import native as nat
from .batch import Batch
from .sim import Simulator


@dataclasses.dataclass
class Request:
    rid: int
    kind: str                 # "nowcast" | "calibration" | "control"
    scenario: object          # scenario.Scenario (its T is the horizon)
    arrival: float            # seconds after the stream starts
    observed: Optional[np.ndarray] = None     # [n_bins, n_sensors] calibration targets
    target_link: int = 0      # control: link whose count is to be halved
    # filled by the engine
    admitted: float = float("nan")
    finished: float = float("nan")
    result: Optional[dict] = None

    @property
    def needs_grad(self):
        return self.kind in ("calibration", "control")

    @property
    def vehicle_steps(self):
        return self.scenario.N * self.scenario.T


def loss_cotangent(req: Request, counts: np.ndarray) -> np.ndarray:
    """dL/dcounts of the request's loss: calibration -- mean squared error of the
    sensor counts against the observations (Methods "Optimization"); control --
    squared error of the target link's total count against half its value."""
    sc = req.scenario
    yb = np.zeros(counts.shape, np.float32)
    if req.kind == "calibration":
        s = sc.sensors
        diff = counts[:, s].astype(np.float32) - req.observed
        yb[:, s] = 2.0 * diff / diff.size
    elif req.kind == "control":
        tot = float(counts[:, req.target_link].sum())
        yb[:, req.target_link] = 2.0 * (tot - 0.5 * tot)
    return yb


def run_request_alone(req: Request, device: int = 0, ckpt_every: int = 180, route_cap: int = 256) -> dict:
    """The same request processed on its own (the reference for mix parity and
    for serial execution)."""
    sc = req.scenario
    sim = Simulator(sc, device=device, ckpt_every=ckpt_every if req.needs_grad else 0, route_cap=route_cap)
    out = sim.rollout(sc.T)
    res = dict(counts=out["counts"], speed=out["speed"], travel_time=out["travel_time"])
    if req.needs_grad:
        res["grad"] = sim.backward(loss_cotangent(req, out["counts"]))
    sim.close()
    return res


def handle_bytes_bound(sc, ckpt_every: int, route_cap: int) -> float:
    """Upper bound of sim_device_bytes for a scenario (admission before the
    handle exists): slot arena, per-link and per-vehicle state, outputs, and
    for a gradient request the checkpoints and the route log."""
    slots = float(np.sum(np.floor(sc.length.astype(np.float64) * sc.kappa / sc.dn) + 2))
    nb = -(-sc.T // sc.obs_every)
    b = 32.0 * slots + (320.0 + 12.0 * nb) * sc.L + 48.0 * sc.N + 4.0 * sc.Z * sc.V + 16.0 * sc.V
    if ckpt_every > 0:
        b += (sc.T // ckpt_every + 1) * (16.0 * slots + 64.0 * sc.L + 4.0 * sc.V + 4.0 * sc.N)
        b += (8.0 * (route_cap + 7) + 8.0) * sc.N
    return b


class Engine:
    def __init__(self, device: int = 0, hbm_budget: float = 150e9, chunk: int = 240, ckpt_every: int = 180,
                 route_cap: int = 256, creators: int = 2, reversers: int = 0, max_in_flight: Optional[int] = None,
                 order: str = "srw", prefetch: int = 2):
        import torch
        self.torch = torch
        self.device = device
        self.budget = hbm_budget
        if order not in ("srw", "fifo"):
            raise ValueError("order must be 'srw' (shortest remaining work) or 'fifo'")
        self.max_in_flight = max_in_flight
        self.prefetch = prefetch
        self.order = order
        self.in_flight = 0                      # admitted and not finished (creating, ready, running, reversing)
        self.ready: List[tuple] = []            # built simulators waiting to run: (request, simulator, bytes)
        self.chunk = chunk
        self.ckpt_every = ckpt_every
        self.route_cap = route_cap
        self.stream = torch.cuda.Stream(device=device)
        self.bwd_streams = [torch.cuda.Stream(device=device) for _ in range(reversers)]
        self.active: List[tuple] = []          # (request, simulator, bytes)
        self.reversers = reversers
        self.pending_bwd: List[tuple] = []     # reversers = 0: (request, simulator, bytes, outputs) due
        self.batch: Optional[Batch] = None
        self.batch_members: List[int] = []
        self.used = 0.0
        self.lock = threading.Lock()
        self.worker_error = None
        self.t0 = None
        self.bwd_q: "queue.Queue" = queue.Queue()
        self.create_q: "queue.Queue" = queue.Queue()
        self.ready_q: "queue.Queue" = queue.Queue()
        self.bwd_threads = [threading.Thread(target=self._bwd_worker, args=(k,), daemon=True)
                            for k in range(reversers)]
        self.create_threads = [threading.Thread(target=self._create_worker, args=(k,), daemon=True)
                               for k in range(creators)]
        self.create_streams = [torch.cuda.Stream(device=device) for _ in range(creators)]
        for th in self.bwd_threads + self.create_threads:
            th.start()

    # -------------------------------------------------------------- helpers
    def now(self):
        return time.perf_counter() - self.t0

    def _estimate_extra(self, req: Request) -> float:
        """Device bytes beyond the handle: reverse-pass workspace share."""
        if not req.needs_grad:
            return 0.0
        sc = req.scenario
        slots = float(np.sum(np.floor(sc.length.astype(np.float64) * sc.kappa / sc.dn) + 2))
        # two tape sets: per step 9 B per slot, 68 B per link and 20 B per origin
        # queue (queue states, records, merge words and merge sums)
        return (18.0 * (self.ckpt_every + 1) * slots + 2.0 * (self.ckpt_every + 1) * (68.0 * sc.L + 20.0 * sc.V)
                + 16.0 * sc.N * self.route_cap)

    def _reverse(self, req, sim, nbytes, out, stream):
        """The reverse pass of a gradient request whose forward is done; its
        result and the release of its memory."""
        with self.torch.cuda.device(self.device):
            sim.set_stream(stream)                     # out of the batch
            if out is None:
                out = sim.outputs()
            g = sim.backward(loss_cotangent(req, out["counts"]))
            req.result = dict(counts=out["counts"], speed=out["speed"], travel_time=out["travel_time"], grad=g)
            sim.close()
        with self.lock:
            self.used -= nbytes
            self.in_flight -= 1
        req.finished = self.now()

    def _bwd_worker(self, k: int):
        while True:
            item = self.bwd_q.get()
            if item is None:
                return
            try:
                self._reverse(*item, self.bwd_streams[k])
            except Exception as e:          # reported by the main loop
                self.worker_error = e
                return

    def _create_worker(self, k: int):
        torch = self.torch
        try:                 # the thread's first simulator pays one-time set-up costs
            from . import scenario as S
            with torch.cuda.device(self.device):
                Simulator(S.tiny_grid(n_vehicles=50, T=20), device=self.device, stream=self.create_streams[k]).close()
        except Exception as e:
            self.worker_error = e
            return
        while True:
            item = self.create_q.get()
            if item is None:
                return
            req, reserved = item
            try:
                with torch.cuda.device(self.device):
                    sim = Simulator(req.scenario, device=self.device, stream=self.create_streams[k],
                                    ckpt_every=self.ckpt_every if req.needs_grad else 0, route_cap=self.route_cap)
                    sim.set_stream(self.stream)          # drains the creation stream
                nbytes = float(sim.device_bytes()) + self._estimate_extra(req)
                with self.lock:
                    self.used += nbytes - reserved
            except Exception as e:                      # reported by the main loop
                self.worker_error = e
                return
            self.ready_q.put((req, sim, nbytes))

    def _rebuild(self, new=()):
        if self.batch is not None:
            self.batch.close()
            self.batch = None
        if self.active:
            self.batch = Batch([s for (_, s, _) in self.active])
            for req in new:
                i = next(i for i, (r, _, _) in enumerate(self.active) if r is req)
                self.batch.start(i, req.scenario.T)

    def _admit(self, req: Request) -> bool:
        """Reserve an upper bound of the request's device memory and hand it to
        the creation thread; False if it does not fit yet."""
        reserved = handle_bytes_bound(req.scenario, self.ckpt_every if req.needs_grad else 0,
                                      self.route_cap) + self._estimate_extra(req)
        with self.lock:
            if self.max_in_flight is not None and self.in_flight >= self.max_in_flight + self.prefetch:
                return False
            if self.used + reserved > self.budget and (self.used > 0 or self.active):
                return False
            self.used += reserved
            self.in_flight += 1
        self.create_q.put((req, reserved))
        return True

    def _finish_forward(self, req, sim, nbytes, out=None):
        if req.needs_grad:
            if self.reversers == 0:
                self.pending_bwd.append((req, sim, nbytes, out))
            else:
                self.bwd_q.put((req, sim, nbytes, out))
            return
        if out is None:
            out = sim.outputs()
        req.result = dict(counts=out["counts"], speed=out["speed"], travel_time=out["travel_time"])
        sim.close()
        with self.lock:
            self.used -= nbytes
            self.in_flight -= 1
        req.finished = self.now()

    def _create_and_run(self, req):
        """A request that finds the engine idle (nothing created, ready, running
        or reversing): its simulator built on this thread and its forward run
        at once, with no hand-over to a creation thread."""
        with self.lock:
            self.in_flight += 1
        sim = Simulator(req.scenario, device=self.device, stream=self.stream,
                        ckpt_every=self.ckpt_every if req.needs_grad else 0, route_cap=self.route_cap)
        nbytes = float(sim.device_bytes()) + self._estimate_extra(req)
        with self.lock:
            self.used += nbytes
        req.admitted = self.now()
        self._run_alone(req, sim, nbytes)

    def _run_alone(self, req, sim, nbytes):
        """A request with nothing beside it: one rollout of its own simulator
        (a single persistent launch), as serial execution runs it."""
        out = sim.rollout(req.scenario.T)
        self._finish_forward(req, sim, nbytes, out)

    # -------------------------------------------------------------- main loop
    def run(self, requests: List[Request], poll: float = 0.0005, max_seconds: float = 3600.0):
        """Serve the requests (arrival times in seconds from now); returns them
        with results and timings."""
        # the main loop and the creation threads hand the interpreter lock to
        # one another around every library call: a short switch interval keeps
        # each hand-over well below a millisecond (the default is 5 ms)
        switch = sys.getswitchinterval()
        sys.setswitchinterval(min(switch, 2e-4))
        try:
            return self._run(requests, poll, max_seconds)
        finally:
            sys.setswitchinterval(switch)

    def _run(self, requests: List[Request], poll: float, max_seconds: float):
        torch = self.torch
        pending = sorted(requests, key=lambda r: r.arrival)
        self.t0 = time.perf_counter()
        k = 0
        waiting: List[Request] = []
        with torch.cuda.device(self.device):
            while True:
                if self.worker_error is not None or not all(th.is_alive() for th in self.bwd_threads + self.create_threads):
                    raise RuntimeError(f"serving worker failed: {self.worker_error!r}")
                if self.now() > max_seconds:
                    raise RuntimeError("serving run exceeded its time limit")
                while k < len(pending) and pending[k].arrival <= self.now():
                    waiting.append(pending[k])
                    k += 1
                now = self.now()
                if self.order == "srw":
                    waiting.sort(key=lambda r: request_priority(r, now))
                if waiting and self.in_flight == 0:      # idle: the first request as serial execution runs it
                    self._create_and_run(waiting.pop(0))
                    continue
                waiting = [req for req in waiting if not self._admit(req)]
                while True:                              # simulators built by the creation thread
                    try:
                        self.ready.append(self.ready_q.get_nowait())
                    except queue.Empty:
                        break
                if self.order == "srw":
                    self.ready.sort(key=lambda a: request_priority(a[0], now))
                if self.pending_bwd:                     # a due reverse pass first: it finishes a request
                    if self.order == "srw":
                        self.pending_bwd.sort(key=lambda a: request_priority(a[0], now))
                    self._reverse(*self.pending_bwd.pop(0), self.stream)
                    continue
                new = []
                while self.ready and (self.max_in_flight is None or len(self.active) < self.max_in_flight):
                    req, sim, nbytes = self.ready.pop(0)
                    req.admitted = self.now()
                    self.active.append((req, sim, nbytes))
                    new.append(req)
                if len(new) == 1 and len(self.active) == 1 and (self.max_in_flight == 1 or not self.ready):
                    self._run_alone(*self.active.pop())
                    continue
                if new:
                    self._rebuild(new)
                if not self.active:
                    if all(np.isfinite(r.finished) for r in requests):
                        break
                    # idle: wake as soon as a simulator is ready, at the next
                    # arrival, or after `poll` seconds, whichever comes first
                    timeout = poll
                    if k < len(pending):
                        timeout = min(timeout, max(pending[k].arrival - self.now(), 0.0))
                    try:
                        self.ready.append(self.ready_q.get(timeout=timeout))
                    except queue.Empty:
                        pass
                    continue
                fin = self.batch.advance(self.chunk)
                if fin.any():
                    done = [self.active[i] for i in np.nonzero(fin)[0]]
                    self.active = [a for i, a in enumerate(self.active) if not fin[i]]
                    self._rebuild()
                    for item in done:
                        self._finish_forward(*item)
            for _ in self.bwd_threads:
                self.bwd_q.put(None)
            for _ in self.create_threads:
                self.create_q.put(None)
            for th in self.bwd_threads + self.create_threads:
                th.join()
        return requests


def request_work(req: Request) -> float:
    """Work of a request for shortest-remaining-work admission: its
    vehicle-steps, three times for a gradient request (forward, segment
    recomputation and reverse step)."""
    return float(req.vehicle_steps) * (3.0 if req.needs_grad else 1.0)


WORK_PER_SECOND = 5e10      # request_work units the engine completes per second (measured order)


def request_priority(req: Request, now: float) -> float:
    """Admission order (lower first): the request's work in seconds of engine
    time less the time it has waited since arrival, so that shortest work
    goes first but a long request overtakes newer short ones once it has
    waited about its own run time (no starvation)."""
    return request_work(req) / WORK_PER_SECOND - (now - req.arrival)


def latency_stats(reqs: List[Request]) -> dict:
    lat = np.array([r.finished - r.arrival for r in reqs])
    return dict(p50_s=float(np.percentile(lat, 50)), p99_s=float(np.percentile(lat, 99)),
                mean_s=float(lat.mean()), max_s=float(lat.max()))


def run_serial(requests: List[Request], device: int = 0, ckpt_every: int = 180) -> List[dict]:
    """Serial single-scenario execution in arrival order (each request alone,
    one after another), with the same arrival times."""
    t0 = time.perf_counter()
    out = []
    for req in sorted(requests, key=lambda r: r.arrival):
        now = time.perf_counter() - t0
        if now < req.arrival:
            time.sleep(req.arrival - now)
        res = run_request_alone(req, device=device, ckpt_every=ckpt_every)
        fin = time.perf_counter() - t0
        out.append(dict(rid=req.rid, arrival=req.arrival, finished=fin, result=res))
    return out


_NETWORK_CACHE = {}


def network_family(n_links: int, seed: int = 4):
    """A network of the serving family (same generator as the city workload,
    n_links / 3 nodes), with 1,000,000 vehicles to draw requests from; cached."""
    from . import scenario as S
    key = (n_links, seed)
    if key not in _NETWORK_CACHE:
        n_nodes = max(30, n_links // 3)
        zo = max(4, min(80, n_nodes // 150))
        zd = max(6, min(128, n_nodes // 94))
        _NETWORK_CACHE[key] = S.city(seed=seed + n_links, n_nodes=n_nodes, n_links=n_links, n_vehicles=1_000_000,
                                     T=3600, n_origin_zones=zo, n_dest_zones=zd, name=f"net{n_links}")
    return _NETWORK_CACHE[key]


def make_request_stream(n: int = 256, rate: float = 4.0, seed: int = 4,
                        sizes=(2000, 4500, 9000, 18000, 36000), n_range=(50_000, 1_000_000),
                        horizons=None, n_sensors: int = 200):
    """Poisson request stream: 50% one-hour nowcasts (3,600-step forward), 25%
    30-minute calibration gradients, 25% 30-minute control candidates (gradient
    w.r.t. link costs); networks drawn from the family, vehicle counts
    log-uniform over n_range.  Calibration targets are synthetic counts (a fixed
    Poisson draw per sensor and bin); control candidates get cost sensitivities
    beta ~ U(0, 5) and a target link."""
    from .scenario import _i32, _f32
    horizons = horizons or {"nowcast": 3600, "calibration": 1800, "control": 1800}
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for rid in range(n):
        t += rng.exponential(1.0 / rate)
        kind = rng.choice(["nowcast", "nowcast", "calibration", "control"])
        base = network_family(int(rng.choice(sizes)), seed)
        nv = int(np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1]))))
        idx = np.sort(rng.choice(base.N, size=min(nv, base.N), replace=False))
        T = horizons[kind]
        sc = base.copy(name=f"{kind}_{rid}", N=len(idx), origin=base.origin[idx], dest_zone=base.dest_zone[idx],
                       dep_step=base.dep_step[idx], od=base.od[idx], T=T, seed=1000 + rid, scenario_id=rid)
        req = Request(rid=rid, kind=str(kind), scenario=sc, arrival=t)
        if kind == "calibration":
            sens = _i32(np.sort(rng.choice(sc.L, size=min(n_sensors, sc.L), replace=False)))
            req.scenario = sc.copy(sensors=sens)
            nb = (T + sc.obs_every - 1) // sc.obs_every
            req.observed = rng.poisson(20.0, size=(nb, len(sens))).astype(np.float32)
        elif kind == "control":
            req.scenario = sc.copy(beta=_f32(rng.uniform(0.0, 5.0, size=sc.L)))
            req.target_link = int(rng.integers(0, sc.L))
        out.append(req)
    return out
