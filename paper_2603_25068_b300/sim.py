"""Python front end of the CUDA simulator (marshalling only).

    sim = Simulator(scenario)          # copies the scenario to the GPU
    out = sim.rollout()                # dict of numpy arrays (host)
    out = sim.rollout(device=True)     # dict of torch CUDA tensors, async on sim.stream
"""
from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np

from . import native as nat


def _p(a):
    return C.c_void_p(a.ctypes.data) if a is not None else None


class Simulator:
    def __init__(self, sc, device: int = 0, stream=None, ckpt_every: int = 0, route_cap: int = 64):
        self.sc = sc
        self.lib = nat.lib()
        self._keep = []
        a = self._arr
        net = nat.sim_network(V=sc.V, L=sc.L, tail=a(sc.tail, np.int32), head=a(sc.head, np.int32),
                              length=a(sc.length, np.float32), q_fx=a(sc.q_fx, np.int32), F=sc.F,
                              phi=a(sc.phi, np.float32), psi=a(sc.psi, np.float32), Z=sc.Z,
                              node_zone=a(sc.node_zone, np.int32), dest_feat=a(sc.dest_feat, np.float32))
        dem = nat.sim_demand(N=sc.N, origin=a(sc.origin, np.int32), dest_zone=a(sc.dest_zone, np.int32),
                             dep_step=a(sc.dep_step, np.int32), od=a(sc.od, np.int32), n_od=sc.n_od,
                             od_lambda=a(sc.od_lambda, np.float32))
        par = self._params(sc.u, sc.kappa, sc.alpha, sc.beta, sc.cost, sc.w, sc.alpha_origin)
        if stream is not None and not isinstance(stream, int):
            stream = stream.cuda_stream
        self.stream_ptr = stream
        opt = nat.sim_options(dt=sc.dt, dn=sc.dn, tau_gumbel=sc.tau, M=sc.M, eps_arr=sc.eps_arr,
                              eps_tag=sc.eps_tag, seed=sc.seed, scenario_id=sc.scenario_id,
                              obs_every=sc.obs_every, ckpt_every=ckpt_every, route_cap=route_cap,
                              device=device, stream=stream)
        h = C.c_void_p()
        rc = self.lib.sim_create(C.byref(net), C.byref(dem), C.byref(par), C.byref(opt), C.byref(h))
        nat.check(rc, None)
        self.h = h
        self.device = device
        self.T = None
        self._keep = []

    def _arr(self, x, dt):
        x = np.ascontiguousarray(np.asarray(x, dt))
        self._keep.append(x)
        return _p(x)

    def _params(self, u, kappa, alpha, beta, cost, w, alpha_origin):
        a = self._arr
        return nat.sim_params(u=a(u, np.float32), kappa=a(kappa, np.float32), alpha=a(alpha, np.float32),
                              beta=a(beta, np.float32), cost=a(cost, np.float32), w=a(w, np.float32),
                              alpha_origin=float(alpha_origin))

    def close(self):
        if getattr(self, "h", None):
            self.lib.sim_destroy(self.h)
            self.h = None

    __del__ = close

    def _check(self, rc):
        nat.check(rc, self.h)

    # ------------------------------------------------------------------ params
    def set_params(self, u=None, kappa=None, alpha=None, beta=None, cost=None, w=None, alpha_origin=None):
        sc = self.sc
        self._keep = []
        par = self._params(sc.u if u is None else u, sc.kappa if kappa is None else kappa,
                           sc.alpha if alpha is None else alpha, sc.beta if beta is None else beta,
                           sc.cost if cost is None else cost, sc.w if w is None else w,
                           sc.alpha_origin if alpha_origin is None else alpha_origin)
        self._check(self.lib.sim_set_params(self.h, C.byref(par)))
        self._keep = []

    def set_params_device(self, u, kappa, alpha, beta, cost, w, alpha_origin):
        """Replace the parameters from torch CUDA tensors on the simulator's
        device (float32; alpha_origin a one-element tensor) without a host
        round trip: the copies are enqueued on the simulator's stream, which the
        caller orders after the tensors' producer.  The tensors must stay alive
        until that stream has passed this call."""
        import torch
        dev = torch.device("cuda", self.device)
        ts = [t.detach() for t in (u, kappa, alpha, beta, cost, w, alpha_origin)]
        for t, n in zip(ts, (self.sc.L,) * 5 + (self.sc.F, 1)):
            if t.device != dev or t.dtype != torch.float32 or not t.is_contiguous() or t.numel() != n:
                raise ValueError("device parameters: contiguous float32 tensors of the simulator's device "
                                 "with one entry per link (w: per feature, alpha_origin: one)")
        par = nat.sim_params(*(C.c_void_p(t.data_ptr()) for t in ts[:6]), alpha_origin=0.0)
        self._check(self.lib.sim_set_params_device(self.h, C.byref(par), C.c_void_p(ts[6].data_ptr())))
        self._dev_params = ts          # alive until the next call replaces them

    # ------------------------------------------------------------------ running
    def n_bins(self, T=None):
        return self.lib.sim_n_bins(self.sc.T if T is None else T, self.sc.obs_every)

    def reset(self, T=None):
        self.T = self.sc.T if T is None else T
        self._check(self.lib.sim_reset(self.h, self.T))

    def step(self, n=1):
        self._check(self.lib.sim_step(self.h, n))

    @property
    def t(self):
        return self.lib.sim_time(self.h)

    def set_stream(self, stream):
        """Move the handle's work to another stream (torch.cuda.Stream or handle)."""
        if stream is not None and not isinstance(stream, int):
            stream = stream.cuda_stream
        self._check(self.lib.sim_set_stream(self.h, stream))
        self.stream_ptr = stream

    def torch_stream(self):
        """The handle's stream as a torch stream (for ordering torch work
        before or after the simulator's device work)."""
        import torch
        ptr = self.lib.sim_get_stream(self.h)
        if not ptr:
            return torch.cuda.default_stream(self.device)
        return torch.cuda.ExternalStream(ptr, device=torch.device("cuda", self.device))

    def device_bytes(self):
        return self.lib.sim_device_bytes(self.h)

    def set_partition_weights(self, w=None):
        """Per-link weights of the persistent executor's work partition (host
        array of L, relative; None restores queue capacity + 16).  Results are
        unchanged; only which CTA owns which links moves."""
        if w is None:
            self._check(self.lib.sim_set_partition_weights(self.h, None))
            return
        w = np.ascontiguousarray(np.asarray(w, np.float32))
        if w.shape != (self.sc.L,):
            raise ValueError(f"partition weights need shape ({self.sc.L},), got {w.shape}")
        self._check(self.lib.sim_set_partition_weights(self.h, _p(w)))

    def persist_groups(self):
        """First link of each CTA's group (G + 1 bounds), or None when the
        persistent executor is unavailable."""
        G = self.lib.sim_persist_groups(self.h, None)
        if G < 0:
            self._check(-1)
        if G == 0:
            return None
        b = np.zeros(G + 1, np.int32)
        if self.lib.sim_persist_groups(self.h, _p(b)) != G:
            raise RuntimeError("sim_persist_groups failed")
        return b

    RECOMPUTE = {"overlap": 0, "serial": 1}

    def set_recompute(self, name: str):
        """Segment recomputation of the reverse pass: "overlap" (beside the
        reverse kernels, two tape sets) or "serial" (one persistent recording
        launch per segment, one tape set).  Gradients do not depend on it."""
        self._check(self.lib.sim_set_recompute(self.h, self.RECOMPUTE[name]))

    EXECUTORS = {"auto": 0, "step": 1, "persistent": 2}

    def set_executor(self, name: str):
        """Forward executor: "auto", "step" (two kernels per step, graph per
        horizon) or "persistent" (one cooperative launch per run)."""
        self._check(self.lib.sim_set_executor(self.h, self.EXECUTORS[name]))

    @property
    def executor(self) -> str:
        """Executor the next forward run uses ("step" or "persistent")."""
        return {1: "step", 2: "persistent"}[self.lib.sim_get_executor(self.h)]

    def rollout(self, T: Optional[int] = None, device: bool = False, out=None):
        """Run a whole rollout.  With device=True the outputs are torch CUDA
        tensors written asynchronously on the simulator's stream (``out`` may
        supply preallocated ones)."""
        T = self.sc.T if T is None else T
        self.T = T
        nb, L = self.n_bins(T), self.sc.L
        if device:
            import torch
            dev = torch.device("cuda", self.device)
            if out is None:
                out = dict(counts=torch.empty((nb, L), dtype=torch.int32, device=dev),
                           speed=torch.empty((nb, L), dtype=torch.float32, device=dev),
                           travel_time=torch.empty((nb, L), dtype=torch.float32, device=dev))
            o = nat.sim_outputs(counts=C.c_void_p(out["counts"].data_ptr()),
                                speed=C.c_void_p(out["speed"].data_ptr()),
                                travel_time=C.c_void_p(out["travel_time"].data_ptr()), on_device=1)
            self._check(self.lib.sim_rollout(self.h, T, C.byref(o)))
            return out
        res = dict(counts=np.zeros((nb, L), np.int32), speed=np.zeros((nb, L), np.float32),
                   travel_time=np.zeros((nb, L), np.float32), n_waiting=np.zeros(T + 1, np.int64),
                   n_on=np.zeros(T + 1, np.int64), n_arrived=np.zeros(T + 1, np.int64))
        o = nat.sim_outputs(*(_p(res[k]) for k in ("counts", "speed", "travel_time", "n_waiting",
                                                   "n_on", "n_arrived")), 0)
        self._check(self.lib.sim_rollout(self.h, T, C.byref(o)))
        return res

    def outputs(self):
        """Outputs of the run so far (a rollout, or reset + steps)."""
        T = self.T
        nb, L = self.n_bins(T), self.sc.L
        res = dict(counts=np.zeros((nb, L), np.int32), speed=np.zeros((nb, L), np.float32),
                   travel_time=np.zeros((nb, L), np.float32), n_waiting=np.zeros(T + 1, np.int64),
                   n_on=np.zeros(T + 1, np.int64), n_arrived=np.zeros(T + 1, np.int64))
        o = nat.sim_outputs(*(_p(res[k]) for k in ("counts", "speed", "travel_time", "n_waiting",
                                                   "n_on", "n_arrived")), 0)
        self._check(self.lib.sim_get_outputs(self.h, C.byref(o)))
        return res

    def backward(self, dL_dcounts, dL_dxT=None):
        """Gradient of sum(dL_dcounts * counts) (+ sum(dL_dxT * final positions))
        with respect to the parameters, through the last rollout (needs
        ckpt_every > 0).  Host arrays in, dict of float32 numpy arrays out."""
        sc = self.sc
        yb = np.ascontiguousarray(np.asarray(dL_dcounts, np.float32))
        xb = None if dL_dxT is None else np.ascontiguousarray(np.asarray(dL_dxT, np.float32))
        g = dict(u=np.zeros(sc.L, np.float32), kappa=np.zeros(sc.L, np.float32), alpha=np.zeros(sc.L, np.float32),
                 beta=np.zeros(sc.L, np.float32), cost=np.zeros(sc.L, np.float32), w=np.zeros(sc.F, np.float32),
                 alpha_origin=np.zeros(1, np.float32), od_lambda=np.zeros(sc.n_od, np.float32))
        o = nat.sim_grads(*(_p(g[k]) for k in ("u", "kappa", "alpha", "beta", "cost", "w", "alpha_origin",
                                               "od_lambda")), 0)
        self._check(self.lib.sim_backward(self.h, _p(yb), _p(xb), 0, C.byref(o)))
        return g

    def backward_device(self, dL_dcounts, dL_dxT=None):
        """As backward() with torch CUDA tensors in and out (no host copies of
        the gradients)."""
        import torch
        sc = self.sc
        dev = torch.device("cuda", self.device)
        yb = dL_dcounts.to(device=dev, dtype=torch.float32).contiguous()
        xb = None if dL_dxT is None else dL_dxT.to(device=dev, dtype=torch.float32).contiguous()
        g = dict(u=torch.empty(sc.L, device=dev), kappa=torch.empty(sc.L, device=dev),
                 alpha=torch.empty(sc.L, device=dev), beta=torch.empty(sc.L, device=dev),
                 cost=torch.empty(sc.L, device=dev), w=torch.empty(sc.F, device=dev),
                 alpha_origin=torch.empty(1, device=dev), od_lambda=torch.empty(sc.n_od, device=dev))
        o = nat.sim_grads(*(C.c_void_p(g[k].data_ptr()) for k in ("u", "kappa", "alpha", "beta", "cost", "w",
                                                                   "alpha_origin", "od_lambda")), 1)
        self._check(self.lib.sim_backward(self.h, C.c_void_p(yb.data_ptr()),
                                          None if xb is None else C.c_void_p(xb.data_ptr()), 1, C.byref(o)))
        return g

    def state(self, fields=None):
        """Exported state as host arrays; ``fields`` (names) limits the copy."""
        sc = self.sc
        d = dict(veh_link=np.zeros(sc.N, np.int32), veh_pos=np.zeros(sc.N, np.float64),
                 veh_rank=np.zeros(sc.N, np.int32), veh_entry=np.zeros(sc.N, np.int32),
                 link_credit=np.zeros(sc.L, np.int64), link_exits=np.zeros(sc.L, np.int64),
                 fifo_off=np.zeros(sc.V, np.int32))
        if fields is not None:
            d = {k: d[k] for k in fields}
        v = nat.sim_state_view(*(_p(d.get(k)) for k in ("veh_link", "veh_pos", "veh_rank", "veh_entry",
                                                        "link_credit", "link_exits", "fifo_off")))
        self._check(self.lib.sim_get_state(self.h, C.byref(v)))
        return d

    def set_state(self, state: dict, t: int):
        """Continue from a given state at step t (the dict layout of state(),
        e.g. the oracle's); the next step() runs step t."""
        sc = self.sc
        arrs = dict(veh_link=np.ascontiguousarray(state["veh_link"], np.int32),
                    veh_pos=np.ascontiguousarray(state["veh_pos"], np.float64),
                    veh_rank=np.ascontiguousarray(state["veh_rank"], np.int32),
                    veh_entry=np.ascontiguousarray(state["veh_entry"], np.int32),
                    link_credit=np.ascontiguousarray(state["link_credit"], np.int64),
                    link_exits=np.ascontiguousarray(state["link_exits"], np.int64),
                    fifo_off=np.ascontiguousarray(state["fifo_off"], np.int32))
        v = nat.sim_state_view(*(_p(arrs[k]) for k in ("veh_link", "veh_pos", "veh_rank", "veh_entry",
                                                        "link_credit", "link_exits", "fifo_off")))
        self._check(self.lib.sim_set_state(self.h, C.byref(v), int(t)))

    def records(self):
        sc = self.sc
        d = dict(link_cand=np.zeros(sc.L, np.int32), link_target=np.zeros(sc.L, np.int32),
                 node_cand=np.zeros(sc.V, np.int32), node_target=np.zeros(sc.V, np.int32),
                 link_in=np.zeros(sc.L, np.int32))
        r = nat.sim_records(*(_p(d[k]) for k in ("link_cand", "link_target", "node_cand",
                                                  "node_target", "link_in")))
        self._check(self.lib.sim_get_records(self.h, C.byref(r)))
        return d


def static_arguments(sc, T: int, device: int = 0, stream=None):
    """The ctypes structures sim_rollout_static takes for scenario ``sc``
    (host arrays), with the list of arrays that must stay alive while they
    are in use: (net, dem, par, opt, keep)."""
    keep = []

    def a(x, dt):
        x = np.ascontiguousarray(np.asarray(x, dt))
        keep.append(x)
        return _p(x)

    net = nat.sim_network(V=sc.V, L=sc.L, tail=a(sc.tail, np.int32), head=a(sc.head, np.int32),
                          length=a(sc.length, np.float32), q_fx=a(sc.q_fx, np.int32), F=sc.F,
                          phi=a(sc.phi, np.float32), psi=a(sc.psi, np.float32), Z=sc.Z,
                          node_zone=a(sc.node_zone, np.int32), dest_feat=a(sc.dest_feat, np.float32))
    dem = nat.sim_demand(N=sc.N, origin=a(sc.origin, np.int32), dest_zone=a(sc.dest_zone, np.int32),
                         dep_step=a(sc.dep_step, np.int32), od=a(sc.od, np.int32), n_od=sc.n_od,
                         od_lambda=a(sc.od_lambda, np.float32))
    par = nat.sim_params(u=a(sc.u, np.float32), kappa=a(sc.kappa, np.float32), alpha=a(sc.alpha, np.float32),
                         beta=a(sc.beta, np.float32), cost=a(sc.cost, np.float32), w=a(sc.w, np.float32),
                         alpha_origin=float(sc.alpha_origin))
    if stream is not None and not isinstance(stream, int):
        stream = stream.cuda_stream
    opt = nat.sim_options(dt=sc.dt, dn=sc.dn, tau_gumbel=sc.tau, M=sc.M, eps_arr=sc.eps_arr,
                          eps_tag=sc.eps_tag, seed=sc.seed, scenario_id=sc.scenario_id,
                          obs_every=sc.obs_every, ckpt_every=0, route_cap=0, device=device, stream=stream)
    return net, dem, par, opt, keep


def rollout_static(sc, T: Optional[int] = None, device: int = 0, stream=None):
    """Forward rollout through sim_rollout_static, the entry point that allocates
    no device memory (for callers that may not allocate: plug-ins whose host
    application owns every device allocation, real-time loops that must not
    block in cudaMalloc).  Host outputs."""
    lib = nat.lib()
    T = sc.T if T is None else T
    net, dem, par, opt, keep = static_arguments(sc, T, device, stream)
    nb = lib.sim_n_bins(T, sc.obs_every)
    res = dict(counts=np.zeros((nb, sc.L), np.int32), speed=np.zeros((nb, sc.L), np.float32),
               travel_time=np.zeros((nb, sc.L), np.float32), n_waiting=np.zeros(T + 1, np.int64),
               n_on=np.zeros(T + 1, np.int64), n_arrived=np.zeros(T + 1, np.int64))
    o = nat.sim_outputs(*(_p(res[k]) for k in ("counts", "speed", "travel_time", "n_waiting",
                                               "n_on", "n_arrived")), 0)
    rc = lib.sim_rollout_static(C.byref(net), C.byref(dem), C.byref(par), C.byref(opt), T, C.byref(o))
    if rc != nat.SIM_OK:
        raise nat.SimError(rc, "sim_rollout_static failed")
    return res
