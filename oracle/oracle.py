"""ctypes front end of the CPU oracle (oracle/ts_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg.  The product path never imports this module.

``OracleSim(scenario, precision="fp64")`` runs the double-precision reference;
``precision="fp32"`` runs the same source built with float arithmetic, which takes
every floating-point decision in the kernel's precision (see the file header of
ts_oracle.c).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ts_oracle.c")
_LIBS = {"fp64": os.path.join(_HERE, "libts_oracle64.so"),
         "fp32": os.path.join(_HERE, "libts_oracle32.so")}
_lock = threading.Lock()
_loaded = {}


def build(force: bool = False) -> None:
    """Compile both oracle builds with gcc (plain -O2, no fast-math, no FMA
    contraction so float results follow IEEE single-precision operation by
    operation)."""
    for prec, out in _LIBS.items():
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", out + ".tmp", _SRC, "-lm"]
        if prec == "fp32":
            cmd.insert(1, "-DORACLE_FP32")
        subprocess.check_call(cmd)
        os.replace(out + ".tmp", out)


class _Scen(C.Structure):
    _fields_ = [("V", C.c_int32), ("L", C.c_int32), ("F", C.c_int32), ("Z", C.c_int32),
                ("N", C.c_int32), ("n_od", C.c_int32),
                ("tail", C.c_void_p), ("head", C.c_void_p),
                ("length", C.c_void_p), ("u", C.c_void_p), ("kappa", C.c_void_p),
                ("alpha", C.c_void_p), ("beta", C.c_void_p), ("cost", C.c_void_p),
                ("q_fx", C.c_void_p), ("phi", C.c_void_p), ("psi", C.c_void_p),
                ("w", C.c_void_p), ("node_zone", C.c_void_p), ("dest_feat", C.c_void_p),
                ("origin", C.c_void_p), ("dest_zone", C.c_void_p), ("dep_step", C.c_void_p),
                ("od", C.c_void_p), ("od_lambda", C.c_void_p),
                ("dt", C.c_float), ("dn", C.c_float), ("tau", C.c_float), ("M", C.c_float),
                ("eps_arr", C.c_float), ("eps_tag", C.c_float), ("alpha_origin", C.c_float),
                ("seed", C.c_uint64), ("scenario_id", C.c_uint32), ("obs_every", C.c_int32)]


def _lib(precision: str):
    with _lock:
        if precision not in _loaded:
            build()
            lib = C.CDLL(_LIBS[precision])
            P = C.c_void_p
            lib.or_create.restype = P
            lib.or_create.argtypes = [C.POINTER(_Scen), C.c_int]
            lib.or_reset.argtypes = [P, C.c_int32]
            lib.or_step.argtypes = [P]
            lib.or_run.argtypes = [P, C.c_int32]
            lib.or_time.argtypes = [P]
            lib.or_n_bins.argtypes = [P]
            lib.or_outputs.argtypes = [P] + [P] * 6
            lib.or_export_state.argtypes = [P] + [P] * 7
            lib.or_records.argtypes = [P] + [P] * 8
            lib.or_route.argtypes = [P, C.c_int32, P, P, C.c_int32]
            lib.or_error.restype = C.c_char_p
            lib.or_error.argtypes = [P]
            lib.or_destroy.argtypes = [P]
            lib.or_gumbel.restype = C.c_double
            lib.or_gumbel.argtypes = [C.c_uint64, C.c_uint32, C.c_int32, C.c_int32, C.c_int, C.c_int]
            lib.or_philox4x32_10.argtypes = [P, P, P]
            lib.or_backward.argtypes = [P, P, P, C.c_int] + [P] * 8
            lib.or_positions.argtypes = [P, P]
            lib.or_position_margins.argtypes = [P, P, P]
            lib.or_import_state.argtypes = [P, C.c_int32] + [P] * 7
            lib.or_choice_weights.restype = C.c_int32
            lib.or_choice_weights.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, C.c_double, P, P]
            lib.or_merge_weights.restype = C.c_int32
            lib.or_merge_weights.argtypes = [P, C.c_int32, C.c_int32, C.c_double, P, P, P]
            lib.or_log32.restype = C.c_float
            lib.or_log32.argtypes = [C.c_float]
            _loaded[precision] = lib
        return _loaded[precision]


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def philox4x32_10(ctr, key):
    lib = _lib("fp64")
    c = np.asarray(ctr, np.uint32).copy()
    k = np.asarray(key, np.uint32).copy()
    out = np.zeros(4, np.uint32)
    lib.or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def log32(x: float) -> float:
    return float(_lib("fp32").or_log32(C.c_float(x)))


def gumbel(seed, scen, vid, t, stream, slot, precision="fp64"):
    return float(_lib(precision).or_gumbel(seed, scen, vid, t, stream, slot))


class OracleSim:
    """One scenario in the oracle.  ``keep_history`` records every step for the
    reverse-mode pass."""

    def __init__(self, sc, precision: str = "fp64", keep_history: bool = False):
        self.sc = sc
        self.precision = precision
        self.lib = _lib(precision)
        self._keep = []

        def arr(a, dt):
            a = np.ascontiguousarray(np.asarray(a, dt))
            self._keep.append(a)
            return _p(a)

        s = _Scen()
        s.V, s.L, s.F, s.Z, s.N, s.n_od = sc.V, sc.L, sc.F, sc.Z, sc.N, sc.n_od
        s.tail, s.head = arr(sc.tail, np.int32), arr(sc.head, np.int32)
        s.length, s.u, s.kappa = arr(sc.length, np.float32), arr(sc.u, np.float32), arr(sc.kappa, np.float32)
        s.alpha, s.beta, s.cost = arr(sc.alpha, np.float32), arr(sc.beta, np.float32), arr(sc.cost, np.float32)
        s.q_fx = arr(sc.q_fx, np.int32)
        s.phi, s.psi, s.w = arr(sc.phi, np.float32), arr(sc.psi, np.float32), arr(sc.w, np.float32)
        s.node_zone, s.dest_feat = arr(sc.node_zone, np.int32), arr(sc.dest_feat, np.float32)
        s.origin, s.dest_zone = arr(sc.origin, np.int32), arr(sc.dest_zone, np.int32)
        s.dep_step, s.od = arr(sc.dep_step, np.int32), arr(sc.od, np.int32)
        s.od_lambda = arr(sc.od_lambda, np.float32)
        s.dt, s.dn, s.tau, s.M = sc.dt, sc.dn, sc.tau, sc.M
        s.eps_arr, s.eps_tag, s.alpha_origin = sc.eps_arr, sc.eps_tag, sc.alpha_origin
        s.seed, s.scenario_id, s.obs_every = sc.seed, sc.scenario_id, sc.obs_every
        self._s = s
        self.h = self.lib.or_create(C.byref(s), 1 if keep_history else 0)
        self.T = None

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.or_destroy(h)
            self.h = None

    def _check(self, rc):
        if rc != 0:
            raise RuntimeError("oracle: " + self.lib.or_error(self.h).decode())

    def reset(self, T=None):
        self.T = self.sc.T if T is None else T
        self._check(self.lib.or_reset(self.h, self.T))

    def step(self, n=1):
        self._check(self.lib.or_run(self.h, n))

    @property
    def t(self):
        return self.lib.or_time(self.h)

    def rollout(self, T=None):
        self.reset(T)
        self.step(self.T)
        return self.outputs()

    def outputs(self):
        sc, T = self.sc, self.T
        nb = self.lib.or_n_bins(self.h)
        counts = np.zeros((nb, sc.L), np.int32)
        speed = np.zeros((nb, sc.L), np.float64)
        tt = np.zeros((nb, sc.L), np.float64)
        nw, non, na = (np.zeros(T + 1, np.int64) for _ in range(3))
        self.lib.or_outputs(self.h, _p(counts), _p(speed), _p(tt), _p(nw), _p(non), _p(na))
        return dict(counts=counts, speed=speed, travel_time=tt, n_waiting=nw, n_on=non, n_arrived=na)

    def state(self):
        sc = self.sc
        d = dict(veh_link=np.zeros(sc.N, np.int32), veh_pos=np.zeros(sc.N, np.float64),
                 veh_rank=np.zeros(sc.N, np.int32), veh_entry=np.zeros(sc.N, np.int32),
                 link_credit=np.zeros(sc.L, np.int64), link_exits=np.zeros(sc.L, np.int64),
                 fifo_off=np.zeros(sc.V, np.int32))
        self.lib.or_export_state(self.h, *(_p(d[k]) for k in ("veh_link", "veh_pos", "veh_rank", "veh_entry",
                                                              "link_credit", "link_exits", "fifo_off")))
        return d

    def records(self):
        """Decisions of the last step, with the margins that flag near-ties:
        top-2 key gaps of each link / origin-node choice and of each merge, and
        the distances of each link's leader from the arrival line
        (arr_margin) and of its rearmost vehicle from the jam spacing
        (vac_margin), all after car-following."""
        sc = self.sc
        d = dict(link_cand=np.zeros(sc.L, np.int32), link_target=np.zeros(sc.L, np.int32),
                 node_cand=np.zeros(sc.V, np.int32), node_target=np.zeros(sc.V, np.int32),
                 link_in=np.zeros(sc.L, np.int32), link_margin=np.zeros(sc.L),
                 node_margin=np.zeros(sc.V), merge_margin=np.zeros(sc.L),
                 arr_margin=np.zeros(sc.L), vac_margin=np.zeros(sc.L))
        self.lib.or_records(self.h, *(_p(d[k]) for k in ("link_cand", "link_target", "node_cand", "node_target",
                                                         "link_in", "link_margin", "node_margin", "merge_margin")))
        self.lib.or_position_margins(self.h, _p(d["arr_margin"]), _p(d["vac_margin"]))
        return d

    def set_state(self, state: dict, t: int):
        """Continue from a given state at step t (the layout of state(); a run
        without history).  The observation bin containing t restarts at t."""
        a = dict(veh_link=np.ascontiguousarray(state["veh_link"], np.int32),
                 veh_pos=np.ascontiguousarray(state["veh_pos"], np.float64),
                 veh_rank=np.ascontiguousarray(state["veh_rank"], np.int32),
                 veh_entry=np.ascontiguousarray(state["veh_entry"], np.int32),
                 link_credit=np.ascontiguousarray(state["link_credit"], np.int64),
                 link_exits=np.ascontiguousarray(state["link_exits"], np.int64),
                 fifo_off=np.ascontiguousarray(state["fifo_off"], np.int32))
        self._check(self.lib.or_import_state(self.h, int(t), *(_p(a[k]) for k in (
            "veh_link", "veh_pos", "veh_rank", "veh_entry", "link_credit", "link_exits", "fifo_off"))))

    def choice_weights(self, t, tau, link=-1, node=-1):
        """Relaxed link-choice weights softmax((V + g)/tau) of the candidate at
        source link ``link`` (or origin node ``node``) at step t of the recorded
        rollout, and the slot the forward chose; None when it made no choice."""
        pi = np.zeros(64)
        slot = np.zeros(1, np.int32)
        n = self.lib.or_choice_weights(self.h, int(t), int(link), int(node), float(tau), _p(pi), _p(slot))
        if n < 0:
            raise RuntimeError("oracle: choice weights need a recorded rollout")
        return None if n == 0 else (pi[:n].copy(), int(slot[0]))

    def merge_weights(self, t, m, tau):
        """Relaxed merge weights softmax((alpha_src + g')/tau) of the valid
        candidates of link m at step t, with their vehicle ids and win flags."""
        cap = self.sc.L + self.sc.V
        w, vid, won = np.zeros(cap), np.zeros(cap, np.int32), np.zeros(cap, np.int32)
        n = self.lib.or_merge_weights(self.h, int(t), int(m), float(tau), _p(w), _p(vid), _p(won))
        if n < 0:
            raise RuntimeError("oracle: merge weights need a recorded rollout")
        return w[:n].copy(), vid[:n].copy(), won[:n].astype(bool)

    def backward(self, ybar, xbarT=None, no_tg=False):
        """Reverse mode of the last rollout (needs keep_history=True).  ybar:
        [n_bins, L] adjoint of the bin counts; xbarT: optional [N] adjoint of the
        final positions.  Returns a dict of parameter gradients (float64)."""
        sc = self.sc
        yb = np.ascontiguousarray(np.asarray(ybar, np.float64))
        xb = None if xbarT is None else np.ascontiguousarray(np.asarray(xbarT, np.float64))
        g = dict(u=np.zeros(sc.L), kappa=np.zeros(sc.L), alpha=np.zeros(sc.L), alpha_origin=np.zeros(1),
                 beta=np.zeros(sc.L), cost=np.zeros(sc.L), w=np.zeros(sc.F), od_lambda=np.zeros(sc.n_od))
        rc = self.lib.or_backward(self.h, _p(yb), _p(xb), 1 if no_tg else 0,
                                  *(_p(g[k]) for k in ("u", "kappa", "alpha", "alpha_origin", "beta", "cost",
                                                       "w", "od_lambda")))
        self._check(rc)
        return g

    def positions(self):
        x = np.zeros(self.sc.N, np.float64)
        self.lib.or_positions(self.h, _p(x))
        return x

    def route(self, i):
        n = self.lib.or_route(self.h, i, None, None, 0)
        steps = np.zeros(n, np.int32)
        links = np.zeros(n, np.int32)
        self.lib.or_route(self.h, i, _p(steps), _p(links), n)
        return steps, links
