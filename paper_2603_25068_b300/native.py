"""ctypes binding of libtrafficsim.so (include/trafficsim.h).

Argument marshalling only: every step of the simulation runs in the CUDA
kernels of the library.  There is no CPU fallback; importing this module on a
machine without the built library raises.
"""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB

SIM_OK, SIM_EINVAL, SIM_ENOMEM, SIM_ECUDA, SIM_ETIMEOUT, SIM_ESTATE, SIM_EOVERFLOW = range(7)
FX_ONE = 65536

P = C.c_void_p


class sim_network(C.Structure):
    _fields_ = [("V", C.c_int32), ("L", C.c_int32), ("tail", P), ("head", P), ("length", P),
                ("q_fx", P), ("F", C.c_int32), ("phi", P), ("psi", P), ("Z", C.c_int32),
                ("node_zone", P), ("dest_feat", P)]


class sim_demand(C.Structure):
    _fields_ = [("N", C.c_int32), ("origin", P), ("dest_zone", P), ("dep_step", P), ("od", P),
                ("n_od", C.c_int32), ("od_lambda", P)]


class sim_params(C.Structure):
    _fields_ = [("u", P), ("kappa", P), ("alpha", P), ("beta", P), ("cost", P), ("w", P),
                ("alpha_origin", C.c_float)]


class sim_options(C.Structure):
    _fields_ = [("dt", C.c_float), ("dn", C.c_float), ("tau_gumbel", C.c_float), ("M", C.c_float),
                ("eps_arr", C.c_float), ("eps_tag", C.c_float), ("seed", C.c_uint64),
                ("scenario_id", C.c_uint32), ("obs_every", C.c_int32), ("ckpt_every", C.c_int32),
                ("route_cap", C.c_int32), ("device", C.c_int32), ("stream", P)]


class sim_outputs(C.Structure):
    _fields_ = [("counts", P), ("speed", P), ("travel_time", P), ("n_waiting", P), ("n_on", P),
                ("n_arrived", P), ("on_device", C.c_int32)]


class sim_grads(C.Structure):
    _fields_ = [("d_u", P), ("d_kappa", P), ("d_alpha", P), ("d_beta", P), ("d_cost", P),
                ("d_w", P), ("d_alpha_origin", P), ("d_od_lambda", P), ("on_device", C.c_int32)]


class sim_state_view(C.Structure):
    _fields_ = [("veh_link", P), ("veh_pos", P), ("veh_rank", P), ("veh_entry", P),
                ("link_credit", P), ("link_exits", P), ("fifo_off", P)]


class sim_records(C.Structure):
    _fields_ = [("link_cand", P), ("link_target", P), ("node_cand", P), ("node_target", P),
                ("link_in", P)]


# every symbol declared in include/trafficsim.h, with its ctypes signature
SIGNATURES = {
    "sim_n_bins": (C.c_int32, [C.c_int32, C.c_int32]),
    "sim_create": (C.c_int, [C.POINTER(sim_network), C.POINTER(sim_demand), C.POINTER(sim_params),
                             C.POINTER(sim_options), C.POINTER(P)]),
    "sim_set_params": (C.c_int, [P, C.POINTER(sim_params)]),
    "sim_set_params_device": (C.c_int, [P, C.POINTER(sim_params), P]),
    "sim_reset": (C.c_int, [P, C.c_int32]),
    "sim_step": (C.c_int, [P, C.c_int32]),
    "sim_rollout": (C.c_int, [P, C.c_int32, C.POINTER(sim_outputs)]),
    "sim_step_counters": (C.c_int, [P, P]),
    "sim_profile_rollout": (C.c_int, [P, C.c_int32, C.POINTER(sim_outputs), P, P]),
    "sim_get_outputs": (C.c_int, [P, C.POINTER(sim_outputs)]),
    "sim_backward": (C.c_int, [P, P, P, C.c_int32, C.POINTER(sim_grads)]),
    "sim_get_state": (C.c_int, [P, C.POINTER(sim_state_view)]),
    "sim_get_records": (C.c_int, [P, C.POINTER(sim_records)]),
    "sim_set_state": (C.c_int, [P, C.POINTER(sim_state_view), C.c_int32]),
    "sim_set_stage": (C.c_int, [P, C.c_int32]),
    "sim_set_stream": (C.c_int, [P, P]),
    "sim_get_stream": (C.c_void_p, [P]),
    "sim_set_executor": (C.c_int, [P, C.c_int32]),
    "sim_get_executor": (C.c_int32, [P]),
    "sim_test_barrier_timeout": (C.c_int, [P, C.c_int32]),
    "sim_set_partition_weights": (C.c_int, [P, P]),
    "sim_persist_groups": (C.c_int32, [P, P]),
    "sim_batch_create": (C.c_int, [C.POINTER(P), C.c_int32, C.POINTER(P)]),
    "sim_batch_start": (C.c_int, [P, C.c_int32, C.c_int32]),
    "sim_batch_advance": (C.c_int, [P, C.c_int32, P]),
    "sim_batch_rollout": (C.c_int, [P, C.c_int32]),
    "sim_batch_destroy": (C.c_int, [P]),
    "sim_release_cached_memory": (C.c_int, [C.c_int32]),
    "sim_set_recompute": (C.c_int, [P, C.c_int32]),
    "sim_batch_set_executor": (C.c_int, [P, C.c_int32]),
    "sim_batch_get_executor": (C.c_int32, [P]),
    "sim_batch_test_barrier_timeout": (C.c_int, [P, C.c_int32]),
    "sim_batch_last_error": (C.c_char_p, [P]),
    "sim_rollout_static": (C.c_int, [C.POINTER(sim_network), C.POINTER(sim_demand), C.POINTER(sim_params),
                                     C.POINTER(sim_options), C.c_int32, C.POINTER(sim_outputs)]),
    "sim_time": (C.c_int32, [P]),
    "sim_device_bytes": (C.c_size_t, [P]),
    "sim_destroy": (C.c_int, [P]),
    "sim_last_error": (C.c_char_p, [P]),
}

_lib = None


def lib():
    """Load libtrafficsim.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is missing: run `python -m paper_2603_25068_b300.build`")
        L = C.CDLL(LIB)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class SimError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[code {code}] {msg}")
        self.code = code


def check(rc, h=None):
    if rc != SIM_OK:
        msg = lib().sim_last_error(h)
        raise SimError(rc, msg.decode() if msg else "")
