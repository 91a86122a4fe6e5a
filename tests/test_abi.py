"""The C-ABI library loads and exports every symbol include/trafficsim.h declares
(no GPU needed: nothing is called that touches a device)."""
import ctypes
import os
import re

from paper_2603_25068_b300 import build, native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "trafficsim.h")).read()
    return sorted(set(re.findall(r"SIM_API\s+[\w\s\*]+?\b(sim_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("sim_create", "sim_step", "sim_rollout", "sim_backward", "sim_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    build.build()
    lib = ctypes.CDLL(build.LIB)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert set(declared_symbols()) <= set(native.SIGNATURES), "binding misses a declared entry point"


def test_pure_host_entry_points():
    lib = native.lib()
    assert lib.sim_n_bins(300, 300) == 1
    assert lib.sim_n_bins(301, 300) == 2
    assert lib.sim_n_bins(0, 300) == 0
    # NULL handle: reported, not crashed
    assert lib.sim_destroy(None) == 0
    assert lib.sim_time(None) == -1
    assert lib.sim_step(None, 1) == native.SIM_EINVAL


def test_static_rollout_checks_arguments_before_any_device_work():
    """sim_rollout_static rejects bad arguments and sizes beyond its limits on
    the host, before it touches a device (so this runs without a GPU)."""
    import ctypes as C
    import numpy as np
    from paper_2603_25068_b300 import scenario as S
    from paper_2603_25068_b300.sim import static_arguments
    lib = native.lib()
    sc = S.tiny_grid(n_vehicles=20, T=10)

    def call(T=10, on_device=0, counters=True, **edit):
        net, dem, par, opt, keep = static_arguments(sc, T)
        for k, v in edit.items():
            obj, field = k.split("__")
            setattr(dict(net=net, dem=dem, par=par, opt=opt)[obj], field, v)
        n = np.zeros(T + 1, np.int64)
        out = native.sim_outputs(None, None, None, n.ctypes.data if counters else None, None, None, on_device)
        return lib.sim_rollout_static(C.byref(net), C.byref(dem), C.byref(par), C.byref(opt), T, C.byref(out))

    assert call(net__phi=None) == native.SIM_EINVAL               # F > 0 needs phi, psi and w
    assert call(net__psi=None) == native.SIM_EINVAL
    assert call(par__w=None) == native.SIM_EINVAL
    assert call(par__kappa=None) == native.SIM_EINVAL
    assert call(dem__origin=None) == native.SIM_EINVAL
    assert call(on_device=1) == native.SIM_EINVAL                 # counters are summed on the host
    assert call(T=0) == native.SIM_EINVAL
    assert call(T=8193) == native.SIM_EOVERFLOW                   # beyond the step limit
    assert call(dem__N=70000) == native.SIM_EOVERFLOW             # beyond the vehicle limit
    assert lib.sim_rollout_static(None, None, None, None, 10, None) == native.SIM_EINVAL
