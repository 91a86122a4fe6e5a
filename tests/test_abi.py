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
