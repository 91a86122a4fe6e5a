"""The allocation-free rollout entry point (sim_rollout_static) against the
ordinary one (sim_create + sim_rollout).

sim_rollout_static exists for callers that may not allocate device memory:
plug-ins inside a host application whose memory manager owns every device
allocation, and real-time loops where cudaMalloc / cudaFree could block the
host and synchronise the device.  It keeps all state in one fixed device array
shared by every call, so two calls in a row must each re-initialise it, give
the same outputs as the ordinary path, and leave the device's free memory as
it was.  This file is collected last so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2603_25068_b300 import scenario as S

pytestmark = pytest.mark.gpu


def _outputs_match(a, b, T):
    np.testing.assert_array_equal(a["counts"], b["counts"])
    for k in ("n_waiting", "n_on", "n_arrived"):
        np.testing.assert_array_equal(a[k], b[k][:T + 1], err_msg=k)
    np.testing.assert_allclose(a["travel_time"], b["travel_time"], rtol=1e-6, atol=0)
    np.testing.assert_allclose(a["speed"], b["speed"], rtol=1e-4, atol=1e-5)


@pytest.mark.parametrize("make", [lambda: S.tiny_grid(), lambda: S.city_small()])
def test_static_rollout_matches_ordinary_rollout_twice(make):
    import torch
    assert torch.cuda.is_available()
    from paper_2603_25068_b300.sim import Simulator, rollout_static
    sc = make()
    g = Simulator(sc)
    ref = g.rollout()
    g.close()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(0)[0]
    first = rollout_static(sc)
    free1 = torch.cuda.mem_get_info(0)[0]
    second = rollout_static(sc)
    free2 = torch.cuda.mem_get_info(0)[0]
    _outputs_match(first, ref, sc.T)
    _outputs_match(second, ref, sc.T)
    # nothing is allocated: the device's free memory is unchanged by either call
    # (the scratch array is part of the loaded module, present before the first)
    assert free1 == free0 and free2 == free0, (free0, free1, free2)


def test_static_rollout_rejects_sizes_beyond_its_limit():
    import torch
    assert torch.cuda.is_available()
    from paper_2603_25068_b300.native import SimError, SIM_EOVERFLOW
    from paper_2603_25068_b300.sim import rollout_static
    sc = S.city_small(n_vehicles=70000)            # above the 65,536-vehicle limit
    with pytest.raises(SimError) as e:
        rollout_static(sc, T=10)
    assert e.value.code == SIM_EOVERFLOW
