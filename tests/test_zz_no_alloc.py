"""The allocation-free rollout entry point (sim_rollout_static) against the
ordinary one (sim_create + sim_rollout).

sim_rollout_static exists for callers that may not allocate device memory:
code that runs while a stream is being captured into a CUDA graph, plug-ins
whose host process owns every device allocation, and real-time loops.  It keeps
all state in one fixed device array shared by every call, so two calls in a
row must each re-initialise it and give the same outputs as the ordinary path.
This file is collected last so that a run stopping at the first failure has
already run every other test.
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
    ref = Simulator(sc).rollout()
    first = rollout_static(sc)
    second = rollout_static(sc)
    _outputs_match(first, ref, sc.T)
    _outputs_match(second, ref, sc.T)


def test_static_rollout_rejects_sizes_beyond_its_limit():
    import torch
    assert torch.cuda.is_available()
    from paper_2603_25068_b300.native import SimError, SIM_EOVERFLOW
    from paper_2603_25068_b300.sim import rollout_static
    sc = S.city_small(n_vehicles=70000)            # above the 65,536-vehicle limit
    with pytest.raises(SimError) as e:
        rollout_static(sc, T=10)
    assert e.value.code == SIM_EOVERFLOW
