"""Serving with continuous batching: requests of different kinds, networks and
sizes arrive while others run; each result equals the result of the same request
processed alone (forward outputs bitwise; gradients up to the order of double
additions in the reverse pass), and the result of the oracle: counts bitwise
against its float build, speeds and travel times to 1e-4 / 1e-6 relative,
gradients against its reverse mode (gradcheck.py)."""
import numpy as np
import pytest

from gradcheck import compare_grads
from oracle.oracle import OracleSim

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("reversers", [0, 2])
def test_served_results_equal_results_alone(reversers):
    """reversers = 0: reverse passes between forward chunks on the engine's
    stream; 2: on worker threads beside the forward work."""
    from paper_2603_25068_b300 import serve
    # arrivals close enough together that several requests are ready at once
    reqs = serve.make_request_stream(n=8, rate=400.0, seed=7, sizes=(600, 1200), n_range=(3000, 20000),
                                     horizons={"nowcast": 400, "calibration": 300, "control": 300}, n_sensors=50)
    kinds = {r.kind for r in reqs}
    assert {"nowcast"} < kinds
    eng = serve.Engine(hbm_budget=20e9, chunk=25, ckpt_every=60, reversers=reversers)
    eng.run(reqs)
    st = serve.latency_stats(reqs)
    assert st["p99_s"] >= st["p50_s"] > 0
    # several requests were in flight together
    overlap = sum(1 for a in reqs for b in reqs if a is not b and a.admitted < b.finished and b.admitted < a.finished)
    assert overlap > 0
    for r in reqs:
        alone = serve.run_request_alone(r, ckpt_every=60)
        for k in ("counts", "speed", "travel_time"):
            np.testing.assert_array_equal(r.result[k], alone[k], err_msg=f"{r.kind} {k}")
        if r.needs_grad:
            for k, g in alone["grad"].items():
                scale = max(1e-6, float(np.abs(g).max()))
                np.testing.assert_allclose(r.result["grad"][k], g, rtol=0, atol=1e-5 * scale, err_msg=f"{r.kind} {k}")
        # against the oracle
        sc = r.scenario
        o = OracleSim(sc, "fp32", keep_history=r.needs_grad)
        ref = o.rollout(sc.T)
        np.testing.assert_array_equal(r.result["counts"], ref["counts"], err_msg=r.kind)
        np.testing.assert_allclose(r.result["travel_time"], ref["travel_time"], rtol=1e-6, atol=0)
        np.testing.assert_allclose(r.result["speed"], ref["speed"], rtol=1e-4, atol=1e-5)
        if r.needs_grad:
            yb = serve.loss_cotangent(r, ref["counts"]).astype(np.float64)
            compare_grads(r.result["grad"], o.backward(yb))


def test_admission_respects_the_budget():
    from paper_2603_25068_b300 import serve
    reqs = serve.make_request_stream(n=4, rate=1000.0, seed=8, sizes=(600,), n_range=(3000, 6000),
                                     horizons={"nowcast": 120, "calibration": 120, "control": 120})
    one = max(serve.Simulator(r.scenario).device_bytes() for r in reqs)
    eng = serve.Engine(hbm_budget=1.5 * one + 1e8, chunk=20, ckpt_every=60)   # about one request at a time
    eng.run(reqs)
    assert all(np.isfinite(r.finished) for r in reqs)
    order = sorted(reqs, key=lambda r: r.admitted)
    # with room for about one request, admissions wait for earlier results
    assert any(b.admitted >= a.finished - 1e-3 for a, b in zip(order, order[1:]))
