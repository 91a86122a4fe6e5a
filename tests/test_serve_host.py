"""Host logic of the serving engine (no GPU): the requests' loss cotangents,
the Poisson request stream and its mix, the memory bound used for admission,
the admission priority, and the latency statistics."""
import numpy as np
import pytest

from paper_2603_25068_b300 import scenario as S
from paper_2603_25068_b300 import serve


def test_loss_cotangents_are_the_loss_gradients():
    rng = np.random.default_rng(0)
    sc = S.tiny_grid().copy(sensors=np.array([2, 5, 11], np.int32))
    counts = rng.integers(0, 40, size=(4, sc.L)).astype(np.float32)
    obs = rng.integers(0, 40, size=(4, 3)).astype(np.float32)
    req = serve.Request(rid=0, kind="calibration", scenario=sc, arrival=0.0, observed=obs)

    def mse(c):
        return float(np.mean((c[:, sc.sensors].astype(np.float64) - obs) ** 2))
    g = serve.loss_cotangent(req, counts)
    for b, j in [(0, 2), (3, 11), (1, 5)]:
        e = np.zeros_like(counts)
        e[b, j] = 0.5
        assert g[b, j] == pytest.approx((mse(counts + e) - mse(counts - e)) / 1.0, rel=1e-6)
    assert np.count_nonzero(g[:, [k for k in range(sc.L) if k not in (2, 5, 11)]]) == 0
    # control: (total - goal)^2 with the goal at half the total, on the target column only
    req = serve.Request(rid=1, kind="control", scenario=sc, arrival=0.0, target_link=7)
    g = serve.loss_cotangent(req, counts)
    tot = float(counts[:, 7].sum())
    assert np.all(g[:, 7] == pytest.approx(2.0 * (tot - 0.5 * tot)))
    assert np.count_nonzero(np.delete(g, 7, axis=1)) == 0
    req = serve.Request(rid=2, kind="nowcast", scenario=sc, arrival=0.0)
    assert not req.needs_grad and np.count_nonzero(serve.loss_cotangent(req, counts)) == 0


def test_request_stream_is_poisson_with_the_configured_mix():
    reqs = serve.make_request_stream(n=600, rate=4.0, seed=7, sizes=(2000,), n_range=(1000, 20000))
    t = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 0.25) < 0.025                   # rate 4 per second
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.12         # exponential gaps
    kinds = [r.kind for r in reqs]
    assert abs(kinds.count("nowcast") / 600 - 0.5) < 0.07
    assert abs(kinds.count("calibration") / 600 - 0.25) < 0.06
    n = np.array([r.scenario.N for r in reqs])
    assert n.min() >= 1000 and n.max() <= 20000
    for r in reqs:
        sc = r.scenario
        assert sc.T == (3600 if r.kind == "nowcast" else 1800)
        if r.kind == "calibration":
            nb = -(-sc.T // sc.obs_every)
            assert r.observed.shape == (nb, len(sc.sensors))
        if r.kind == "control":
            assert 0 <= r.target_link < sc.L
            assert sc.beta.min() >= 0.0 and sc.beta.max() <= 5.0
    assert len({r.scenario.scenario_id for r in reqs}) == 600   # independent noise per request


def test_memory_bound_grows_with_the_work():
    base = S.city_small()
    small = serve.handle_bytes_bound(base, 0, 64)
    assert small > 0
    assert serve.handle_bytes_bound(base.copy(N=2 * base.N), 0, 64) > small
    grad = serve.handle_bytes_bound(base, 180, 64)
    assert grad > small                                       # checkpoints and route log
    assert serve.handle_bytes_bound(base, 60, 64) > grad       # more checkpoints
    assert serve.handle_bytes_bound(base, 180, 256) > grad     # longer route log


def test_latency_statistics():
    sc = S.tiny_grid()
    reqs = []
    for k, lat in enumerate(np.arange(1, 101, dtype=np.float64)):
        r = serve.Request(rid=k, kind="nowcast", scenario=sc, arrival=float(k))
        r.finished = float(k) + lat
        reqs.append(r)
    st = serve.latency_stats(reqs)
    assert st["p50_s"] == pytest.approx(50.5) and st["max_s"] == 100.0 and st["mean_s"] == pytest.approx(50.5)
    assert st["p99_s"] == pytest.approx(np.percentile(np.arange(1, 101), 99))


def test_admission_priority_is_shortest_work_with_aging():
    """Shortest work first among requests that arrived together; a long request
    that has waited about its own run time goes ahead of newer short ones (no
    starvation); a gradient request counts three times its vehicle-steps."""
    from paper_2603_25068_b300 import scenario as S
    small = S.tiny_grid(n_vehicles=200, T=100)
    big = S.tiny_grid(n_vehicles=1000, T=300)
    a = serve.Request(rid=0, kind="nowcast", scenario=big, arrival=0.0)
    b = serve.Request(rid=1, kind="nowcast", scenario=small, arrival=0.0)
    g = serve.Request(rid=2, kind="calibration", scenario=small, arrival=0.0)
    assert serve.request_priority(b, 0.0) < serve.request_priority(g, 0.0) < serve.request_priority(a, 0.0)
    assert serve.request_work(g) == 3 * serve.request_work(b)
    wait = serve.request_work(a) / serve.WORK_PER_SECOND
    late = serve.Request(rid=3, kind="nowcast", scenario=small, arrival=1.5 * wait)
    assert serve.request_priority(a, 1.5 * wait) < serve.request_priority(late, 1.5 * wait)
