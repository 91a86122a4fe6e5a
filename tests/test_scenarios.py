"""Host-side checks of the input generators behind the platoon and paper-mode
rows: the platoon transform keeps every time and capacity in physical units,
and the paper-mode problem follows the paper's experimental setting."""
import numpy as np

from paper_2603_25068_b300 import scenario as S

FX_ONE = 65536.0


def test_platoon_transform_keeps_physical_units():
    sc = S.random_small(seed=1, side=3, n_vehicles=60, T=600).copy(obs_every=300)
    p = S.with_platoons(sc, 5.0)
    assert (p.dn, p.dt) == (5.0, 5.0)
    # capacity in vehicles per second is kept: credit q dt per step
    np.testing.assert_allclose(p.q_fx / FX_ONE / p.dt, sc.q_fx / FX_ONE / sc.dt, rtol=0, atol=1.0 / FX_ONE / p.dt)
    # horizon, bins and departures keep their length in seconds
    assert p.T * p.dt == sc.T * sc.dt
    assert p.obs_every * p.dt == sc.obs_every * sc.dt
    np.testing.assert_array_equal(p.dep_step, sc.dep_step // 5)
    # the agents and the network are those of the source scenario
    assert p.N == sc.N and p.L == sc.L
    np.testing.assert_array_equal(p.kappa, sc.kappa)
    # dn = 1 is the identity on every field
    q = S.with_platoons(sc, 1.0)
    for f in ("T", "dt", "dn", "obs_every"):
        assert getattr(q, f) == getattr(sc, f), f
    np.testing.assert_array_equal(q.q_fx, sc.q_fx)
    np.testing.assert_array_equal(q.dep_step, sc.dep_step)


def test_paper_mode_follows_the_experimental_setting():
    model, truth = S.paper_mode(n_vehicles=2000, T=600, dep_window=600)
    assert (model.V, model.L, model.N) == (48, 100, 2000)
    assert len(model.sensors) == 80 and np.array_equal(model.sensors, truth.sensors)
    assert len(np.unique(model.sensors)) == 80
    for k, (lo, hi) in S.PAPER_RANGES.items():
        t = getattr(truth, k).astype(np.float64)
        assert np.all(t >= lo - 1e-6) and np.all(t <= hi + 1e-6), k
        assert t.std() > 0.15 * (hi - lo), k                   # drawn over the range, not constant
        np.testing.assert_allclose(getattr(model, k), 0.5 * (lo + hi), rtol=1e-6)
    np.testing.assert_array_equal(model.cost, 1.0)
    # same network and demand on both sides; only the link parameters differ
    for f in ("tail", "head", "length", "origin", "dest_zone", "dep_step"):
        np.testing.assert_array_equal(getattr(model, f), getattr(truth, f), err_msg=f)
    # origins spread evenly over the nodes, no trip to its own origin
    assert np.bincount(model.origin, minlength=48).max() - np.bincount(model.origin, minlength=48).min() <= 1
    assert np.all(model.dest_zone != model.node_zone[model.origin])


def test_noisy_counts_have_ten_percent_noise():
    rng = np.random.default_rng(0)
    c = np.full((200, 50), 1000.0)
    n = S.noisy_counts(c, rng)
    rel = (n - c) / c
    assert abs(rel.mean()) < 0.002 and abs(rel.std() - 0.1) < 0.003
    assert np.all(n == np.rint(n)) and np.all(S.noisy_counts(np.zeros((3, 3)), rng) == 0)
