"""Pins of the CPU oracle to facts fixed by the paper or by mathematics
(no GPU).  Each test names the passage it follows."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle.oracle import OracleSim, gumbel, log32, philox4x32_10
from paper_2603_25068_b300 import scenario as S

PRECISIONS = ["fp64", "fp32"]


# ---------------------------------------------------------------- random numbers
def test_philox_known_answers():
    """Philox4x32-10 known-answer vectors published with Random123
    (Salmon et al., SC'11)."""
    assert list(philox4x32_10([0, 0, 0, 0], [0, 0])) == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    assert list(philox4x32_10([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2)) == [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]
    assert list(philox4x32_10([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344],
                              [0xA4093822, 0x299F31D0])) == [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_log32_error_bound():
    """The float logarithm used for Gumbel keys stays within 2 ulp of log."""
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.uniform(2 ** -24, 1.0, 4000), rng.uniform(1e-7, 20.0, 4000),
                         np.float32(1.0) - np.arange(1, 200, dtype=np.float32) * np.float32(2 ** -24),
                         np.array([2 ** -24, 0.5, 1.0 - 2 ** -24, 16.6, 1.4142135, 1.4142137])])
    xs = xs.astype(np.float32)
    worst = 0.0
    for x in xs:
        got = log32(float(x))
        ref = math.log(float(x))
        ulp = np.spacing(np.float32(abs(ref))) if ref != 0 else np.float32(2 ** -149)
        worst = max(worst, abs(got - ref) / float(ulp))
    assert worst <= 2.0, worst


@pytest.mark.parametrize("prec", PRECISIONS)
def test_gumbel_distribution(prec):
    """g = -log(-log U) is Gumbel(0,1): mean = Euler-Mascheroni constant,
    variance pi^2/6, and exp(-exp(-g)) is uniform (SI-B, Eq. gumbel)."""
    n = 40000
    g = np.array([gumbel(12345, 7, i, 3, 0, k, prec) for i in range(n // 4) for k in range(4)])
    se = math.pi / math.sqrt(6) / math.sqrt(n)
    assert abs(g.mean() - 0.5772156649) < 4 * se
    assert abs(g.var() - math.pi ** 2 / 6) < 0.05
    u = np.exp(-np.exp(-g))
    assert stats.kstest(u, "uniform").pvalue > 1e-3


# ---------------------------------------------------------------- car-following
@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("length,u", [(100.0, 13.9), (100.0, 10.0), (237.0, 8.3), (60.0, 25.0)])
def test_lone_vehicle_link_time(prec, length, u):
    """A lone vehicle moves at free-flow speed (Eq. newell_model, first term) and
    is capped at the link end by the TG clip (Eq. eq:tg); it is at the end after
    ceil((L - eps)/(u dt)) steps and leaves in that step."""
    sc = S.line_network(n_links=3, length=length, u=u, N=1, T=200)
    o = OracleSim(sc, prec)
    out = o.rollout()
    k = math.ceil((np.float32(length) - 0.01) / np.float32(u))
    arr = np.nonzero(out["n_arrived"])[0][0]
    assert arr == 1 + 3 * k            # departs at step 0, enters link 0 at t = 1
    tt = out["travel_time"][0]
    np.testing.assert_allclose(tt[:3], k, rtol=0, atol=1e-12)


@pytest.mark.parametrize("dn", [5.0, 30.0])
@pytest.mark.parametrize("prec", PRECISIONS)
def test_lone_platoon_link_time(prec, dn):
    """A lone platoon of dn vehicles (Methods: dt = tau dn, tau = 1 s) moves
    u dt per step: it is at each link's end after k = ceil((L - eps)/(u dt))
    steps, and its link time is k dt seconds."""
    length, u = 1000.0, 13.9
    sc = S.with_platoons(S.line_network(n_links=3, length=length, u=u, N=1, T=2000), dn)
    out = OracleSim(sc, prec).rollout()
    k = math.ceil((np.float32(length) - 0.01) / (np.float32(u) * np.float32(sc.dt)))
    arr = np.nonzero(out["n_arrived"])[0][0]
    assert arr == 1 + 3 * k
    np.testing.assert_allclose(out["travel_time"][0][:3], k * sc.dt, rtol=1e-6)


@pytest.mark.parametrize("dt", [1.0, 0.1, 0.02])
def test_lone_vehicle_small_dt_limit(dt):
    """With dt = tau dn, tau = 1 (Methods), the link time of a lone vehicle
    tends to L/u as dt -> 0: |TT - L/u| <= dt."""
    length, u = 100.0, 13.9
    T = int(round(60 / dt))
    sc = S.line_network(n_links=1, length=length, u=u, N=1, T=T).copy(dt=dt, dn=dt, obs_every=T)
    o = OracleSim(sc, "fp64")
    out = o.rollout()
    tt = out["travel_time"][0][0]
    assert abs(tt - length / u) <= dt + 1e-9


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("u,kappa", [(10.0, 0.2), (13.9, 0.2), (20.0, 0.4)])
def test_entry_flow_equals_newell_capacity(prec, u, kappa):
    """A saturated origin feeds a long link at the capacity of Newell's model
    with dt = tau dn, tau = 1: q = u kappa / (1 + u kappa) (Eq. newell_model with
    the vacancy rule X_min > dn/kappa of SI-B)."""
    N = 600
    sc = S.line_network(n_links=1, length=5000.0, u=u, kappa=kappa, q=1.0, N=N, T=500)
    o = OracleSim(sc, prec)
    out = o.rollout()
    entered = N - out["n_waiting"]
    rate = (entered[450] - entered[50]) / 400.0
    cap = u * kappa / (1.0 + u * kappa)
    assert abs(rate - cap) < 0.01, (rate, cap)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_exit_flow_limited_by_outflow_credit(prec):
    """The outflow credit (0.5 veh/s) bounds the discharge of a saturated link."""
    N = 300
    sc = S.line_network(n_links=2, length=300.0, u=13.9, kappa=0.2, q=0.5, N=N, T=600)
    o = OracleSim(sc, prec)
    out = o.rollout()
    arr = out["n_arrived"]
    rate = (arr[500] - arr[200]) / 300.0
    assert abs(rate - 0.5) < 0.01


# ---------------------------------------------------------------- invariants
def _per_step_invariants(sc, prec):
    o = OracleSim(sc, prec)
    o.reset()
    prev_exits = np.zeros(sc.L, np.int64)
    s = (np.float64(sc.dn) / sc.kappa.astype(np.float64))
    for t in range(sc.T):
        o.step()
        st = o.state()
        link, pos, rank, entry = st["veh_link"], st["veh_pos"], st["veh_rank"], st["veh_entry"]
        on = link >= 0
        # positions inside the link (SI-A: no backward motion, inside boundaries)
        assert np.all(pos[on] >= 0) and np.all(pos[on] <= sc.length[link[on]] + 1e-9)
        # FIFO / no overtaking: queue order by position equals order of entry
        for j in np.unique(link[on]):
            ids = np.nonzero(link == j)[0]
            order = ids[np.argsort(rank[ids])]
            assert np.all(np.diff(entry[order]) > 0)
            gaps = -np.diff(pos[order])
            assert np.all(gaps >= s[j] * (1 - 1e-5) - 1e-4), (t, j, gaps.min(), s[j])
            assert len(ids) <= math.floor(sc.length[j] / s[j]) + 1
        # at most one exit per link per step, never above the credit
        d = st["link_exits"] - prev_exits
        assert d.min() >= 0 and d.max() <= 1
        prev_exits = st["link_exits"].copy()
        assert np.all(st["link_credit"] >= 0)
    out = o.outputs()
    tot = out["n_waiting"] + out["n_on"] + out["n_arrived"]
    assert np.all(tot == sc.N)
    # counts of the final state agree with the state itself
    return out


@pytest.mark.parametrize("prec", PRECISIONS)
def test_invariants_tiny_grid(prec):
    sc = S.tiny_grid()
    out = _per_step_invariants(sc.copy(T=150, obs_every=150), prec)
    assert out["n_on"].max() > 100


@pytest.mark.parametrize("prec", PRECISIONS)
def test_invariants_dense_small(prec):
    sc = S.random_small(seed=3, side=3, n_vehicles=120, T=120)
    _per_step_invariants(sc, prec)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_invariants_platoons(prec):
    # agents of 5 vehicles (step 5 s, jam spacing 5 / kappa, credit 5 per transfer)
    sc = S.with_platoons(S.random_small(seed=3, side=3, n_vehicles=120, T=600), 5.0)
    _per_step_invariants(sc, prec)


@pytest.mark.parametrize("dn", [1, 5, 30])
@pytest.mark.parametrize("prec", PRECISIONS)
def test_platoon_discharge_rate_is_capacity(prec, dn):
    """Platoons of dn vehicles with a step of dn seconds (Methods: dt = tau dn,
    tau = 1 s): the credit grows by q dt per step and a transfer takes dn of it,
    so a saturated link still discharges q = 0.5 vehicles per second."""
    N = 300
    sc = S.with_platoons(S.line_network(n_links=2, length=300.0, u=13.9, kappa=0.2, q=0.5, N=N, T=10), dn)
    T = int(np.ceil(N * dn / 0.5 / sc.dt)) + int(np.ceil(120.0 / sc.dt)) + 10     # + the free-flow trip
    out = OracleSim(sc.copy(T=T, obs_every=T), prec).rollout()
    arr = out["n_arrived"]
    assert arr[-1] == N
    i0, i1 = np.searchsorted(arr, 0.2 * N), np.searchsorted(arr, 0.8 * N)
    rate = (arr[i1] - arr[i0]) * dn / ((i1 - i0) * sc.dt)
    assert abs(rate - 0.5) < 0.01, rate


# ---------------------------------------------------------------- choice model
def _star(beta, n_veh, tau=0.5, seed=0):
    k = len(beta)
    tail = [0] * k + list(range(1, k + 1))
    head = list(range(1, k + 1)) + [0] * k
    b = np.concatenate([beta, np.zeros(k)])
    # every leaf is in the destination zone: a vehicle leaves at the end of its
    # first link, so the origin queue head is the only candidate of each step
    zone = [0] + [1] * k
    # one departure every 2 steps: an entrant has always moved past the jam
    # spacing before the next candidate comes, so no choice is ever blocked
    return S.custom(tail, head, length=500.0, origin=np.zeros(n_veh), dest_node=np.ones(n_veh),
                    dep_step=2 * np.arange(n_veh), u=20.0, beta=b, T=2 * n_veh + 40, tau=tau,
                    seed=seed, node_zone=zone)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_choice_frequencies_are_softmax(prec):
    """argmax(V + g) with Gumbel noise samples the logit probabilities
    z = softmax(V) (SI-B, Eqs. softmax and gumbel): chi-square test."""
    beta = np.array([0.0, 1.0, 2.0])
    n = 3000
    sc = _star(beta, n)
    o = OracleSim(sc, prec)
    o.rollout()
    first = np.array([o.route(i)[1][0] for i in range(n)])
    obs = np.bincount(first, minlength=3)[:3]
    p = np.exp(beta) / np.exp(beta).sum()
    chi2 = ((obs - n * p) ** 2 / (n * p)).sum()
    assert stats.chi2.sf(chi2, 2) > 1e-3, (obs, n * p)


def test_forward_is_temperature_free():
    """The one-hot of the Gumbel-softmax sample is argmax(log z + g), which does
    not depend on the temperature (Eqs. gumbel, straigththrough)."""
    sc = S.random_small(seed=5, n_vehicles=60, T=80)
    a = OracleSim(sc.copy(tau=0.5), "fp64").rollout()
    b = OracleSim(sc.copy(tau=0.01), "fp64").rollout()
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])


def _fork_merge(seed, betaX, betaY, alphaA, alphaB):
    # A=0, B=1, C=2, D1=3, D2=4; links 0:A->C 1:B->C 2:C->D1 (X) 3:C->D2 (Y) 4:D1->A 5:D2->B
    tail = [0, 1, 2, 2, 3, 4]
    head = [2, 2, 3, 4, 0, 1]
    beta = [0, 0, betaX, betaY, 0, 0]
    alpha = [alphaA, alphaB, 1, 1, 1, 1]
    return S.custom(tail, head, length=100.0, origin=[0, 1], dest_node=[3, 3], dep_step=[0, 0],
                    u=10.0, beta=beta, alpha=alpha, T=40, seed=seed)


def test_brute_force_fork_and_merge():
    """Two vehicles reach a fork at the same step.  Enumerating the decision
    sequences (link choice, merge, re-draw with fresh noise) gives exact
    probabilities of (link entered by vehicle 0, link entered by vehicle 1);
    the oracle's empirical frequencies over seeds must match (SI-B link and
    merge choice)."""
    bX, bY, aA, aB = 0.3, 1.0, 1.0, 2.0
    pX = math.exp(bX) / (math.exp(bX) + math.exp(bY))
    pY = 1 - pX
    P0 = math.exp(aA) / (math.exp(aA) + math.exp(aB))      # vehicle 0 wins a merge
    P1 = 1 - P0
    exact = {(2, 2): 0.0, (2, 3): 0.0, (3, 2): 0.0, (3, 3): 0.0}
    # different picks: both enter; same pick: the winner enters, the loser re-draws
    exact[(2, 3)] += pX * pY
    exact[(3, 2)] += pY * pX
    for same, p in ((2, pX), (3, pY)):
        for loser_pick, q in ((2, pX), (3, pY)):
            exact[(same, loser_pick)] += p * p * P0 * q      # vehicle 0 won
            exact[(loser_pick, same)] += p * p * P1 * q      # vehicle 1 won
    n = 3000
    obs = {k: 0 for k in exact}
    for s in range(n):
        o = OracleSim(_fork_merge(s, bX, bY, aA, aB), "fp64")
        o.reset(20)
        o.step(20)
        r0, r1 = o.route(0)[1], o.route(1)[1]
        obs[(int(r0[1]), int(r1[1]))] += 1
    keys = sorted(exact)
    e = np.array([exact[k] for k in keys]) * n
    ob = np.array([obs[k] for k in keys])
    assert abs(sum(exact.values()) - 1) < 1e-12
    chi2 = ((ob - e) ** 2 / e).sum()
    assert stats.chi2.sf(chi2, 3) > 1e-3, (ob, e)


# ---------------------------------------------------------------- link speeds (P25 reading)
def _lone_vehicle_bin_speeds(length, u, dt, eps, n_links, n_bins, obs_every):
    """Closed form of the bin speeds of one vehicle crossing a chain of equal
    links in free flow: on each link it makes k = ceil((L - eps)/(u dt))
    car-following steps, the s-th moving it to min(s u dt, L) (the TG clip),
    and leaves in the k-th; it departs at step 0 and is on link l during steps
    1 + l k .. (l + 1) k.  Speed of a link in a bin = distance travelled on it
    in the bin / (vehicle-steps on it in the bin x dt)."""
    udt = u * dt
    k = math.ceil((length - eps) / udt)
    dist = np.zeros((n_bins, 2 * n_links))
    steps = np.zeros((n_bins, 2 * n_links))
    for l in range(n_links):
        for s in range(1, k + 1):
            t = 1 + l * k + (s - 1)
            b = t // obs_every
            if b < n_bins:
                dist[b, l] += min(s * udt, length) - min((s - 1) * udt, length)
                steps[b, l] += 1
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(steps > 0, dist / (steps * dt), 0.0), k


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("length,u,obs_every", [(200.0, 13.9, 5), (200.0, 13.9, 7), (237.0, 8.3, 11),
                                                (100.0, 10.0, 200)])
def test_lone_vehicle_bin_speed(prec, length, u, obs_every):
    """Mean link speed of a bin (reading P25: distance over vehicle-time on the
    link in the bin) for a lone vehicle: u in bins of unclipped free flow, the
    clipped last metres over one step where it reaches the end, 0 on empty
    links, in every bin in closed form."""
    T = 200
    sc = S.line_network(n_links=3, length=length, u=u, N=1, T=T).copy(obs_every=obs_every)
    out = OracleSim(sc, prec).rollout()
    nb = out["speed"].shape[0]
    exp, k = _lone_vehicle_bin_speeds(float(np.float32(length)), float(np.float32(u)), 1.0, 0.01, 3, nb,
                                      obs_every)
    np.testing.assert_allclose(out["speed"], exp, rtol=1e-5, atol=1e-9)
    if obs_every >= 3 * k + 1:       # one bin holds the whole trip: distance L per link over k steps
        np.testing.assert_allclose(out["speed"][0][:3], min(k * np.float32(u), np.float32(length)) / k, rtol=1e-6)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_speed_counts_waiting_vehicle_steps(prec):
    """A vehicle held at the end of a link by the outflow credit keeps counting
    vehicle-steps at zero displacement (P25 denominator), and its link time
    counts the wait (travel time = exit step + 1 - entry step).  Link 1 of a
    chain lets 1 veh out per 65536 / q_fx steps: vehicle 0 (departing at 0)
    leaves it at step 2k, vehicle 1 (departing at 50) arrives at step 50 + 2k
    and waits until the credit refills at step 2k + ceil(65536 / q_fx)."""
    length, u = 200.0, 13.9
    sc = S.line_network(n_links=3, length=length, u=u, N=2, dep=[0, 50], T=400).copy(obs_every=400)
    q = sc.q_fx.copy()
    q[1] = 655                                    # 0.01 veh/s
    sc = sc.copy(q_fx=q)
    out = OracleSim(sc, prec).rollout()
    k = math.ceil((np.float32(length) - 0.01) / np.float32(u))
    d = min(k * float(np.float32(u)), float(np.float32(length)))
    s2 = max(50 + 2 * k, 2 * k + math.ceil(65536 / 655))        # vehicle 1's exit step from link 1
    steps1 = k + (s2 - (51 + k) + 1)                             # vehicle-steps on link 1
    np.testing.assert_allclose(out["speed"][0][1], 2 * d / steps1, rtol=1e-6)
    np.testing.assert_allclose(out["speed"][0][0], d / k, rtol=1e-6)
    np.testing.assert_allclose(out["travel_time"][0][1], (k + (s2 + 1 - (51 + k))) / 2, rtol=1e-12)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_standing_queue_has_zero_speed(prec):
    """Ten vehicles queue on link 1 of a chain whose exit passes one vehicle per
    101 steps (q_fx = 655).  Exits happen at steps 2k + 101 m; in a bin with no
    exit every queued vehicle stands (headway exactly the jam spacing, Eq.
    newell_model second term 0), so the link's bin speed is 0, while the bin's
    vehicle-steps are not."""
    length, u = 200.0, 13.9
    sc = S.line_network(n_links=3, length=length, u=u, N=10, T=400).copy(obs_every=50)
    q = sc.q_fx.copy()
    q[1] = 655
    out = OracleSim(sc.copy(q_fx=q), prec).rollout()
    k = math.ceil((np.float32(length) - 0.01) / np.float32(u))
    exits = [2 * k + 101 * m for m in range(5)]
    assert exits[3] < 350 and exits[4] >= 400 and k == 15
    assert out["speed"][7][1] == 0.0 and out["travel_time"][7][1] == 0.0      # steps 350-399
    o = OracleSim(sc.copy(q_fx=q), prec)
    o.reset(400)
    o.step(375)
    assert (o.state()["veh_link"] == 1).sum() == 6                           # the queue is there


# ------------------------------------------------- relaxed weights as the temperature goes to 0
def test_relaxed_choice_weights_tend_to_the_forward_one_hot():
    """The Gumbel-softmax weights softmax((V + g)/tau) whose straight-through
    one-hot the forward takes (SI-B Eqs. gumbel, straigththrough) tend to the
    one-hot of the chosen link as tau -> 0: argmax pi is the forward's choice,
    1 - pi_chosen <= (deg - 1) exp(-gap / tau) with gap the top-2 key gap, pi
    sharpens monotonically, and log(pi_a / pi_b) scales exactly as 1/tau.  The
    merge weights over (alpha_src + g')/tau tend to the winner the same way."""
    sc = S.tiny_grid(T=120)
    o = OracleSim(sc, "fp64", keep_history=True)
    o.reset(sc.T)
    taus = [1.0, 0.1, 0.01, 0.001]
    n_choice = n_merge = 0
    for t in range(sc.T):
        o.step(1)
        r = o.records()
        for j in range(sc.L):
            if r["link_cand"][j] < 0 or r["link_target"][j] == -2:
                continue
            gap = r["link_margin"][j]
            prev = 0.0
            for tau in taus:
                pi, slot = o.choice_weights(t, tau, link=j)
                assert abs(pi.sum() - 1) < 1e-12
                if gap > 0:
                    assert int(np.argmax(pi)) == slot
                    assert 1 - pi[slot] <= (len(pi) - 1) * math.exp(-gap / tau) * (1 + 1e-9) + 1e-15
                assert pi[slot] >= prev - 1e-15
                prev = pi[slot]
            pi1, slot = o.choice_weights(t, 1.0, link=j)
            pi2, _ = o.choice_weights(t, 0.5, link=j)
            ok = (pi1 > 1e-150) & (pi2 > 1e-150)
            np.testing.assert_allclose(np.log(pi2[ok] / pi2[slot]), 2 * np.log(pi1[ok] / pi1[slot]),
                                       rtol=1e-9, atol=1e-9)
            n_choice += 1
        for m in range(sc.L):
            if r["link_in"][m] < 0:
                continue
            gap = r["merge_margin"][m]
            for tau in taus:
                w, vid, won = o.merge_weights(t, m, tau)
                assert won.sum() == 1 and vid[won][0] == r["link_in"][m]
                if np.isfinite(gap) and gap > 0:
                    assert int(np.argmax(w)) == int(np.nonzero(won)[0][0])
                    assert 1 - w[won][0] <= (len(w) - 1) * math.exp(-gap / tau) * (1 + 1e-9) + 1e-15
            n_merge += 1
    assert n_choice > 200 and n_merge > 200
