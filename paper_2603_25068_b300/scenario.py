"""Seeded synthetic scenario generator (inputs only).

This module builds road networks, travel demand and route-choice parameters for
the simulator.  It holds none of the simulation arithmetic: it only draws and
formats inputs.  Both the CUDA path and the CPU oracle consume what it returns,
and nothing else is shared between them.

Input recipe (paper context: Sec. "Experimental setting", SI-F).  The paper's
networks (TNTP Sioux Falls / Chicago Sketch) and its observations are not
available, so every workload here is synthetic with the shapes the paper and the
benchmark configurations describe:

* ``tiny_grid``   5x5 square grid, 80 directed 200 m one-lane links, u = 13.9 m/s,
                  0.5 veh/s capacity, 1,000 vehicles departing in the first 120 s,
                  3-feature linear utility with w ~ N(0, 1), 300 steps.
* ``city``        12,000 random points, Delaunay graph thinned to a spanning tree
                  plus the shortest remaining edges (18,000 undirected = 36,000
                  directed links), lognormal lengths (median 150 m, sigma 0.6),
                  1-4 lanes, u ~ U(8, 25) m/s, 80 origin x 128 destination zones
                  (10,240 OD demand parameters), 1,000,000 vehicles departing
                  uniformly over 30 min (Poisson process conditioned on count).
* ``tg_toy``      the two-link single-agent example of SI-C (Fig. S1).

Units: metres, seconds, vehicles.  Capacities are given as integer outflow
credit per time step in units of 2^-16 vehicle (``q_fx``).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

FX_ONE = 65536  # one vehicle of outflow credit


@dataclasses.dataclass
class Scenario:
    name: str
    # network
    V: int
    L: int
    tail: np.ndarray          # int32 [L]  upstream node of each link
    head: np.ndarray          # int32 [L]  downstream node of each link
    length: np.ndarray        # f32 [L]    metres
    lanes: np.ndarray         # int32 [L]
    u: np.ndarray             # f32 [L]    free-flow speed (m/s)
    kappa: np.ndarray         # f32 [L]    jam density (veh/m)
    alpha: np.ndarray         # f32 [L]    merge priority
    beta: np.ndarray          # f32 [L]    cost sensitivity
    cost: np.ndarray          # f32 [L]    link cost (> 0)
    q_fx: np.ndarray          # int32 [L]  outflow credit per step, 2^-16 veh
    F: int
    phi: np.ndarray           # f32 [L, F] link features
    psi: np.ndarray           # f32 [L, F] weights of the destination feature
    w: np.ndarray             # f32 [F]    route-choice coefficients
    Z: int
    node_zone: np.ndarray     # int32 [V]  destination zone of each node
    dest_feat: np.ndarray     # f32 [Z, V] destination feature (-minutes to zone)
    # demand
    N: int
    origin: np.ndarray        # int32 [N]  origin node
    dest_zone: np.ndarray     # int32 [N]
    dep_step: np.ndarray      # int32 [N]  step at which the vehicle joins its origin queue
    od: np.ndarray            # int32 [N]  OD demand group
    n_od: int
    od_lambda: np.ndarray     # f32 [n_od] demand parameter (expected vehicles)
    # run options
    T: int = 300
    dt: float = 1.0
    dn: float = 1.0
    tau: float = 0.5
    M: float = 99999.0
    eps_arr: float = 1e-2
    eps_tag: float = 1e-6
    alpha_origin: float = 2.505
    seed: int = 0
    scenario_id: int = 0
    obs_every: int = 300
    sensors: Optional[np.ndarray] = None   # int32 sensor link ids (loss links)
    coords: Optional[np.ndarray] = None

    def copy(self, **kw) -> "Scenario":
        d = {f.name: getattr(self, f.name) for f in dataclasses.fields(self)}
        for k, v in d.items():
            if isinstance(v, np.ndarray):
                d[k] = v.copy()
        d.update(kw)
        return Scenario(**d)

    def summary(self) -> dict:
        return dict(name=self.name, V=self.V, L=self.L, N=self.N, F=self.F, Z=self.Z,
                    n_od=self.n_od, T=self.T, tau=self.tau, seed=self.seed)


# ----------------------------------------------------------------------------
# helpers (graph construction and input formatting only)
# ----------------------------------------------------------------------------

def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _capacity_fx(q_veh_per_s, dt):
    return _i32(np.rint(np.asarray(q_veh_per_s, np.float64) * dt * FX_ONE))


def _dest_feature(V, tail, head, tt, node_zone, Z):
    """-(free-flow minutes from each node to the nearest node of each zone)."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import dijkstra
    # reversed graph: distance from zone nodes along reversed links = distance to zone
    g = csr_matrix((tt.astype(np.float64), (head, tail)), shape=(V, V))
    out = np.zeros((Z, V), np.float64)
    for z in range(Z):
        src = np.nonzero(node_zone == z)[0]
        d = dijkstra(g, directed=True, indices=src, min_only=True)
        out[z] = d
    if not np.all(np.isfinite(out)):
        raise ValueError("network is not strongly connected")
    return _f32(-out / 60.0)


def _check_strongly_connected(V, tail, head):
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components
    g = csr_matrix((np.ones(len(tail)), (tail, head)), shape=(V, V))
    n, _ = connected_components(g, directed=True, connection="strong")
    if n != 1:
        raise ValueError(f"network has {n} strongly connected components")


# ----------------------------------------------------------------------------
# configurations
# ----------------------------------------------------------------------------

def tiny_grid(seed: int = 0, n_vehicles: int = 1000, T: int = 300, tau: float = 0.5,
              side: int = 5, spacing: float = 200.0) -> Scenario:
    """5x5 grid, 80 directed links, 1,000 vehicles, 3-feature utility, w ~ N(0,1)."""
    rng = np.random.default_rng(seed)
    V = side * side
    tails, heads = [], []
    for r in range(side):
        for c in range(side):
            n = r * side + c
            if c + 1 < side:
                tails += [n, n + 1]; heads += [n + 1, n]
            if r + 1 < side:
                tails += [n, n + side]; heads += [n + side, n]
    tail, head = _i32(tails), _i32(heads)
    L = len(tail)
    length = _f32(np.full(L, spacing))
    lanes = _i32(np.ones(L))
    u = _f32(np.full(L, 13.9))
    kappa = _f32(np.full(L, 0.2))
    alpha = _f32(np.full(L, 2.505))
    beta = _f32(np.zeros(L))
    cost = _f32(np.ones(L))
    q_fx = _capacity_fx(np.full(L, 0.5), 1.0)
    # features: (-free-flow minutes / 10 ... scaled), destination, -cost
    F = 3
    tt = length.astype(np.float64) / u.astype(np.float64)
    phi = np.zeros((L, F), np.float32)
    psi = np.zeros((L, F), np.float32)
    phi[:, 0] = -tt / 60.0
    psi[:, 1] = 1.0
    phi[:, 2] = -cost
    w = _f32(rng.normal(size=F))
    Z = V
    node_zone = _i32(np.arange(V))
    dest_feat = _dest_feature(V, tail, head, tt, node_zone, Z)
    N = n_vehicles
    origin = rng.integers(0, V, size=N)
    dest = rng.integers(0, V - 1, size=N)
    dest = np.where(dest >= origin, dest + 1, dest)           # o != d
    t_dep = rng.uniform(0.0, 120.0, size=N)
    dep_step = _i32(np.floor(t_dep))
    od = _i32(origin * V + dest)
    # compact OD ids
    uniq, od_c = np.unique(od, return_inverse=True)
    counts = np.bincount(od_c)
    _check_strongly_connected(V, tail, head)
    return Scenario(name="tiny_grid", V=V, L=L, tail=tail, head=head, length=length,
                    lanes=lanes, u=u, kappa=kappa, alpha=alpha, beta=beta, cost=cost,
                    q_fx=q_fx, F=F, phi=_f32(phi), psi=_f32(psi), w=w, Z=Z,
                    node_zone=node_zone, dest_feat=dest_feat, N=N, origin=_i32(origin),
                    dest_zone=_i32(dest), dep_step=dep_step, od=_i32(od_c),
                    n_od=len(uniq), od_lambda=_f32(counts), T=T, tau=tau, seed=seed,
                    obs_every=300, sensors=_i32(np.arange(L)))


def _planar_graph(rng, n_nodes, n_undirected):
    from scipy.spatial import Delaunay
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import minimum_spanning_tree
    pts = rng.uniform(0.0, 1.0, size=(n_nodes, 2))
    tri = Delaunay(pts)
    s = tri.simplices
    e = np.concatenate([s[:, [0, 1]], s[:, [1, 2]], s[:, [0, 2]]])
    e.sort(axis=1)
    e = np.unique(e, axis=0)
    elen = np.linalg.norm(pts[e[:, 0]] - pts[e[:, 1]], axis=1)
    # random spanning tree: minimum spanning tree under random weights
    rw = rng.uniform(1.0, 2.0, size=len(e))
    g = csr_matrix((rw, (e[:, 0], e[:, 1])), shape=(n_nodes, n_nodes))
    t = minimum_spanning_tree(g).tocoo()
    tree = np.stack([np.minimum(t.row, t.col), np.maximum(t.row, t.col)], 1)
    key = lambda a: a[:, 0].astype(np.int64) * n_nodes + a[:, 1]
    in_tree = np.isin(key(e), key(tree))
    rest = np.nonzero(~in_tree)[0]
    rest = rest[np.argsort(elen[rest], kind="stable")]
    need = n_undirected - len(tree)
    if need < 0 or need > len(rest):
        raise ValueError("cannot reach the requested edge count")
    keep = np.concatenate([tree, e[rest[:need]]])
    return pts, keep


def _kmeans_labels(rng, pts, k, iters=25):
    c = pts[rng.choice(len(pts), size=k, replace=False)]
    for _ in range(iters):
        d = ((pts[:, None, :] - c[None, :, :]) ** 2).sum(-1)
        lab = d.argmin(1)
        for j in range(k):
            m = lab == j
            if m.any():
                c[j] = pts[m].mean(0)
    d = ((pts[:, None, :] - c[None, :, :]) ** 2).sum(-1)
    return d.argmin(1)


def city_features(length, u, lanes, cost, w_tt=1.0, w_dest=6.0, w_len=0.0, w_const=0.0):
    """16 route-choice features: (free-flow minutes, destination, length km,
    constant) for each of 4 lane classes.  Returns phi, psi, w."""
    L = len(length)
    F = 16
    phi = np.zeros((L, F), np.float32)
    psi = np.zeros((L, F), np.float32)
    tt_min = length.astype(np.float64) / u.astype(np.float64) / 60.0
    for c in range(4):
        m = lanes == (c + 1)
        phi[m, 4 * c + 0] = -tt_min[m]
        psi[m, 4 * c + 1] = 1.0
        phi[m, 4 * c + 2] = -length[m] / 1000.0
        phi[m, 4 * c + 3] = 1.0
    w = np.tile(np.array([w_tt, w_dest, w_len, w_const], np.float32), 4)
    return _f32(phi), _f32(psi), _f32(w)


def city(seed: int = 1, n_nodes: int = 12000, n_links: int = 36000,
         n_vehicles: int = 1_000_000, T: int = 3600, tau: float = 0.5,
         n_origin_zones: int = 80, n_dest_zones: int = 128,
         dep_window: float = 1800.0, capacity_mult: Optional[np.ndarray] = None,
         name: str = "city", demand_mult: Optional[np.ndarray] = None,
         demand_seed: Optional[int] = None) -> Scenario:
    """Random planar city network with zone-based OD demand (see module doc).
    demand_mult scales the OD demand parameters and demand_seed (default: seed)
    draws the vehicles from them, so that a second draw of the demand can share
    the network of the first."""
    rng = np.random.default_rng(seed)
    pts, und = _planar_graph(rng, n_nodes, n_links // 2)
    tail = _i32(np.concatenate([und[:, 0], und[:, 1]]))
    head = _i32(np.concatenate([und[:, 1], und[:, 0]]))
    L = len(tail)
    V = n_nodes
    length = _f32(np.clip(rng.lognormal(np.log(150.0), 0.6, size=L), 10.0, 3000.0))
    lanes = _i32(rng.integers(1, 5, size=L))
    u = _f32(rng.uniform(8.0, 25.0, size=L))
    kappa = _f32(0.2 * lanes)
    alpha = _f32(np.full(L, 2.505))
    beta = _f32(np.zeros(L))
    cost = _f32(np.ones(L))
    q = 0.5 * lanes.astype(np.float64)
    if capacity_mult is not None:
        q = q * capacity_mult
    q_fx = _capacity_fx(q, 1.0)
    phi, psi, w = city_features(length, u, lanes, cost)
    F = phi.shape[1]
    _check_strongly_connected(V, tail, head)
    ozone = _kmeans_labels(rng, pts, n_origin_zones)
    dzone = _i32(_kmeans_labels(rng, pts, n_dest_zones))
    tt = length.astype(np.float64) / u.astype(np.float64)
    dest_feat = _dest_feature(V, tail, head, tt, dzone, n_dest_zones)
    n_od = n_origin_zones * n_dest_zones
    lam = rng.lognormal(0.0, 1.0, size=n_od)
    lam = lam / lam.sum() * n_vehicles
    if demand_mult is not None:
        lam = lam * demand_mult
        lam = lam / lam.sum() * n_vehicles
    if demand_seed is not None:
        rng = np.random.default_rng(demand_seed)
    counts = rng.multinomial(n_vehicles, lam / lam.sum())
    od = _i32(np.repeat(np.arange(n_od), counts))
    oz = od // n_dest_zones
    dz = od % n_dest_zones
    zone_nodes = [np.nonzero(ozone == z)[0] for z in range(n_origin_zones)]
    origin = np.empty(n_vehicles, np.int64)
    for z in range(n_origin_zones):
        m = np.nonzero(oz == z)[0]
        if len(m) == 0:
            continue
        nodes = zone_nodes[z]
        origin[m] = nodes[rng.integers(0, len(nodes), size=len(m))]
    # an origin inside the destination zone would arrive without travelling:
    # redraw it uniformly among the nodes outside that zone
    bad = np.nonzero(dzone[origin] == dz)[0]
    for i in bad:
        cand = np.nonzero(dzone != dz[i])[0]
        origin[i] = cand[rng.integers(0, len(cand))]
    t_dep = rng.uniform(0.0, dep_window, size=n_vehicles)
    dep_step = _i32(np.floor(t_dep))
    perm = rng.permutation(n_vehicles)      # vehicle ids are not grouped by OD
    return Scenario(name=name, V=V, L=L, tail=tail, head=head, length=length, lanes=lanes,
                    u=u, kappa=kappa, alpha=alpha, beta=beta, cost=cost, q_fx=q_fx, F=F,
                    phi=phi, psi=psi, w=w, Z=n_dest_zones, node_zone=dzone,
                    dest_feat=dest_feat, N=n_vehicles, origin=_i32(origin[perm]),
                    dest_zone=_i32(dz[perm]), dep_step=dep_step[perm], od=od[perm],
                    n_od=n_od, od_lambda=_f32(lam), T=T, tau=tau, seed=seed,
                    obs_every=300, coords=pts.astype(np.float32))


def city_small(seed: int = 11, n_nodes: int = 400, n_links: int = 1200,
               n_vehicles: int = 20000, T: int = 600, **kw) -> Scenario:
    """A few-hundred-node instance of the city family for oracle-sized parity."""
    return city(seed=seed, n_nodes=n_nodes, n_links=n_links, n_vehicles=n_vehicles,
                T=T, n_origin_zones=8, n_dest_zones=12, dep_window=min(1800.0, T * 0.5),
                name="city_small", **kw)


def tg_toy(u1: float = 2.0, u2: float = 1.0, T: int = 11) -> Scenario:
    """SI-C toy: one agent, Link 1 (15 m) then Link 2 (15 m), free flow.

    Nodes 0 -> 1 -> 2 plus return links so the network is strongly connected;
    the agent departs at step 0 from node 0 with destination node 2, enters
    Link 1 at x = 0 at t = 1 and is observed at the end of the horizon.
    """
    V = 3
    tail = _i32([0, 1, 1, 2])
    head = _i32([1, 2, 0, 1])
    L = 4
    length = _f32([15.0, 15.0, 15.0, 15.0])
    u = _f32([u1, u2, 1.0, 1.0])
    F = 1
    phi = np.zeros((L, F), np.float32)
    psi = np.zeros((L, F), np.float32)
    tt = length.astype(np.float64) / np.maximum(u.astype(np.float64), 1e-3)
    node_zone = _i32([0, 1, 2])
    return Scenario(name="tg_toy", V=V, L=L, tail=tail, head=head, length=length,
                    lanes=_i32(np.ones(L)), u=u, kappa=_f32(np.full(L, 0.2)),
                    alpha=_f32(np.full(L, 2.505)), beta=_f32(np.zeros(L)),
                    cost=_f32(np.ones(L)), q_fx=_capacity_fx(np.full(L, 1.0), 1.0), F=F,
                    phi=_f32(phi), psi=_f32(psi), w=_f32([0.0]), Z=3, node_zone=node_zone,
                    dest_feat=_dest_feature(V, tail, head, tt, node_zone, 3), N=1,
                    origin=_i32([0]), dest_zone=_i32([2]), dep_step=_i32([0]),
                    od=_i32([0]), n_od=1, od_lambda=_f32([1.0]), T=T, tau=0.5, seed=0,
                    obs_every=T)


def line_network(n_links: int = 3, length: float = 100.0, u: float = 10.0,
                 kappa: float = 0.2, q: float = 1.0, N: int = 1, dep=None,
                 T: int = 100, tau: float = 0.5, seed: int = 0) -> Scenario:
    """A chain 0 -> 1 -> ... -> n with return links; all vehicles go from node 0
    to the last node.  Used for closed-form checks (lone vehicle, capacity)."""
    V = n_links + 1
    tails = list(range(n_links)) + list(range(1, V))
    heads = list(range(1, V)) + list(range(n_links))
    tail, head = _i32(tails), _i32(heads)
    L = len(tail)
    lengths = _f32(np.full(L, length))
    us = _f32(np.full(L, u))
    F = 1
    tt = lengths.astype(np.float64) / us.astype(np.float64)
    node_zone = _i32(np.arange(V))
    dep = np.zeros(N, np.int32) if dep is None else _i32(dep)
    return Scenario(name="line", V=V, L=L, tail=tail, head=head, length=lengths,
                    lanes=_i32(np.ones(L)), u=us, kappa=_f32(np.full(L, kappa)),
                    alpha=_f32(np.full(L, 2.505)), beta=_f32(np.zeros(L)),
                    cost=_f32(np.ones(L)), q_fx=_capacity_fx(np.full(L, q), 1.0), F=F,
                    phi=np.zeros((L, F), np.float32), psi=np.zeros((L, F), np.float32),
                    w=_f32([0.0]), Z=V, node_zone=node_zone,
                    dest_feat=_dest_feature(V, tail, head, tt, node_zone, V), N=N,
                    origin=_i32(np.zeros(N)), dest_zone=_i32(np.full(N, V - 1)),
                    dep_step=dep, od=_i32(np.zeros(N)), n_od=1,
                    od_lambda=_f32([float(N)]), T=T, tau=tau, seed=seed, obs_every=T)


def with_platoons(sc: Scenario, dn: float, tau_s: float = 1.0) -> Scenario:
    """The same scenario with agents that are platoons of dn vehicles (Methods:
    step length dt = tau_s dn, jam spacing dn / kappa, a transfer needs dn of
    outflow credit).  Times keep their length in seconds: the outflow capacity in
    vehicles per second (so the credit per step becomes q dt), the departure
    times, the horizon and the observation bins.  The agents are those of sc;
    for the same number of vehicles draw sc with N / dn of them."""
    dt = float(tau_s) * float(dn)
    r = sc.dt / dt
    q = sc.q_fx.astype(np.float64) / 65536.0 / sc.dt
    return sc.copy(dn=float(dn), dt=dt, q_fx=_capacity_fx(q, dt),
                   dep_step=_i32(np.floor(sc.dep_step.astype(np.float64) * r)),
                   T=max(1, int(np.ceil(sc.T * r))),
                   obs_every=max(1, int(round(sc.obs_every * r))))


def random_small(seed: int = 0, side: int = 3, n_vehicles: int = 40, T: int = 80,
                 tau: float = 0.5, length_range=(20.0, 60.0)) -> Scenario:
    """Small grid with heterogeneous links and parameters, dense enough that
    queues, spillback and merges with several candidates occur; used to compare
    the compact oracle against the dense tensor formulation."""
    rng = np.random.default_rng(seed)
    sc = tiny_grid(seed=seed, n_vehicles=n_vehicles, T=T, tau=tau, side=side)
    L = sc.L
    length = _f32(rng.uniform(*length_range, size=L))
    lanes = _i32(rng.integers(1, 3, size=L))
    u = _f32(rng.uniform(8.0, 16.0, size=L))
    kappa = _f32(rng.uniform(0.18, 0.22, size=L) * lanes)
    alpha = _f32(rng.uniform(0.01, 5.0, size=L))
    beta = _f32(rng.uniform(0.0, 5.0, size=L))
    cost = _f32(rng.uniform(0.5, 2.0, size=L))
    q_fx = _capacity_fx(rng.uniform(0.3, 1.0, size=L), 1.0)
    tt = length.astype(np.float64) / u.astype(np.float64)
    phi = np.zeros((L, 3), np.float32)
    psi = np.zeros((L, 3), np.float32)
    phi[:, 0] = -tt / 60.0
    psi[:, 1] = 1.0
    phi[:, 2] = rng.normal(size=L)
    w = _f32([1.0, 4.0, 0.3])
    dest_feat = _dest_feature(sc.V, sc.tail, sc.head, tt, sc.node_zone, sc.Z)
    dep = _i32(rng.integers(0, max(1, T // 3), size=n_vehicles))
    return sc.copy(name="random_small", length=length, lanes=lanes, u=u, kappa=kappa,
                   alpha=alpha, beta=beta, cost=cost, q_fx=q_fx, phi=_f32(phi),
                   psi=_f32(psi), w=w, dest_feat=dest_feat, dep_step=dep)


def custom(tail, head, length, origin, dest_node, dep_step, u=10.0, kappa=0.2, alpha=2.505,
           beta=0.0, cost=1.0, q=1.0, T=50, tau=0.5, seed=0, w=None, phi=None, psi=None,
           node_zone=None, name="custom") -> Scenario:
    """Hand-built network (scalars broadcast to every link).  Destination zones
    are the nodes themselves unless ``node_zone`` is given."""
    tail, head = _i32(tail), _i32(head)
    L = len(tail)
    V = int(max(tail.max(), head.max())) + 1
    bc = lambda v: _f32(np.broadcast_to(np.asarray(v, np.float64), (L,)))
    length, u_, kap, al, be, co = bc(length), bc(u), bc(kappa), bc(alpha), bc(beta), bc(cost)
    if phi is None:
        phi = np.zeros((L, 1), np.float32)
        psi = np.zeros((L, 1), np.float32)
        w = np.zeros(1, np.float32)
    F = phi.shape[1]
    node_zone = _i32(np.arange(V) if node_zone is None else node_zone)
    Z = int(node_zone.max()) + 1
    tt = length.astype(np.float64) / u_.astype(np.float64)
    _check_strongly_connected(V, tail, head)
    origin = _i32(origin)
    N = len(origin)
    dz = node_zone[_i32(dest_node)]
    return Scenario(name=name, V=V, L=L, tail=tail, head=head, length=length,
                    lanes=_i32(np.ones(L)), u=u_, kappa=kap, alpha=al, beta=be, cost=co,
                    q_fx=_capacity_fx(np.broadcast_to(np.asarray(q, np.float64), (L,)), 1.0),
                    F=F, phi=_f32(phi), psi=_f32(psi), w=_f32(w), Z=Z, node_zone=node_zone,
                    dest_feat=_dest_feature(V, tail, head, tt, node_zone, Z), N=N,
                    origin=origin, dest_zone=_i32(dz), dep_step=_i32(dep_step),
                    od=_i32(np.zeros(N)), n_od=1, od_lambda=_f32([float(N)]), T=T, tau=tau,
                    seed=seed, obs_every=T)


def hub(n_spokes: int = 11, n_vehicles: int = 400, T: int = 400, seed: int = 0) -> Scenario:
    """Star network whose centre has n_spokes out-links (a choice set wider
    than the slots a persistent CTA evaluates in parallel) and whose spokes are
    joined in a ring; vehicles travel between random spokes.  Heterogeneous
    lengths, beta and alpha make the choices and merges uneven."""
    rng = np.random.default_rng(seed)
    K = n_spokes
    tail, head = [], []
    for i in range(1, K + 1):
        tail += [0, i, i]
        head += [i, 0, i % K + 1]
    L = len(tail)
    o = rng.integers(1, K + 1, size=n_vehicles)
    dest = (o - 1 + rng.integers(1, K, size=n_vehicles)) % K + 1
    return custom(tail, head, length=rng.uniform(30.0, 90.0, size=L), origin=o, dest_node=dest,
                  dep_step=rng.integers(0, T // 2, size=n_vehicles), beta=rng.uniform(0.0, 2.0, size=L),
                  alpha=rng.uniform(0.5, 4.0, size=L), q=0.6, T=T, seed=seed, name="hub").copy(obs_every=60)


PAPER_RANGES = {"u": (13.9, 22.2), "kappa": (0.18, 0.22), "beta": (0.0, 5.0), "alpha": (0.01, 5.0)}


def paper_mode(seed: int = 0, n_nodes: int = 48, n_links: int = 100, n_vehicles: int = 20_000,
               T: int = 1800, dep_window: float = 1800.0, coverage: float = 0.8, q: float = 1.5,
               w_dest: float = 6.0):
    """Paper-mode calibration problem shaped like the paper's Sioux Falls runs
    (Methods, experimental setting): a planar network of n_nodes / n_links,
    utility beta / c with c = 1 plus one fixed destination term (w_dest times
    minus the free-flow minutes to the destination; with no destination term
    the choice does not steer vehicles home and the network jams), vehicles
    spread evenly over the nodes as origins with random destinations,
    departures uniform over dep_window seconds.  The truth draws u, kappa,
    beta, alpha per link uniformly from the paper's ranges; the model starts
    at the range means.  Sensors: a `coverage` fraction of the links.
    Returns (model, truth), both with `sensors` set."""
    rng = np.random.default_rng(seed)
    pts, und = _planar_graph(rng, n_nodes, n_links // 2)
    tail = _i32(np.concatenate([und[:, 0], und[:, 1]]))
    head = _i32(np.concatenate([und[:, 1], und[:, 0]]))
    L = len(tail)
    length = _f32(np.clip(rng.lognormal(np.log(1500.0), 0.5, size=L), 200.0, 8000.0))   # km-scale links
    origin = _i32(np.arange(n_vehicles) % n_nodes)
    dest = _i32((origin + rng.integers(1, n_nodes, size=n_vehicles)) % n_nodes)
    dep = _i32(np.sort(rng.integers(0, max(1, int(dep_window)), size=n_vehicles)))
    truth_p = {k: _f32(rng.uniform(lo, hi, size=L)) for k, (lo, hi) in PAPER_RANGES.items()}
    mean_p = {k: _f32(np.full(L, 0.5 * (lo + hi))) for k, (lo, hi) in PAPER_RANGES.items()}
    sensors = _i32(np.sort(rng.choice(L, size=int(round(coverage * L)), replace=False)))

    def make(p, name):
        sc = custom(tail, head, length=length, origin=origin, dest_node=dest, dep_step=dep, u=p["u"],
                    kappa=p["kappa"], alpha=p["alpha"], beta=p["beta"], cost=1.0, q=q, T=T, seed=seed,
                    phi=np.zeros((L, 1), np.float32), psi=np.ones((L, 1), np.float32), w=_f32([w_dest]),
                    name=name)
        return sc.copy(obs_every=300, sensors=sensors, coords=pts)

    return make(mean_p, "paper_mode"), make(truth_p, "paper_mode_truth")


def noisy_counts(counts, rng, rel=0.1):
    """Observed counts: simulated counts with multiplicative Gaussian noise of
    relative size `rel` (10 % in the paper), rounded and kept >= 0."""
    c = np.asarray(counts, np.float64)
    return np.maximum(0.0, np.rint(c * (1.0 + rel * rng.standard_normal(c.shape))))


def calibration(n_sensors: int = 2000, T: int = 1800, seed_truth: int = 2, **kw):
    """Calibration-gradient workload: the city network and 30-minute rollouts
    with 5-minute counts on n_sensors links; observations come from a hidden
    ground-truth draw of the 10,240 demand parameters (lambda* = lambda
    exp(N(0, 0.3^2))) and the 16 route-choice coefficients (w* = w + N(0, 0.5^2)).
    Returns (model scenario at the mean parameters, truth scenario)."""
    model = city(T=T, name="calibration", **kw)
    rng = np.random.default_rng(seed_truth)
    mult = np.exp(rng.normal(0.0, 0.3, size=model.n_od))
    truth = city(T=T, name="calibration_truth", demand_mult=mult, demand_seed=seed_truth, **kw)
    truth = truth.copy(w=_f32(model.w + rng.normal(0.0, 0.5, size=model.F)))
    sensors = _i32(np.sort(rng.choice(model.L, size=min(n_sensors, model.L), replace=False)))
    return model.copy(sensors=sensors), truth.copy(sensors=sensors)


def batched_scenarios(n: int = 64, seed: int = 3, n_min: int = 10_000, n_max: int = 200_000,
                      n_perturbed: int = 500, T: int = 1800, **city_kw):
    """Control-candidate scenarios on one city network: vehicle counts
    log-uniform over [n_min, n_max], and in each scenario the outflow capacity
    of n_perturbed random links scaled by U(0.7, 1.0); each scenario has its own
    demand draw and random key."""
    rng = np.random.default_rng(seed)
    base = city(T=T, **city_kw)
    out = []
    for k in range(n):
        nk = int(np.exp(rng.uniform(np.log(n_min), np.log(n_max))))
        mult = np.ones(base.L)
        links = rng.choice(base.L, size=min(n_perturbed, base.L), replace=False)
        mult[links] = rng.uniform(0.7, 1.0, size=len(links))
        q = np.rint(base.q_fx.astype(np.float64) * mult)
        r = np.random.default_rng([seed, k])
        idx = r.choice(base.N, size=min(nk, base.N), replace=False)
        idx.sort()
        sc = base.copy(name=f"candidate_{k}", q_fx=_i32(np.maximum(q, 1)), N=len(idx),
                       origin=base.origin[idx], dest_zone=base.dest_zone[idx], dep_step=base.dep_step[idx],
                       od=base.od[idx], seed=int(base.seed) + 1000 * (k + 1), scenario_id=k)
        out.append(sc)
    return out
