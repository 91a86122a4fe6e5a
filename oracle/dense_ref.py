"""Dense literal reference of the method on small inputs (TEST INFRASTRUCTURE).

The paper's own formulation, written out with torch CPU float64 tensors and
torch.autograd standing in for jax.grad:
  * agent state X in R^{N x (L + V)}: X[i, j] = position of agent i on link j,
    -M elsewhere (SI-A); columns L.. are the origin queues as virtual inflow
    links of length 0, one per node;
  * f (SI-A, Alg. S1 with the text's sorted headways): per link, argsort of the
    positions, headways, min(u dt, max(h - dn/kappa, 0)) and the TG clip
    min(x', L + x' - sg(x')) (Eq. eq:tg);
  * g (SI-B, Alg. S2): utility V = beta/c + features (text of SI-B) with -M
    outside the choice set, z = softmax(V), pi = softmax((log z + g)/tau)
    (Eq. gumbel), l' = onehot + pi - sg(pi) (Eq. straigththrough), the masks,
    p = ((I_X>=0 . alpha) * l)^T, V' = p - M 1_{p=0}, the same sampling along the
    agents, a = max(l)^T * a' (max(l) constant), and the transfer
    X <- X - (M + x) * I_remove + (M + x - sg(x)) * I_add (Eq. transfer);
  * counting (SI-D): Q = sum(I_Q + I'_Q - sg(I'_Q)) at the link midpoint, each
    vehicle weighted by the demand weight 1 + (lambda - sg lambda)/lambda.
Discrete decisions are taken on the float64 values; min/max ties of the
car-following update follow the same dead-band tag rule as the oracle.  Gumbel
noise comes from the oracle's Philox generator (the random numbers are inputs).
Only for a few hundred agents and tens of links.
"""
from __future__ import annotations

import numpy as np
import torch

from .oracle import gumbel

FREE, CONG, STOP = 0, 1, 2


class Tape:
    """Records every discrete decision and every stop_gradient value of a run so
    that a second run can evaluate the surrogate F_sur(theta) with all of them
    frozen at theta_0 (the function whose derivative the method takes)."""

    def __init__(self):
        self.items = []
        self.pos = None          # None: recording; else: replay cursor

    def replaying(self):
        return self.pos is not None

    def rewind(self):
        self.pos = 0

    def sg(self, x):
        if self.pos is None:
            v = x.detach().clone()
            self.items.append(v)
            return v
        v = self.items[self.pos]
        self.pos += 1
        return v

    def dec(self, v):
        if self.pos is None:
            self.items.append(v)
            return v
        r = self.items[self.pos]
        self.pos += 1
        return r


def _choice_sets(sc):
    out_links = [[] for _ in range(sc.V)]
    for j in range(sc.L):
        out_links[int(sc.tail[j])].append(j)
    link_set = []
    for l in range(sc.L):
        n = int(sc.head[l])
        cand = [m for m in out_links[n] if int(sc.head[m]) != int(sc.tail[l])]
        link_set.append(cand if cand else list(out_links[n]))
    return out_links, link_set


def run(sc, T=None, ybar=None, xbarT=None, tape=None, params=None):
    """Forward (and, with ybar, reverse) pass.  Returns (outputs, grads, trace).

    tape: a Tape to record (fresh) or to replay (after rewind()): in replay the
    decisions and stop_gradient values are the recorded ones.  params: optional
    dict overriding the parameter values (u, kappa, alpha, alpha_origin, beta,
    cost, w, od_lambda) -- used for finite differences of the surrogate."""
    T = sc.T if T is None else T
    tape = Tape() if tape is None else tape
    sg = tape.sg
    dec = tape.dec
    params = {} if params is None else params
    dt64 = torch.float64
    N, L, V, F = sc.N, sc.L, sc.V, sc.F
    M = float(np.float32(sc.M))
    dt, dn, tau = float(np.float32(sc.dt)), float(np.float32(sc.dn)), float(np.float32(sc.tau))
    eps_arr, eps_tag = float(np.float32(sc.eps_arr)), float(np.float32(sc.eps_tag))
    P = lambda k, a: torch.tensor(np.asarray(params.get(k, a), np.float64), dtype=dt64, requires_grad=True)
    u, kappa, alpha, beta, cost = P("u", sc.u), P("kappa", sc.kappa), P("alpha", sc.alpha), P("beta", sc.beta), P("cost", sc.cost)
    w = P("w", sc.w)
    alpha_o = torch.tensor(float(np.asarray(params.get("alpha_origin", np.float32(sc.alpha_origin))).reshape(-1)[0]),
                           dtype=dt64, requires_grad=True)
    lam = P("od_lambda", sc.od_lambda)
    phi = torch.tensor(sc.phi.astype(np.float64))
    psi = torch.tensor(sc.psi.astype(np.float64))
    length = torch.tensor(sc.length.astype(np.float64))
    dest_feat = torch.tensor(sc.dest_feat.astype(np.float64))
    udt = u * dt
    s = dn / kappa
    U = beta / cost + phi @ w
    G = psi @ w
    half = length * 0.5
    dtag = (eps_tag * (1.0 + length)).detach()
    out_links, link_set = _choice_sets(sc)
    dn_fx = int(round(sc.dn * 65536))
    cap = np.maximum(sc.q_fx.astype(np.int64), dn_fx)
    credit = cap.copy()
    exits_w = [torch.zeros((), dtype=dt64) for _ in range(L)]
    # demand weights (value 1, derivative 1/lambda)
    lam_d = sg(lam)
    wv = 1.0 + (lam[sc.od] - lam_d[sc.od]) / lam_d[sc.od]
    # origin queues: vehicles of each node by (departure step, id)
    fifo = [sorted(np.nonzero(sc.origin == n)[0].tolist(), key=lambda i: (int(sc.dep_step[i]), i)) for n in range(V)]
    fptr = [0] * V
    vlink = np.full(N, -1, np.int64)            # real link, -1 origin queue, -2 arrived
    seq = np.zeros(N, np.int64)
    X = torch.full((N, L + V), -M, dtype=dt64)
    X = X.clone()
    for i in range(N):                           # every agent starts on its origin's virtual link
        X[i, L + int(sc.origin[i])] = 0.0
    nb = (T + sc.obs_every - 1) // sc.obs_every
    Cprev = [torch.zeros((), dtype=dt64) for _ in range(L)]
    ys = []
    trace = []
    for t in range(T):
        # ---------------- f: car-following (SI-A) ----------------
        # every link at once (Alg. S1 maps one link's update over all links):
        # the agents on links in order of (link, -x, entry), i.e. per link
        # argsort(-x) with ties by entry (recorded; a replay takes the record)
        on = np.nonzero(vlink >= 0)[0]
        if len(on):
            if tape.replaying():
                order = dec(None)
            else:
                xo = X[on, vlink[on]].detach().numpy()
                order = dec(on[np.lexsort((seq[on], -xo, vlink[on]))])
            lk = vlink[order]
            tl = torch.tensor(lk)
            first = torch.tensor(np.r_[True, lk[1:] != lk[:-1]])           # the link's leader
            xs = X[torch.tensor(order), tl]
            h = torch.where(first, torch.full_like(xs, M), torch.cat([xs[:1], xs[:-1]]) - xs)
            d = h - s[tl]
            dd = d.detach()
            tag = dec(torch.where(dd <= dtag[tl], STOP, torch.where(dd >= udt[tl].detach() - dtag[tl], FREE, CONG)))
            # value min(u dt, max(d, 0)); derivative of the tagged branch
            path = torch.where(tag == FREE, udt[tl] + 0 * d, torch.where(tag == CONG, d, 0 * d))
            val = sg(torch.minimum(udt[tl], torch.clamp(d, min=0.0)))
            dx = val + (path - sg(path))
            xp = xs + dx
            xlim = length[tl] + xp - sg(xp)
            clipped = dec((xp.detach() > xlim.detach()))
            xn = torch.where(clipped, xlim, xp)
            X = X.index_put((torch.tensor(order), tl), xn)
        # ---------------- g: node model (SI-B) ----------------
        credit = np.minimum(credit + sc.q_fx.astype(np.int64), cap)
        def vacancy():                      # rearmost position beyond the jam spacing, or empty
            Xd = X.detach().numpy()
            vac = np.ones(L, bool)
            for j in range(L):
                on = np.nonzero(vlink == j)[0]
                if len(on):
                    vac[j] = float(Xd[on, j].min()) > float(s[j].detach())
            return vac

        def candidates():                   # arrived leaders with credit, heads of origin queues
            Xd = X.detach().numpy()
            out = []                        # (agent, source column, set, is_link)
            for j in range(L):
                on = np.nonzero(vlink == j)[0]
                arr = [i for i in on if Xd[i, j] >= float(length[j]) - eps_arr]
                assert len(arr) <= 1
                if arr and credit[j] >= dn_fx:
                    out.append((arr[0], j, link_set[j], True))
            for n in range(V):
                if fptr[n] < len(fifo[n]) and int(sc.dep_step[fifo[n][fptr[n]]]) <= t:
                    out.append((fifo[n][fptr[n]], L + n, out_links[n], False))
            return out
        rec = tape.replaying()
        vacant = dec(None if rec else vacancy())
        cands = dec(None if rec else candidates())
        sinks = [(i, c) for (i, c, _, is_link) in cands
                 if int(sc.node_zone[int(sc.head[c]) if is_link else c - L]) == int(sc.dest_zone[i])]
        sink_ids = {i for i, _ in sinks}
        Vm = torch.full((N, L), -M, dtype=dt64)
        gm = torch.zeros((N, L), dtype=dt64)
        arrived = torch.zeros(N, dtype=dt64)
        ri, rm, rz, rg = [], [], [], []     # (agent, link of its choice set, its zone, Gumbel)
        for (i, c, cs, is_link) in cands:
            if i in sink_ids:
                continue
            for k, m in enumerate(cs):
                ri.append(int(i)); rm.append(int(m)); rz.append(int(sc.dest_zone[i]))
                rg.append(gumbel(sc.seed, sc.scenario_id, int(i), t, 0, k))
            arrived[i] = 1.0
        if ri:
            ti, tm = torch.tensor(ri), torch.tensor(rm)
            hm = torch.tensor(sc.head[rm].astype(np.int64))
            Vm = Vm.index_put((ti, tm), U[tm] + G[tm] * dest_feat[torch.tensor(rz), hm])
            gm[ti, tm] = torch.tensor(rg, dtype=dt64)
        logz = torch.log_softmax(Vm, dim=1)
        pi = torch.softmax((logz + gm) / tau, dim=1)
        onehot = torch.zeros_like(pi)
        onehot[torch.arange(N), dec(torch.argmax(pi.detach(), dim=1))] = 1.0
        lp = onehot + pi - sg(pi)
        vac_t = torch.tensor(vacant.astype(np.float64))
        l = arrived[:, None] * (vac_t[None, :] * lp)
        # merge priority of each agent's source: its link's alpha, alpha_origin in an origin queue
        alpha_src = torch.cat([alpha, alpha_o.reshape(1)])[torch.tensor(np.where(vlink >= 0, vlink, L))]
        p = (alpha_src[:, None] * l).T                               # L x N
        Vp = p - M * dec((p.detach() == 0).to(dt64))
        gp = torch.tensor([gumbel(sc.seed, sc.scenario_id, i, t, 1, 0) for i in range(N)], dtype=dt64)
        logzp = torch.log_softmax(Vp, dim=1)
        pip = torch.softmax((logzp + gp[None, :]) / tau, dim=1)
        oh = torch.zeros_like(pip)
        oh[torch.arange(L), dec(torch.argmax(pip.detach(), dim=1))] = 1.0
        ap = oh + pip - sg(pip)
        a = sg(l.max(dim=0).values)[:, None] * ap                    # L x N, max(l) constant
        I_x = (vlink[:, None] == np.arange(L + V)[None, :]).astype(np.float64)
        I_x[vlink == -1, :] = 0.0
        for i in range(N):
            if vlink[i] == -1:
                I_x[i, L + int(sc.origin[i])] = 1.0
        I_x = torch.tensor(I_x)
        I_remove = I_x * a.sum(dim=0)[:, None]
        I_add = torch.cat([a.T, torch.zeros((N, V), dtype=dt64)], dim=1)
        amx = dec(X.detach().argmax(dim=1))
        xmax = X[torch.arange(N), amx]                               # x = max along links
        X = X - (M + xmax)[:, None] * I_remove + (M + xmax - sg(xmax))[:, None] * I_add
        # sinks leave the network (constant removal mask)
        for i, c in sinks:
            X = X.index_put((torch.tensor([i]), torch.tensor([c])), X[i, c] - (M + X[i, c]))
        # discrete bookkeeping of the transfers
        def winner_map():
            amax = a.detach()
            return {int(torch.argmax(amax[m])): m for m in range(L) if float(amax[m].max()) > 0.5}
        winners = dec(None if tape.replaying() else winner_map())
        for (i, c, cs, is_link) in cands:
            leaves = i in winners or i in sink_ids
            if not leaves:
                continue
            if is_link:
                credit[c] -= dn_fx
                exits_w[c] = exits_w[c] + wv[i]
            else:
                fptr[c - L] += 1
            if i in sink_ids:
                vlink[i] = -2
            else:
                vlink[i] = winners[i]
                seq[i] = t + 1
        trace.append(dict(vlink=vlink.copy(), winners=dict(winners), sinks=sorted(sink_ids),
                          cands=sorted(int(c[0]) for c in cands)))
        # ---------------- observation (SI-D) ----------------
        if (t + 1) % sc.obs_every == 0 or t + 1 == T:
            y = []
            for j in range(L):
                xc = X[:, j]
                ind = dec((xc.detach() >= half[j]).to(dt64))
                sgm = torch.sigmoid((5.0 / length[j]) * (xc - half[j]))
                Q = (wv * (ind + sgm - sg(sgm))).sum()
                C = exits_w[j] + Q
                y.append(C - Cprev[j])
                Cprev[j] = C
            ys.append(torch.stack(y))
    Y = torch.stack(ys)                                             # n_bins x L
    xT = torch.zeros(N, dtype=dt64)
    xT_list = []
    for i in range(N):
        j = int(vlink[i])
        xT_list.append(X[i, j] if j >= 0 else torch.zeros((), dtype=dt64))
    xT = torch.stack(xT_list)
    outputs = dict(counts=np.rint(Y.detach().numpy()).astype(np.int64), x_T=xT.detach().numpy(),
                   vlink=vlink.copy())
    grads = None
    loss = None
    if ybar is not None:
        loss = (Y * torch.tensor(np.asarray(ybar, np.float64))).sum()
        if xbarT is not None:
            loss = loss + (xT * torch.tensor(np.asarray(xbarT, np.float64))).sum()
        outputs["loss"] = float(loss.detach())
    if ybar is not None and not tape.replaying():
        params = [u, kappa, alpha, alpha_o, beta, cost, w, lam]
        gs = torch.autograd.grad(loss, params, allow_unused=True)
        names = ["u", "kappa", "alpha", "alpha_origin", "beta", "cost", "w", "od_lambda"]
        grads = {k: (np.zeros(p.shape) if g is None else g.numpy().reshape(p.shape)) for k, g, p in zip(names, gs, params)}
        grads["alpha_origin"] = np.atleast_1d(grads["alpha_origin"])
    return outputs, grads, trace
