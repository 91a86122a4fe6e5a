"""Lockstep comparison of a float32 simulator with the FP64 oracle, with
near-tie flags and resynchronisation (used by test_oracle_lockstep.py on the
CPU and test_gpu_fp64_lockstep.py on the GPU).

Both sides start from the same state and take one step at a time.  The float
side takes every decision in float32.  A decision can go the other way in
float32 only where its margin in the FP64 oracle is smaller than what float32
resolves:
  * the arrival test of a link's leader, x >= L - eps_arr (SI-B Alg. S2), or
    the vacancy test of a link's rearmost vehicle, x_min > dn / kappa (SI-B,
    merge validity), within DELTA_POS metres of its threshold;
  * the top-2 gap of a link choice, argmax(V + g) (SI-B Eqs. gumbel and
    straigththrough), or of a merge, argmax(alpha_src + g') (SI-B merge
    choice), below DELTA_G.
At the first integer mismatch of a step every differing decision must be
explained by such a near-tie of the oracle in that step (at its own link or
node, or at the target link it involves).  The step is then flagged, the
oracle's state is copied into the float side and the run goes on.  Any other
mismatch fails.  Off flagged steps the integer state (vehicle links, queue
order, outflow credit, exits, origin queues) and every decision must be
identical, and the float outputs are measured against FP64.
"""
from __future__ import annotations

import numpy as np

DELTA_POS = 5e-3     # metres: position compares (arrival line, jam spacing)
DELTA_G = 1e-4       # key units: top-2 gaps of the choice and merge argmaxes

RECORDS = ("link_cand", "link_target", "node_cand", "node_target", "link_in")
INT_STATE = ("veh_link", "veh_rank", "link_credit", "link_exits", "fifo_off")
TGT_SINK, TGT_BLOCKED = -2, -3


class UnexplainedMismatch(AssertionError):
    pass


def explain(gr, orr):
    """Near-ties of the oracle's step that explain every decision in which the
    float side's records ``gr`` differ from the oracle's ``orr``.  Returns the
    list of (kind, site, margin); raises UnexplainedMismatch otherwise."""
    am, vm = orr["arr_margin"], orr["vac_margin"]
    lm, nm, mm = orr["link_margin"], orr["node_margin"], orr["merge_margin"]

    def near_vac(m):
        return m >= 0 and abs(vm[m]) < DELTA_POS

    reasons, bad, touched = [], [], set()

    def target_mismatch(kind, src, og, gg, margin):
        # the same candidate chose differently: its choice keys were within
        # DELTA_G, or the chosen link's vacancy was within DELTA_POS (a blocked
        # record hides the link, but without a choice near-tie both sides chose
        # the one the other side names)
        if TGT_SINK in (og, gg):
            bad.append((kind, src, int(og), int(gg)))
            return
        touched.update(m for m in (og, gg) if m >= 0)
        if margin < DELTA_G:
            reasons.append(("choice", kind, src, float(margin)))
        elif near_vac(og) or near_vac(gg):
            m = og if near_vac(og) else gg
            reasons.append(("vacancy", "link", int(m), float(vm[m])))
        else:
            bad.append((kind, src, int(og), int(gg)))

    cand = np.nonzero(gr["link_cand"] != orr["link_cand"])[0]
    for j in cand:
        if abs(am[j]) < DELTA_POS:
            reasons.append(("arrival", "link", int(j), float(am[j])))
            touched.update(m for m in (orr["link_target"][j], gr["link_target"][j]) if m >= 0)
        else:
            bad.append(("link_cand", int(j), int(orr["link_cand"][j]), int(gr["link_cand"][j])))
    for j in np.setdiff1d(np.nonzero(gr["link_target"] != orr["link_target"])[0], cand):
        target_mismatch("link", int(j), orr["link_target"][j], gr["link_target"][j], lm[j])
    for n in np.nonzero(gr["node_cand"] != orr["node_cand"])[0]:
        bad.append(("node_cand", int(n), int(orr["node_cand"][n]), int(gr["node_cand"][n])))
    for n in np.nonzero((gr["node_target"] != orr["node_target"]) & (gr["node_cand"] == orr["node_cand"]))[0]:
        target_mismatch("node", int(n), orr["node_target"][n], gr["node_target"][n], nm[n])
    for m in np.nonzero(gr["link_in"] != orr["link_in"])[0]:
        if mm[m] < DELTA_G:
            reasons.append(("merge", "link", int(m), float(mm[m])))
        elif near_vac(m):
            reasons.append(("vacancy", "link", int(m), float(vm[m])))
        elif m not in touched:
            bad.append(("link_in", int(m), int(orr["link_in"][m]), int(gr["link_in"][m])))
    if bad:
        raise UnexplainedMismatch(f"decisions differ away from near-ties: {bad[:8]} (explained: {reasons[:8]})")
    return reasons


def _rel_len(a, b, length):
    return float(np.max(np.abs(a - b) / length)) if a.size else 0.0


def _rel(a, b, floor):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor))) if a.size else 0.0


def run(fsim, osim, T, check_outputs=True):
    """Step the float simulator ``fsim`` (GPU Simulator, or the oracle's float
    build) and the FP64 oracle ``osim`` together for T steps.  Both expose
    reset / step / records / state / set_state / outputs.  Returns a report:
    flagged steps with their near-ties, and the largest relative error of each
    float output against FP64 off flagged steps and bins."""
    sc = osim.sc
    fsim.reset(T)
    osim.reset(T)
    flags = []
    flagged_bins = set()
    err = dict(positions=0.0, speed=0.0, travel_time=0.0)
    identical_steps = 0
    for t in range(T):
        fsim.step(1)
        osim.step(1)
        gr, orr = fsim.records(), osim.records()
        gs, os_ = fsim.state(), osim.state()
        same = all(np.array_equal(gr[k], orr[k]) for k in RECORDS)
        same = same and all(np.array_equal(gs[k], os_[k]) for k in INT_STATE)
        on = os_["veh_link"] >= 0
        same = same and np.array_equal(gs["veh_entry"][on], os_["veh_entry"][on])
        if not same:
            if all(np.array_equal(gr[k], orr[k]) for k in RECORDS):
                raise UnexplainedMismatch(f"step {t}: state differs with identical decisions")
            reasons = explain(gr, orr)
            flags.append((t, reasons))
            flagged_bins.add(t // sc.obs_every)
            fsim.set_state(os_, t + 1)
            continue
        identical_steps += 1
        if on.any():
            # positions relative to their link's length (they range over [0, L_j])
            lj = np.asarray(sc.length, np.float64)[os_["veh_link"][on]]
            err["positions"] = max(err["positions"], _rel_len(gs["veh_pos"][on], os_["veh_pos"][on], lj))
            err["positions_abs_m"] = max(err.get("positions_abs_m", 0.0),
                                         float(np.max(np.abs(gs["veh_pos"][on] - os_["veh_pos"][on]))))
    rep = dict(flags=flags, n_flags=len(flags), identical_steps=identical_steps, steps=T,
               flagged_bins=sorted(flagged_bins))
    if check_outputs:
        fo, oo = fsim.outputs(), osim.outputs()
        keep = np.array([b not in flagged_bins for b in range(fo["counts"].shape[0])])
        rep["bins_compared"] = int(keep.sum())
        np.testing.assert_array_equal(fo["counts"][keep], oo["counts"][keep])
        for k in ("speed", "travel_time"):
            a, b = np.asarray(fo[k][keep], np.float64), np.asarray(oo[k][keep], np.float64)
            err[k] = _rel(a, b, 1e-6) if a.size else 0.0
        if not flags:
            for k in ("n_waiting", "n_on", "n_arrived"):
                np.testing.assert_array_equal(fo[k][:T + 1], oo[k][:T + 1], err_msg=k)
    rep["max_rel_err"] = err
    return rep
