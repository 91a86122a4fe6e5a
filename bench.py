"""Benchmark of the simulator hot path on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One benchmark step = one forward rollout of the city-scale workload
(12,000 nodes / 36,000 links, 1,000,000 vehicles, 3,600 steps of dt = 1 s):
every simulator step of the path (departures, car-following, credit and arrival,
link choice, merge, transfer, observation) runs in the CUDA kernels.  The
metric is vehicle-steps per second (N * T / rollout time); x-real-time is
T dt / rollout time.  Prints one JSON line on rank 0.

Timing: W untimed rollouts, then K rollouts each timed with CUDA events on the
stream the kernels run on; the ~40 MB working set is smaller than L2, so L2 is
flushed (256 MB write) before every timed rollout.  Under torchrun every rank
runs an independent replica (the single-scenario path does not shard) and the
slowest rank's time is used.

--impl reference times the CPU oracle (double precision, one thread) on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = ("city-scale forward rollout: random planar graph 12,000 nodes / 36,000 links, "
            "1,000,000 vehicles from 10,240 OD parameters departing over 30 min, 3,600 steps of dt=1 s")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--T", type=int, default=3600)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--small", action="store_true", help="small network (for profiling captures)")
    ap.add_argument("--stage", type=int, default=0, help="queue slots per link block (0 = autotune)")
    ap.add_argument("--executor", default="auto", choices=["auto", "step", "persistent"],
                    help="forward executor of the timed rollouts")
    ap.add_argument("--no-compare", action="store_true", help="skip timing the other forward executor")
    ap.add_argument("--no-fwd-bwd", action="store_true", help="skip the calibration-gradient leg")
    ap.add_argument("--no-platoons", action="store_true", help="skip the platoon (dn = 30) leg")
    ap.add_argument("--no-calib-loop", action="store_true", help="skip the calibration-loop leg")
    ap.add_argument("--calib-iters", type=int, default=60, help="most iterations (the early stop comes first)")
    ap.add_argument("--no-paper-mode", action="store_true", help="skip the paper-mode calibration leg")
    ap.add_argument("--paper-iters", type=int, default=20)
    ap.add_argument("--paper-lr", type=float, default=0.02, help="paper-mode AdamW step, in units of each range")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-scenario leg")
    ap.add_argument("--batch-n", type=int, default=64)
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg")
    ap.add_argument("--serve-requests", type=int, default=256)
    return ap.parse_args()


from paper_2603_25068_b300.replicas import dist_env, slowest, whole_job_rate  # noqa: E402


def make_scenario(args):
    from paper_2603_25068_b300 import scenario as S
    if args.small:
        sc = S.city(seed=1, n_nodes=3000, n_links=9000, n_vehicles=250_000, T=args.T,
                    n_origin_zones=20, n_dest_zones=32, name="city_quarter")
    else:
        sc = S.city(seed=1, T=args.T)
    return sc


# ------------------------------------------------------------------ CPU oracle
# The CPU arm times the fp64 oracle on one fixed window of the rollout: its
# first CPU_WINDOW steps (the first 5-minute bin), the same window for the
# reference arm and for the cpu_baseline leg, which also times the GPU on it.
# The oracle needs minutes for the whole hour, so the window is a bounded
# sample; it is front-loaded (departures under way, few vehicles on links), so
# its total rate (N x steps / wall) flatters the CPU and the active rate
# (vehicle-steps on links / wall) is the comparable figure.
CPU_WINDOW = 300


def oracle_window(sc, steps):
    """The double-precision oracle over steps [0, steps) of sc: wall seconds
    and vehicle-steps on links (sum over the steps of the vehicles on links at
    their start)."""
    from oracle.oracle import OracleSim
    o = OracleSim(sc, "fp64")
    o.reset(sc.T)
    t0 = time.perf_counter()
    o.step(steps)
    wall = time.perf_counter() - t0
    n_on = o.outputs()["n_on"][:steps]
    return wall, float(np.sum(n_on))


def cpu_cores_used():
    return 1


def window_text(sc, steps, active):
    return (f"fp64 oracle over steps 0-{steps - 1} of the {sc.T}-step rollout of the same workload (its "
            f"first {steps * sc.dt / 60:g} minutes: departures under way, {active:,.0f} vehicle-steps on "
            f"links out of {sc.N * steps:,} vehicle-steps), 1 thread")


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    sc = make_scenario(args)
    steps = min(CPU_WINDOW, sc.T)
    times, active = [], 0.0
    for k in range(args.warmup + args.steps):
        wall, active = oracle_window(sc, steps)
        if k >= args.warmup:
            times.append(wall)
    vs = sc.N * steps * len(times) / sum(times)
    line = {
        "impl": "reference", "metric": "vehicle-steps/s", "value": vs, "unit": "vehicle-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * statistics.mean(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(args, sc, 1),
        "cpu_baseline": {"value": vs, "unit": "vehicle-steps/s", "cores": cpu_cores_used(),
                         "kind": "oracle", "sample": window_text(sc, steps, active),
                         "active_value": active * len(times) / sum(times)},
        "e2e": {"value": vs, "unit": "vehicle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_of(args, sc, ws):
    """The workload description of both arms' lines."""
    return {"workload": WORKLOAD if not args.small else "city_quarter (profiling case)",
            "step": f"one {sc.T}-step forward rollout", "vehicles": sc.N, "links": sc.L,
            "l2": "flushed (256 MB write) before each timed rollout", "parallelism": f"replicas x{ws}"}


def run_cpu_baseline(args, sc, sim, out, flush, dev, stream):
    """The oracle on the CPU window of the workload, the GPU on the same window,
    and two more oracle timings: the tiny grid in full and the first 300 steps
    of the calibration gradient (forward with history + reverse mode)."""
    import torch
    from oracle.oracle import OracleSim
    from paper_2603_25068_b300 import scenario as S
    from paper_2603_25068_b300.sim import Simulator
    steps = min(CPU_WINDOW, sc.T)
    wall, active = oracle_window(sc, steps)
    # the GPU on the same window
    sim.rollout(steps, device=True, out=out)
    ms = []
    for k in range(5):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.rollout(steps, device=True, out=out)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms.append(e0.elapsed_time(e1))
    g_s = float(np.median(ms)) / 1000.0
    # the tiny grid (5 x 5, 1,000 vehicles, 300 steps) in full
    tiny = S.tiny_grid()
    t0 = time.perf_counter()
    OracleSim(tiny, "fp64").rollout()
    t_tiny = time.perf_counter() - t0
    tg = Simulator(tiny, device=dev.index, stream=stream)
    tg.rollout()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(10):
        tg.rollout()
    g_tiny = (time.perf_counter() - t0) / 10
    tg.close()
    # the calibration gradient's first 300 steps, forward + reverse
    model, _ = S.calibration()
    cal = model.copy(T=300, obs_every=60)
    yb = np.zeros((5, cal.L))
    yb[:, cal.sensors] = np.random.default_rng(9).normal(size=(5, len(cal.sensors)))
    t0 = time.perf_counter()
    o = OracleSim(cal, "fp64", keep_history=True)
    o.rollout()
    o.backward(yb)
    t_cal = time.perf_counter() - t0
    del o
    cs = Simulator(cal, device=dev.index, stream=stream, ckpt_every=60, route_cap=256)
    cs.rollout()
    cs.backward(yb.astype(np.float32))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    cs.rollout()
    cs.backward(yb.astype(np.float32))
    torch.cuda.synchronize(dev)
    g_cal = time.perf_counter() - t0
    cs.close()
    return {"value": sc.N * steps / wall, "unit": "vehicle-steps/s", "cores": cpu_cores_used(), "kind": "oracle",
            "sample": window_text(sc, steps, active), "host_cores": os.cpu_count(),
            "active_value": active / wall,
            "gpu_same_window": {"ms": 1000 * g_s, "value": sc.N * steps / g_s, "active_value": active / g_s,
                                "ratio": wall / g_s},
            "tiny_grid_full": {"workload": "5 x 5 grid, 1,000 vehicles, 300 steps (whole rollout)",
                               "oracle_s": t_tiny, "gpu_s": g_tiny,
                               "oracle_vehicle_steps_per_s": tiny.N * tiny.T / t_tiny},
            "calibration_first_300_steps": {"workload": f"calibration gradient, first 300 of {model.T} steps "
                                                        "(forward + reverse mode, checkpoints every 60 on the GPU)",
                                            "oracle_s": t_cal, "gpu_s": g_cal, "ratio": t_cal / g_cal}}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.p is not None:
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                out, _ = self.p.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except (ValueError, IndexError):
                continue
            for k, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(k)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ byte model
def avg_choice_degree(sc):
    deg = np.bincount(sc.tail, minlength=sc.V)
    # choice set after a link: out-degree of its head minus the U-turn
    d = deg[sc.head].astype(np.float64)
    has_u = np.zeros(sc.L)
    key = set(zip(sc.tail.tolist(), sc.head.tolist()))
    for j in range(sc.L):
        has_u[j] = (int(sc.head[j]), int(sc.tail[j])) in key
    d = np.where(d - has_u > 0, d - has_u, d)
    return float(d.mean())


def kernel_a_bytes(sc, n_on, n_cand, deg):
    """Algorithmic bytes of the node-model / car-following kernel for one step:
    8 B per vehicle on the network (read + write its position), 32 B per link
    (queue head/length, credit, length/speed/spacing), 8 B per origin queue
    (pointer, head departure step), and 60 + 24 deg B per node-model candidate
    (vehicle, destination, choice set, per-candidate-link utility terms,
    destination feature and vacancy, merge word)."""
    return 8.0 * n_on + 32.0 * sc.L + 8.0 * sc.V + (60.0 + 24.0 * deg) * n_cand


NOMINAL_HBM_GBS = 7700.0           # B300 HBM3e nominal bandwidth (context beside the measured peak)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2603_25068_b300", "csrc")
    for f in sorted(os.listdir(csrc)):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, workload_key, launch_units):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(kernel, {}).get(workload_key)
    if not e or e.get("source_hash") != source_hash():
        return None
    # scale a smaller capture to one launch of this workload by units processed
    return e["dram_bytes_per_launch"] * launch_units / e["units_per_launch"]


# ------------------------------------------------------------------ fwd + bwd
def run_platoons(args, dev, stream, flush, ws):
    """Platoon form of the forward rollout (Methods: dt = tau dn, tau = 1 s):
    the city network's 1,000,000 vehicles as 33,334 agents of 30 vehicles, one
    hour in 120 steps of 30 s, departures over the first 30 minutes."""
    import torch
    from paper_2603_25068_b300 import scenario as S
    from paper_2603_25068_b300.sim import Simulator
    dn = 30
    sc = S.with_platoons(S.city(n_vehicles=1_000_000 // dn), dn)
    sim = Simulator(sc, device=dev.index, stream=stream)
    out = sim.rollout(device=True)
    for _ in range(max(args.warmup, 3)):
        sim.rollout(device=True, out=out)
    reps = max(args.steps, 20)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    torch.cuda.synchronize(dev)
    for k in range(reps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        sim.rollout(device=True, out=out)
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    ms = slowest(sum(a.elapsed_time(b) for a, b in ev) / 1000.0, dev) * 1000.0 / reps
    n_arr = int(sim.outputs()["n_arrived"][-1]) if hasattr(sim, "outputs") else None
    sim.close()
    horizon_s = sc.T * sc.dt
    return {"workload": f"city network, {sc.N * dn:,} vehicles as {sc.N:,} platoons of {dn}, "
                        f"{sc.T} steps of {sc.dt:g} s (one hour)",
            "ms_per_rollout": ms, "x_real_time": horizon_s / (ms / 1000.0),
            "agent_steps_per_s": ws * sc.N * sc.T / (ms / 1000.0),
            "vehicle_seconds_per_s": ws * sc.N * dn * horizon_s / (ms / 1000.0),
            "executor": "persistent", "arrived_platoons": n_arr,
            "timing": "CUDA events on the simulator's stream, L2 flushed before each rollout"}


def run_chicago_twin(args, dev, stream, flush, ws):
    """A synthetic network shaped like the paper's nowcasting case (Results,
    nowcasting: the Chicago Sketch network of 993 nodes and 2,571 links, about
    one million vehicles as platoons of 30, a one-hour horizon).  The network
    itself is not available: the city generator at 993 nodes and 2,570
    directed links (its links come in opposite pairs), 1,000,020 vehicles as
    33,334 platoons of 30 departing over the first 30 minutes, 120 steps of
    30 s.  Context beside the paper's 3.0 s forward on an H200, not a target."""
    import torch
    from paper_2603_25068_b300 import scenario as S
    from paper_2603_25068_b300.sim import Simulator
    dn = 30
    sc = S.with_platoons(S.city(seed=5, n_nodes=993, n_links=2570, n_vehicles=33_334, T=3600,
                                n_origin_zones=20, n_dest_zones=32, name="chicago_shaped"), dn)
    sim = Simulator(sc, device=dev.index, stream=stream)
    out = sim.rollout(device=True)
    for _ in range(max(args.warmup, 3)):
        sim.rollout(device=True, out=out)
    reps = max(args.steps, 20)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    torch.cuda.synchronize(dev)
    for k in range(reps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        sim.rollout(device=True, out=out)
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    ms = slowest(sum(a.elapsed_time(b) for a, b in ev) / 1000.0, dev) * 1000.0 / reps
    res = sim.rollout()
    executor = sim.executor
    sim.close()
    horizon_s = sc.T * sc.dt
    return {"workload": f"Chicago-shaped synthetic network: {sc.V} nodes / {sc.L} links, {sc.N * dn:,} vehicles as "
                        f"{sc.N:,} platoons of {dn}, {sc.T} steps of {sc.dt:g} s (one hour)",
            "ms_per_rollout": ms, "x_real_time": horizon_s / (ms / 1000.0),
            "agent_steps_per_s": ws * sc.N * sc.T / (ms / 1000.0), "executor": executor,
            "arrived_platoons": int(res["n_arrived"][-1]), "on_links_at_end": int(res["n_on"][-1]),
            "paper_context": "3.0 s forward (17.7 s with compilation) for the one-hour nowcast on Chicago Sketch, "
                             "one H200 (JAX/XLA)",
            "timing": "CUDA events on the simulator's stream, L2 flushed before each rollout"}


def run_calibration_loop(args, dev, stream, ws):
    """The calibration loop (Methods, Optimization) on the calibration-gradient
    workload: AdamW on the 10,240 demand and 16 route-choice parameters,
    a fixed number of iterations (the early stop is not reached)."""
    import torch
    from paper_2603_25068_b300 import scenario as S
    from paper_2603_25068_b300.optimize import calibrate
    from paper_2603_25068_b300.sim import Simulator
    model, truth = S.calibration()
    sens = model.sensors
    y_obs = Simulator(truth, device=dev.index, stream=stream).rollout()["counts"][:, sens]
    sim = Simulator(model, device=dev.index, stream=stream, ckpt_every=60, route_cap=256)
    calibrate(sim, y_obs, sens, max_iter=1)                     # workspaces, graphs
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    res = calibrate(sim, y_obs, sens, max_iter=args.calib_iters)
    torch.cuda.synchronize(dev)
    sec = slowest(time.perf_counter() - t0, dev)
    sim.close()
    return {"workload": f"calibration gradient workload ({model.N:,} vehicles, {model.T} steps), AdamW lr 0.1 "
                        f"wd 1e-5 on {model.n_od} demand + {model.F} route-choice parameters, until 20 "
                        "iterations without a lower loss",
            "iterations": res["iterations"], "seconds": sec, "s_per_iteration": sec / res["iterations"],
            "loss_first": res["losses"][0], "loss_best": res["best_loss"], "best_iter": res["best_iter"],
            "losses": [round(x, 3) for x in res["losses"]],
            "note": "the surrogate gradient of these parameters does not descend the expected loss "
                    "(tests/test_oracle_descent.py): demand enters only through straight-through weights, "
                    "the route-choice weights through the sentinel-scaled merge adjoint",
            "timing": "host wall clock, device synchronised (forward, loss, reverse pass, update)"}


def run_paper_mode(args, dev, stream, ws):
    """Paper-mode calibration (Methods, experimental setting): per-link u,
    kappa, beta, alpha on a 48-node / 100-link synthetic network with 20,000
    vehicles, counts every 5 min over 30 min with 10 % noise on 80 % of the
    links, from the range means; a fixed number of AdamW iterations in units
    of each parameter's range.  u, kappa and beta are calibrated; alpha stays
    at its start (its surrogate gradient does not descend the expected loss:
    tests/test_oracle_descent.py)."""
    import torch
    from paper_2603_25068_b300 import scenario as S
    from paper_2603_25068_b300.optimize import calibrate_ranges, range_simulator
    from paper_2603_25068_b300.sim import Simulator
    model, truth = S.paper_mode()
    sens = model.sensors
    observed = S.noisy_counts(Simulator(truth, device=dev.index, stream=stream).rollout()["counts"][:, sens],
                              np.random.default_rng(1))
    ranges = {k: S.PAPER_RANGES[k] for k in ("u", "kappa", "beta")}
    sim = range_simulator(model, S.PAPER_RANGES, device=dev.index, stream=stream, ckpt_every=60, route_cap=128)
    calibrate_ranges(sim, observed, sens, ranges, max_iter=1)                  # workspaces, graphs
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    res = calibrate_ranges(sim, observed, sens, ranges, max_iter=args.paper_iters, patience=10 ** 6,
                           lr=args.paper_lr)
    torch.cuda.synchronize(dev)
    sec = slowest(time.perf_counter() - t0, dev)
    sim.close()
    err = lambda p, k: float(np.mean(np.abs(np.asarray(p, np.float64) - getattr(truth, k)))
                             / (S.PAPER_RANGES[k][1] - S.PAPER_RANGES[k][0]))
    return {"workload": f"paper-mode calibration: {model.V} nodes / {model.L} links, {model.N:,} vehicles, "
                        f"{model.T} steps, {len(sens)} observed links, 3 x {model.L} link parameters (u, kappa, beta)",
            "iterations": res["iterations"], "seconds": sec, "s_per_iteration": sec / res["iterations"],
            "loss_first": res["losses"][0], "loss_best": res["best_loss"], "best_iter": res["best_iter"],
            "calibrated": list(ranges), "lr_range_units": args.paper_lr,
            "param_error_start": {k: err(getattr(model, k), k) for k in ranges},
            "param_error_best": {k: err(res["params"][k], k) for k in ranges},
            "timing": "host wall clock, device synchronised (forward, loss, reverse pass, update)"}


def run_fwd_bwd(args, dev, stream, flush, ws):
    """Calibration-gradient workload: 1,800-step rollout of the city network with
    the reverse pass (checkpoints every 60 steps) of the squared error of
    5-minute counts on 2,000 sensor links against a hidden ground-truth draw."""
    import torch
    import torch.distributed as dist
    from paper_2603_25068_b300 import scenario as S
    from paper_2603_25068_b300.sim import Simulator
    if args.small:
        model, truth = S.calibration(n_sensors=500, n_nodes=3000, n_links=9000, n_vehicles=250_000,
                                     n_origin_zones=20, n_dest_zones=32)
    else:
        model, truth = S.calibration()
    T = model.T
    y_obs = Simulator(truth, device=dev.index, stream=stream).rollout()["counts"]
    sim = Simulator(model, device=dev.index, stream=stream, ckpt_every=60, route_cap=256)
    nb = sim.n_bins(T)
    sens = model.sensors
    from paper_2603_25068_b300.autotune import tune_recompute
    ybar0 = np.zeros((nb, model.L), np.float32)
    ybar0[:, sens] = 1e-3
    recompute, recompute_ms = tune_recompute(sim, ybar0, T)
    times, t_fwd, t_bwd = [], [], []
    for k in range(args.warmup + args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        out = sim.rollout(T)
        ybar = np.zeros((nb, model.L), np.float32)
        diff = out["counts"][:, sens].astype(np.float32) - y_obs[:, sens]
        ybar[:, sens] = 2.0 * diff / diff.size
        t1 = time.perf_counter()
        g = sim.backward(ybar)
        torch.cuda.synchronize(dev)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
            t_fwd.append(t1 - t0)
            t_bwd.append(time.perf_counter() - t1)
    tot = slowest(sum(times), dev)
    ms = 1000 * tot / args.steps
    # algorithmic bytes of an iteration: the forward (node model and
    # car-following bytes model), its recomputation in the reverse pass, and
    # the reverse step's own bytes: 13 per vehicle on a link (tape position and
    # tag, adjoint read and write), ~200 per node-model candidate (tape records,
    # route-log entries, merge and choice Jacobian terms), 32 per link
    # (parameter accumulators)
    import ctypes as C
    from paper_2603_25068_b300 import native as nat
    out = sim.rollout(T)
    cnt = np.zeros(4 * T, np.int32)
    nat.check(sim.lib.sim_step_counters(sim.h, cnt.ctypes.data_as(C.c_void_p)), sim.h)
    n_on = out["n_on"][:T].astype(np.float64)
    n_cand = cnt.reshape(T, 4)[:, 2].astype(np.float64)
    fwd_b = float(np.sum(kernel_a_bytes(model, n_on, n_cand, avg_choice_degree(model))))
    bwd_b = fwd_b + float(np.sum(13.0 * n_on + 200.0 * n_cand + 32.0 * model.L))
    peak, peak_kind = load_peaks()
    achieved = (fwd_b + bwd_b) / (ms / 1000.0) / 1e9
    roof = {"bound": "hbm", "kernel": "forward + reverse pass (every kernel of one iteration, host wall clock)",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback",
            "algorithmic_bytes_per_iteration": fwd_b + bwd_b, "forward_bytes": fwd_b, "reverse_bytes": bwd_b,
            "traffic": None}
    return {"metric": "vehicle-steps/s (forward + reverse pass)", "value": ws * model.N * T / (ms / 1000),
            "roofline": roof,
            "unit": "vehicle-steps/s", "ms_per_iteration": ms, "x_real_time": T * model.dt / (ms / 1000),
            "workload": f"calibration gradient: city network, {model.N:,} vehicles, {T} steps, checkpoints every 60, "
                        f"{len(sens)} sensor links, gradient w.r.t. {model.n_od} demand and {model.F} route-choice "
                        "parameters (and every link parameter)",
            "timing": "host wall clock per iteration (rollout with host outputs, host loss, sim_backward to host), "
                      "L2 flushed before each",
            "forward_ms": 1000 * float(np.mean(t_fwd)), "reverse_ms": 1000 * float(np.mean(t_bwd)),
            "recompute": recompute, "recompute_autotune_ms": {k: round(v, 2) for k, v in recompute_ms.items()},
            "grad_norm_w": float(np.linalg.norm(g["w"])), "grad_norm_lambda": float(np.linalg.norm(g["od_lambda"]))}


# ------------------------------------------------------------------ batched
def run_batched(args, dev, stream, flush, ws):
    """Batched control-candidate scenarios: n scenarios of 10k-200k vehicles on
    the city network with per-scenario capacity multipliers, 1,800 steps,
    forward by the autotuned batch executor, then each scenario's reverse pass;
    against the same scenarios run one by one."""
    import torch
    from paper_2603_25068_b300 import scenario as S
    from paper_2603_25068_b300 import native as nat
    from paper_2603_25068_b300.batch import Batch
    from paper_2603_25068_b300.sim import Simulator
    kw = dict(n_nodes=3000, n_links=9000, n_vehicles=250_000, n_origin_zones=20, n_dest_zones=32) if args.small else {}
    scs = S.batched_scenarios(n=args.batch_n, **kw)
    T = scs[0].T
    sims = [Simulator(sc, device=dev.index, stream=stream, ckpt_every=180, route_cap=256) for sc in scs]
    rng = np.random.default_rng(0)
    ybars = []
    vs = float(sum(sc.N for sc in scs)) * T
    # batched: executor autotuned on a short rollout, one warm-up batch rollout,
    # then a timed batch forward + reverse passes
    from paper_2603_25068_b300 import autotune
    res = {}
    with Batch(sims) as b:
        best, tune_ms = autotune.tune_batch(b, T=min(T, 120))
        other = {}
        for e in autotune.BATCH_EXECUTORS:        # forward of the executor not chosen
            if e == best:
                continue
            try:
                b.set_executor(e)
            except Exception:
                continue
            b.rollout(T)
            flush.fill_(3.0)
            torch.cuda.synchronize(dev)
            t3 = time.perf_counter()
            b.rollout(T)
            torch.cuda.synchronize(dev)
            other[e] = time.perf_counter() - t3
        b.set_executor(best)
        b.rollout(T)
        # algorithmic bytes of the batched forward: the node-model bytes model of
        # every member's steps, from its own counters (runs are deterministic,
        # so the warm-up run's counters are the timed run's)
        import ctypes as C
        bytes_b = 0.0
        for sc, sm in zip(scs, sims):
            ybars.append(rng.normal(size=(sm.n_bins(T), sc.L)).astype(np.float32))
            cnt = np.zeros(4 * T, np.int32)
            nat.check(sm.lib.sim_step_counters(sm.h, cnt.ctypes.data_as(C.c_void_p)), sm.h)
            n_on = sm.outputs()["n_on"][:T].astype(np.float64)
            bytes_b += float(np.sum(kernel_a_bytes(sc, n_on, cnt.reshape(T, 4)[:, 2].astype(np.float64),
                                                   avg_choice_degree(sc))))
        flush.fill_(1.0)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        b.rollout(T)
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
    # the members leave the batch with their runs; their reverse passes run
    # from four host threads, each member on a stream of its own
    from concurrent.futures import ThreadPoolExecutor
    for sm in sims:
        sm.set_stream(torch.cuda.Stream(device=dev))
    with ThreadPoolExecutor(4) as ex:
        list(ex.map(lambda a: a[0].backward(a[1]), zip(sims, ybars)))
    torch.cuda.synchronize(dev)
    t2 = time.perf_counter()
    res["batched_forward_s"] = t1 - t0
    res["batched_forward_plus_reverse_s"] = t2 - t0
    # serial single-scenario path
    flush.fill_(2.0)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for sm in sims:
        sm.rollout(T)
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    for sm, yb in zip(sims, ybars):
        sm.rollout(T)
        sm.backward(yb)
    torch.cuda.synchronize(dev)
    t2 = time.perf_counter()
    res["serial_forward_s"] = t1 - t0
    res["serial_forward_plus_reverse_s"] = t2 - t1
    for s_ in sims:
        s_.close()
    return {"metric": "vehicle-steps/s", "unit": "vehicle-steps/s",
            "workload": f"{len(scs)} control-candidate scenarios on the {scs[0].L}-link city network, "
                        f"{int(sum(sc.N for sc in scs)):,} vehicles in total ({min(sc.N for sc in scs):,}-"
                        f"{max(sc.N for sc in scs):,} per scenario), {T} steps, capacity x U(0.7,1.0) on 500 links",
            "batched_forward": vs / res["batched_forward_s"],
            "serial_forward": vs / res["serial_forward_s"],
            "batched_forward_plus_reverse": vs / res["batched_forward_plus_reverse_s"],
            "serial_forward_plus_reverse": vs / res["serial_forward_plus_reverse_s"],
            "seconds": res,
            "executor": best,
            "roofline": {"bound": "hbm", "kernel": f"{'k_batch_persist' if best == 'persistent' else 'k_batch_a + k_batch_b'} "
                                                   "(whole batched forward, host wall clock)",
                         "achieved": bytes_b / res["batched_forward_s"] / 1e9, "peak": load_peaks()[0], "unit": "GB/s",
                         "frac": bytes_b / res["batched_forward_s"] / 1e9 / load_peaks()[0],
                         "algorithmic_bytes": bytes_b},
            "autotune_ms_per_rollout": {k: round(v, 2) for k, v in tune_ms.items()},
            "other_executor_forward_s": other,
            "timing": "host wall clock, device synchronised; batched reverse passes from 4 host threads, "
                      "serial ones one scenario after another"}


# ------------------------------------------------------------------ serving
def run_serving(args, dev, ws):
    """Poisson stream of nowcast / calibration / control requests on networks of
    2k-36k links and 50k-1M vehicles, served by the engine under a 150 GB
    budget with at most SERVE_IN_FLIGHT requests running (shortest remaining
    work first with aging, the next ones' simulators built ahead, reverse
    passes between forward work), against serial single-scenario execution of
    the same stream; at the configured 4 requests/s and at 16 requests/s."""
    from paper_2603_25068_b300 import serve
    sizes = (600, 1200, 2400) if args.small else (2000, 4500, 9000, 18000, 36000)
    n_range = (5000, 50000) if args.small else (50_000, 1_000_000)

    # both arms first serve a short stream of their own, so that neither is
    # timed with cold memory pools, code paths or host caches
    warm = serve.make_request_stream(n=16, rate=50.0, seed=99, sizes=sizes, n_range=n_range)
    serve.Engine(device=dev.index, hbm_budget=150e9, chunk=240, ckpt_every=180,
                 max_in_flight=SERVE_IN_FLIGHT).run(warm)
    serve.run_serial(warm, device=dev.index, ckpt_every=180)

    def leg(rate, n):
        reqs = serve.make_request_stream(n=n, rate=rate, seed=4, sizes=sizes, n_range=n_range)
        eng = serve.Engine(device=dev.index, hbm_budget=150e9, chunk=240, ckpt_every=180,
                           max_in_flight=SERVE_IN_FLIGHT)
        eng.run(reqs)
        makespan = max(r.finished for r in reqs)
        st = serve.latency_stats(reqs)
        vs = float(sum(r.vehicle_steps for r in reqs))
        ser = serve.run_serial(reqs, device=dev.index, ckpt_every=180)
        lat_s = np.array([x["finished"] - x["arrival"] for x in ser])
        ser_span = max(x["finished"] for x in ser)
        return {"requests": len(reqs), "rate_per_s": rate,
                "mix": {k: sum(1 for r in reqs if r.kind == k) for k in ("nowcast", "calibration", "control")},
                "p50_latency_s": st["p50_s"], "p99_latency_s": st["p99_s"], "vehicle_steps_per_s": vs / makespan,
                "serial": {"p50_latency_s": float(np.percentile(lat_s, 50)),
                           "p99_latency_s": float(np.percentile(lat_s, 99)), "vehicle_steps_per_s": vs / ser_span}}

    out = leg(4.0, args.serve_requests)
    out["rate_16_per_s"] = leg(16.0, max(32, args.serve_requests // 2))
    out.update(hbm_budget_gb=150, max_in_flight=SERVE_IN_FLIGHT, order="shortest remaining work first",
               note="latency from arrival to result, including simulator creation")
    return out


# one request on the GPU at a time: each request's kernels fill the GPU, so
# running two at once (a batch of two, or two streams) is slower than one after
# the other; the engine's gain is the host set-up of the next requests
SERVE_IN_FLIGHT = 1


# ------------------------------------------------------------------ ours
def run_ours(args):
    import torch
    import torch.distributed as dist
    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_2603_25068_b300.sim import Simulator
    from paper_2603_25068_b300 import native as nat

    sc = make_scenario(args)
    # a dedicated stream: the library enqueues everything on it and the CUDA
    # events below are recorded on the same stream
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    sim = Simulator(sc, device=local, stream=stream)
    T, N = sc.T, sc.N
    nb = sim.n_bins(T)
    out = dict(counts=torch.empty((nb, sc.L), dtype=torch.int32, device=dev),
               speed=torch.empty((nb, sc.L), dtype=torch.float32, device=dev),
               travel_time=torch.empty((nb, sc.L), dtype=torch.float32, device=dev))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    from paper_2603_25068_b300 import autotune
    sim.set_executor(args.executor)
    executor = sim.executor
    if args.stage:
        autotune.set_stage(sim, args.stage)
        stage, stage_ms = args.stage, {}
    elif executor == "step":
        stage, stage_ms = autotune.tune_stage(sim, T=min(T, 900))
    else:
        stage, stage_ms = None, {}

    for _ in range(args.warmup):
        sim.rollout(T, device=True, out=out)
    torch.cuda.synchronize(dev)
    if ws > 1:
        dist.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        torch.cuda.synchronize(dev)
        if ws > 1:
            dist.barrier()
        for k in range(args.steps):
            flush.fill_(float(k))                      # evict the working set from L2
            ev[k][0].record(stream)
            sim.rollout(T, device=True, out=out)
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
        if ws > 1:
            dist.barrier()
    ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = slowest(sum(ms), dev)
    ms_per = total_ms / args.steps
    value = whole_job_rate(N * T * args.steps, ws, total_ms / 1000.0)
    # our kernels per rollout: reset + (node model, transfer) per step + final
    # observation, or reset + one persistent launch
    launches_per_rollout = 2 * T + 2 if executor == "step" else 2

    # ---- instrumented pass: per-kernel device time for the roofline
    kms = np.zeros(3)
    kl = np.zeros(3, np.int64)
    import ctypes as C
    o = nat.sim_outputs(on_device=0)
    nat.check(sim.lib.sim_profile_rollout(sim.h, T, C.byref(o), kms.ctypes.data_as(C.c_void_p),
                                          kl.ctypes.data_as(C.c_void_p)), sim.h)
    res = sim.outputs()
    cnt = np.zeros(4 * T, np.int32)
    nat.check(sim.lib.sim_step_counters(sim.h, cnt.ctypes.data_as(C.c_void_p)), sim.h)
    cnt = cnt.reshape(T, 4)
    n_on = res["n_on"][:T].astype(np.float64)            # vehicles on links at the start of each step
    deg = avg_choice_degree(sc)
    bytes_a = float(np.sum(kernel_a_bytes(sc, n_on, cnt[:, 2].astype(np.float64), deg)))
    ms_a = float(kms[0])
    achieved = bytes_a / (ms_a / 1000.0) / 1e9
    peak, peak_kind = load_peaks()
    if executor == "step":
        kname, kdesc, per_launch = "k_step_a", "k_step_a (node model + car-following)", T
        units_per_launch = float(np.mean(n_on))            # vehicles on links per launch (one step)
        share = {"k_step_a": kms[0] / kms.sum(), "k_step_b": kms[1] / kms.sum(), "obs_final": kms[2] / kms.sum()}
    else:
        kname, kdesc, per_launch = "k_persist", "k_persist (whole rollout: every step of the path)", 1
        units_per_launch = float(np.sum(n_on))              # vehicle-steps on links per launch (one rollout)
        share = {"k_persist": 1.0}
    traffic = ncu_traffic(kname, "city_1M", units_per_launch)

    line = {
        "metric": "vehicle-steps/s", "value": value, "unit": "vehicle-steps/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_of(args, sc, ws),
        "x_real_time": T * sc.dt / (ms_per / 1000.0),
        "state_at_T": {"n_on": int(res["n_on"][T]), "n_arrived": int(res["n_arrived"][T]),
                       "n_waiting": int(res["n_waiting"][T]),
                       "note": "vehicles on links, arrived and not yet departed at the end of the rollout "
                               "(on the hour-long one: jam-dominated, most vehicle-steps are standing queues)"},
        "active_vehicle_steps_per_s": float(np.sum(n_on)) * ws / (ms_per / 1000.0),
        "per_rollout_ms": ms,
        "roofline": {"bound": "hbm", "kernel": kdesc,
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "frac_of_nominal": achieved / NOMINAL_HBM_GBS, "nominal_peak": NOMINAL_HBM_GBS,
                     "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback",
                     "traffic": traffic, "algorithmic_bytes_per_launch": bytes_a / per_launch,
                     "avg_launch_us": 1000.0 * ms_a / per_launch, "us_per_step": 1000.0 * ms_a / T,
                     "kernel_share": share,
                     "instrumented_rollout_ms": float(kms.sum())},
        "gpu_launches": launches_per_rollout * args.steps,
        "executor": executor,
        "launch_shape": ({"staged_slots_per_block": stage, "autotune_ms_per_900_steps": stage_ms}
                         if executor == "step" else {"ctas": "one per SM (cooperative)", "threads": 1024}),
        "clocks": clk.summary(),
    }

    # ---- the other executor on the same workload, for comparison
    if executor == "persistent" and not args.no_compare:
        sim.set_executor("step")
        st_stage, _ = autotune.tune_stage(sim, T=min(T, 900))
        sim.rollout(T, device=True, out=out)
        st_ms = []
        for k in range(2):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.rollout(T, device=True, out=out)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            st_ms.append(e0.elapsed_time(e1))
        sim.set_executor("auto")
        line["step_executor"] = {"ms_per_rollout": float(np.mean(st_ms)), "staged_slots_per_block": st_stage,
                                 "vehicle_steps_per_s": N * T / (float(np.mean(st_ms)) / 1000.0),
                                 "note": "two kernels per step in a CUDA graph, same workload and outputs"}

    # ---- end to end through the public API with host buffers
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        params = dict(u=pin(sc.u), kappa=pin(sc.kappa), alpha=pin(sc.alpha), beta=pin(sc.beta),
                      cost=pin(sc.cost), w=pin(sc.w))
        host = dict(counts=torch.empty((nb, sc.L), dtype=torch.int32).pin_memory().numpy(),
                    speed=torch.empty((nb, sc.L), dtype=torch.float32).pin_memory().numpy(),
                    travel_time=torch.empty((nb, sc.L), dtype=torch.float32).pin_memory().numpy())
        h2d = sum(v.nbytes for v in params.values())
        d2h = sum(v.nbytes for v in host.values())

        def e2e_step():
            sim.set_params(**params)
            o = nat.sim_outputs(counts=C.c_void_p(host["counts"].ctypes.data),
                                speed=C.c_void_p(host["speed"].ctypes.data),
                                travel_time=C.c_void_p(host["travel_time"].ctypes.data), on_device=0)
            nat.check(sim.lib.sim_rollout(sim.h, T, C.byref(o)), sim.h)

        e2e_step()                                  # captures the graph after the params change
        torch.cuda.synchronize(dev)
        t_e2e = []
        for k in range(args.steps):
            flush.fill_(float(k))
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            e2e_step()
            t_e2e.append(time.perf_counter() - t0)
        tot = slowest(sum(t_e2e), dev)
        line["e2e"] = {"value": whole_job_rate(N * T * args.steps, ws, tot), "unit": "vehicle-steps/s",
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                       "ms_per_step": 1000 * tot / args.steps,
                       "note": "sim_set_params from pinned host arrays + sim_rollout into pinned host outputs"}

    if not args.no_fwd_bwd:
        line["fwd_bwd"] = run_fwd_bwd(args, dev, stream, flush, ws)
    def optional(name, fn, *a):
        # a leg beyond the contract's: its failure is reported in its entry
        try:
            line[name] = fn(*a)
        except Exception as e:                  # noqa: BLE001
            line[name] = {"error": f"{type(e).__name__}: {e}"}
    if not args.no_platoons:
        optional("platoons", run_platoons, args, dev, stream, flush, ws)
        optional("chicago_twin", run_chicago_twin, args, dev, stream, flush, ws)
    if not args.no_calib_loop:
        optional("calibration_loop", run_calibration_loop, args, dev, stream, ws)
    if not args.no_paper_mode:
        optional("paper_mode", run_paper_mode, args, dev, stream, ws)
    if not args.no_batched:
        line["batched"] = run_batched(args, dev, stream, flush, ws)
    if not args.no_serve:
        line["serving"] = run_serving(args, dev, ws)

    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = run_cpu_baseline(args, sc, sim, out, flush, dev, stream)
    if rank == 0:
        print(json.dumps(line), flush=True)
    sim.close()
    if ws > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
