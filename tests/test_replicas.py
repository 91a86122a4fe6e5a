"""The multi-GPU path (replicas only), on CPU with the gloo backend: each rank
runs its own replica; the timed duration is the slowest rank's (a MAX
reduction); the whole-job rate counts every rank's units; under torchrun only
rank 0 prints the bench line (the reference arm's other ranks exit without
work)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, values, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2603_25068_b300 import replicas
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    replicas.barrier()
    got = replicas.slowest(values[rank])
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(repr(got))
    dist.destroy_process_group()


def test_slowest_rank_time_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    values = [3.25, 7.5]
    mp.start_processes(_rank_main, args=(2, _free_port(), values, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    for r in range(2):
        assert float(open(tmp_path / f"r{r}.txt").read()) == max(values)


def test_whole_job_rate_counts_every_rank():
    sys.path.insert(0, ROOT)
    from paper_2603_25068_b300 import replicas
    assert replicas.whole_job_rate(1.0e9, 4, 2.0) == 2.0e9
    assert replicas.slowest(1.5) == 1.5            # no process group: the value itself


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
           "--small"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    res = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, res.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    # the same workload description as the GPU arm's line, and the window it times
    assert line["config"]["step"].startswith("one ") and line["config"]["vehicles"] == 250_000
    assert "steps 0-299" in line["cpu_baseline"]["sample"]
    assert 0 < line["cpu_baseline"]["active_value"] < line["value"]
