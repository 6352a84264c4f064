"""The multi-process path of bench.py on CPU: world size 2 over gloo (the
GPU runs use NCCL the same way).  The benchmark runs one independent
replica per rank (no collective on the data path); the job's time is the
maximum over ranks after a barrier, and the whole-job rate counts the units
of every rank."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    assert bench.dist_env() == (ws, rank, rank)
    dist.barrier()
    t = bench.job_time(times[rank], dist, torch.device("cpu"))
    out[rank] = t
    dist.barrier()
    dist.destroy_process_group()


def test_job_time_is_the_slowest_rank_and_the_rate_counts_every_rank():
    ws, port = 2, _free_port()
    times = [0.25, 0.4]
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(ws, port, times, out), nprocs=ws, join=True)
    assert out[0] == out[1] == max(times)
    assert bench.job_rate(10.0, ws, max(times)) == pytest.approx(2 * 10.0 / 0.4)


def test_single_process_is_unchanged():
    assert bench.job_time(0.3, None, None) == 0.3
    assert bench.job_rate(1.0, 1, 0.5) == 2.0


def test_reference_arm_under_torchrun_prints_one_line():
    """`bench.py --impl reference` launched the way a multi-GPU run launches it for
    N = 2 (torchrun, two ranks, gloo): rank 0 alone runs the oracle and prints
    one JSON line, the other rank exits 0 without work."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1"]
    p = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, p.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
