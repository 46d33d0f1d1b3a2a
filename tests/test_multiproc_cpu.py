"""The multi-rank host logic of bench.py on CPU with the gloo backend (the
hot path does not shard: N GPUs run N replicas, the job time is the slowest
rank's, rank 0 reports), and the reference arm under torchrun."""
import json
import multiprocessing as mp
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


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    t_max = bench.max_over_ranks(10.0 + 5.0 * rank, world)
    q.put((rank, t_max, bench.job_rate(1000, world, t_max)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]          # both ranks see the slowest rank's time
    assert all(abs(o[2] - 2 * 1000 / 0.015) < 1e-6 for o in out)  # whole-job rate over both replicas


def test_max_over_ranks_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_rate(100, 1, 1000.0) == 100.0


def test_reference_arm_under_torchrun_two_ranks():
    """Rank 0 alone times the oracle and prints one JSON line; rank 1 exits 0."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--grid", "32", "--steps", "1", "--warmup", "1", "--gpus", "2"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_pass_bytes_match_the_per_node_figures():
    """The roofline's algorithmic bytes per launch: 97 / 24 / 27 / 49 B per node
    for the forward row (or plane), x2, last-axis and inverse row (or plane)
    passes of the FP32 CG iteration (d = 3), plus 44 B per boundary node in the
    inverse pass."""
    import bench
    N = 128 ** 3
    assert bench.pass_bytes("rows_fwd", N, 0) == 97 * N
    assert bench.pass_bytes("cols_x2", N, 0) == 24 * N
    assert bench.pass_bytes("last_axis", N, 0) == 27 * N
    assert bench.pass_bytes("rows_inv", N, 1000) == 49 * N + 44 * 1000
    # the plane passes move the bytes of the row passes they replace (their x2
    # transform stays in shared memory)
    assert bench.pass_bytes("plane_fwd", N, 0) == bench.pass_bytes("rows_fwd", N, 0)
    assert bench.pass_bytes("plane_inv", N, 1000) == bench.pass_bytes("rows_inv", N, 1000)
