"""bench.py's multi-rank path (replicas only: each rank runs its own lattice,
no data-path collective) on the CPU with the gloo backend, world size 2:
the barrier and the maximum of the per-rank times that set the reported
whole-job value."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench

    class A:
        impl = "reference"  # gloo

    w, r, _ = bench.dist_setup(A())
    bench.barrier(w)
    v = bench.max_over_ranks(w, 1.0 + r * 2.5)
    cells = 1000
    value = w * cells * 10 / (v / 1e3) / 1e6  # as run_ours: all ranks' cells / max time
    out[r] = (w, v, value)
    dist.destroy_process_group()


def test_replicas_max_time_over_two_ranks():
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert out[0][0] == 2 and out[1][0] == 2
    assert out[0][1] == out[1][1] == 3.5  # max of 1.0 and 3.5 ms
    assert abs(out[0][2] - 2 * 1000 * 10 / 3.5e-3 / 1e6) < 1e-9


def test_reference_arm_under_torchrun_prints_once():
    """bench.py --impl reference launched as the contract launches N > 1
    (torchrun, two ranks, 127.0.0.1): rank 0 alone times the oracle and prints
    one JSON line; the other rank exits 0 without work."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2", "--L", "64", "--steps", "1",
           "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
