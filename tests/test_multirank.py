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
