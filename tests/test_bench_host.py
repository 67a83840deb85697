"""bench.py's host-side pieces, without a GPU: the closure each workload runs
with, and the CPU oracle's bounded sample of every workload (the reference
arm), one step at reduced sizes."""
import argparse
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def args(workload, stat="fd"):
    return argparse.Namespace(workload=workload, stat=stat, L=512, cells1d=1 << 14, tau=0.8, steps=1, warmup=0,
                              prec="f32", inv="exact", engine="tensor")


@pytest.mark.parametrize("workload,stat,want", [
    ("smooth_t", "fd", "fd"), ("batched", "fd", "fd"), ("d1v3", "fd", "t0"), ("porous", "fd", "mb"),
    ("d1v3", "mb", "mb"), ("porous", "t0", "t0"),
])
def test_settle_closure(workload, stat, want):
    a = args(workload, stat)
    bench.settle_closure(a)
    assert a.stat == want


@pytest.mark.parametrize("workload", ["smooth_t", "batched", "d1v3", "porous"])
def test_oracle_sample_takes_a_finite_step(workload):
    a = args(workload)
    bench.settle_closure(a)
    jobs, what = bench.oracle_jobs(a, 2)
    assert len(jobs) == 2 and what
    for job in jobs:
        f = job["f0"]
        g = bench._oracle_step(job)(f)
        assert g.shape == f.shape and np.isfinite(g).all()
        # one collision conserves the mass of the sample (periodic wrap)
        assert abs(g.sum() - f.sum()) < 1e-12 * abs(f.sum())


def test_oracle_worker_restarts_windows_and_counts_timed_steps():
    """The pool worker times only steps (warm-up and restarts untimed) and
    restarts every window_steps steps, so 20 steps of a 15-step window run
    from two fresh starts, and both windows end in a finite state."""
    a = args("smooth_t")
    jobs, _ = bench.oracle_jobs(a, 1)
    job = dict(jobs[0], steps=20, warmup=1, window_steps=15)
    updates, secs, steps, bad = bench._oracle_window_worker(job)
    assert steps == 20 and updates == 20 * job["f0"][0].size and secs > 0
    assert bad == 0


@pytest.mark.parametrize("workload", ["smooth_t", "batched", "d1v3", "porous"])
def test_workload_config_carries_the_contract_keys(workload):
    """Every workload's config names the workload, states how L2 is handled
    between steps, and the parallelism."""
    from paper_1510_07328_gb300 import inputs

    a = args(workload)
    bench.settle_closure(a)
    probs = inputs.batched(count=4) if workload == "batched" else None
    cfg = bench.workload_config(a, 1, probs)
    assert cfg["workload"].startswith(workload.split("_")[0])
    assert "L2" in cfg["l2"] and cfg["parallelism"] == "single GPU"
    assert bench.workload_config(a, 2, probs)["parallelism"] == "replicas x2"


def test_source_hash_ignores_comments_only():
    """The kernel source hash behind profiles/traffic.json sees what the
    compiler sees: comments and blank lines do not change it, code does, and
    comment markers inside string literals (inline PTX) are kept."""
    base = 'asm("ld.global.f32 %0, [%1]; // not a comment");\nint a = 1;\n'
    assert bench.strip_comments(base) == bench.strip_comments("/* header */\n" + base + "// trailing note\n\n")
    assert bench.strip_comments(base) != bench.strip_comments(base.replace("a = 1", "a = 2"))
    assert "// not a comment" in bench.strip_comments(base)
    assert bench.strip_comments("x = y / z; /* a */ w = 1;") == "x = y / z;   w = 1;"
