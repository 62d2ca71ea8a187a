"""The host logic of an N-GPU run -- process group, barrier, max of the timed
interval, whole-job rate -- checked with two gloo ranks on the CPU, and the
reference arm's rule that only rank 0 reports.  (The data-parallel step itself:
tests/test_dp.py.)"""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    from paper_2207_11620_gb300 import replicas
    w, r, _ = replicas.setup(backend="gloo")
    replicas.barrier(w)
    t = 10.0 + 5.0 * r  # the ranks' timed intervals differ
    m = replicas.max_over_ranks(w, t)
    rate = replicas.job_throughput(w, 1000.0, m)
    replicas.barrier(w)
    replicas.teardown(w)
    q.put((r, w, m, rate))


def test_two_gloo_replicas_agree_on_the_slowest_rank():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(ws))
    assert [o[0] for o in out] == [0, 1]
    for r, w, m, rate in out:
        assert w == 2 and m == 15.0           # the slowest rank's interval on every rank
        assert rate == pytest.approx(2 * 1000.0 / 15.0)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    from paper_2207_11620_gb300 import replicas
    assert replicas.max_over_ranks(1, 3.5) == 3.5
    assert replicas.job_throughput(1, 10.0, 2.0) == 5.0


def test_reference_arm_reports_on_rank_zero_only():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, cwd=ROOT, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
