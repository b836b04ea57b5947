"""The benchmark's multi-rank logic on CPU (world size 2, gloo): every rank
times its own replica of the batch, the reported time is the slowest rank's,
and the whole-job rate counts the units of all ranks.  Independent solves
exchange nothing, so this host logic is the whole of the N > 1 path."""
from __future__ import annotations

import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [120.0, 250.0][rank]          # rank 1 is the slow one
        ms = bench.max_over_ranks(local_ms, "cpu")
        rate = bench.whole_job_rate(3, world, ms / 1e3)
        dist.barrier()
        q.put((rank, ms, rate))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, rate in got:
        assert ms == 250.0                       # the slowest rank's time on every rank
        assert rate == pytest.approx(3 * 2 / 0.25)   # 6 solves in 0.25 s


def test_single_process_is_its_own_maximum():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.5, "cpu") == 42.5
    assert bench.whole_job_rate(3, 1, 0.5) == pytest.approx(6.0)


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the other ranks of the reference arm exit 0 at once and
    print nothing."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_config_matches_gpu_arm():
    """Both arms describe the workload with the same config object."""
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    wl = W.workload_medium()
    c = bench.workload_config(wl, 1, wl.K, len(wl.ics))
    assert c["workload"] == wl.name and c["K"] == wl.K and c["solves_per_step"] == 3
    assert {"grid", "N_slices", "krylov_cap", "n_f", "n_g", "ics", "fine_prec", "l2", "parallelism"} <= set(c)
