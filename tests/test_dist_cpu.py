"""The N > 1 path of the benchmark on CPU: replicas only (independent
requests, no exchange on the data path), so the multi-rank logic is the
max-over-ranks time, the whole-job value and rank 0 alone reporting.  Two
gloo ranks on 127.0.0.1; no GPU."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _ranks(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    tdist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ms = [120.0, 135.5][rank]          # each rank's own timed region
        tdist.barrier()
        m = bench.rank_max(tdist, ms)
        out[rank] = (bench.dist_env(), m, bench.replica_value(10, ws, m))
    finally:
        tdist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    port = 29500 + os.getpid() % 1000
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        procs = [ctx.Process(target=_ranks, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(2):
        env, m, v = res[r]
        assert env == (2, r, r)
        assert m == 135.5
        assert abs(v - 20 / 0.1355) < 1e-9  # 2 ranks x 10 solves over the slowest rank


def test_no_process_group_is_the_rank_itself():
    assert bench.rank_max(None, 7.5) == 7.5
    assert bench.replica_value(4, 1, 500.0) == 8.0


def test_reference_arm_on_a_non_zero_rank_exits_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True,
                       timeout=300, cwd=ROOT)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_gpus_flag_spawns_local_ranks_or_refuses(monkeypatch):
    """`bench.py --gpus N` without a torchrun environment starts N local ranks
    through torch.distributed.run on 127.0.0.1 (one per GPU, the same
    arguments), and refuses when fewer GPUs are visible."""
    calls = []
    monkeypatch.setattr(bench.subprocess, "call", lambda cmd: calls.append(cmd) or 0)
    monkeypatch.setattr(torch.cuda, "device_count", lambda: 4)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--gpus", "2", "--steps", "3"])
    assert bench.spawn_local_ranks(2) == 0
    cmd = calls[0]
    assert cmd[1:4] == ["-m", "torch.distributed.run", "--nnodes=1"]
    assert cmd[cmd.index("--nproc-per-node") + 1] == "2"
    assert cmd[cmd.index("--master-addr") + 1] == "127.0.0.1"
    assert cmd[-4:] == ["--gpus", "2", "--steps", "3"]
    monkeypatch.setattr(torch.cuda, "device_count", lambda: 1)
    assert bench.spawn_local_ranks(2) == 2 and len(calls) == 1
