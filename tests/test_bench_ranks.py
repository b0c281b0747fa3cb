"""The benchmark's multi-rank bookkeeping on CPU (gloo, world size 2): the
job time is the slowest rank's, all ranks' cells count, and the reference
arm prints from rank 0 only.  No GPU is involved."""
import importlib.util
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _rank_main(rank, world, port, local_ms, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        value, max_ms = b.job_throughput(local_ms[rank], 1000, 4, world)
        out.put((rank, value, max_ms))
    finally:
        dist.destroy_process_group()


def test_job_throughput_single_rank():
    b = _bench()
    value, max_ms = b.job_throughput(2000.0, 1_000_000, 10, 1)
    assert max_ms == 2000.0
    assert value == pytest.approx(1_000_000 * 10 / 2.0)


def test_job_throughput_two_gloo_ranks_take_the_slowest():
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    local_ms = [300.0, 500.0]
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, local_ms, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, max_ms in res:
        assert max_ms == 500.0                       # the slowest rank's time on every rank
        assert value == pytest.approx(1000 * 2 * 4 / 0.5)   # both ranks' cells


def test_reference_arm_prints_only_on_rank_zero():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
