"""The multi-process path of bench.py on the CPU: world_size-2 `gloo` ranks
agree on the job's time (the maximum over ranks) and on the whole-job rate,
and the reference arm prints only on rank 0."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout
from types import SimpleNamespace

import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(1.0 + rank, dist, "cpu")
        out[rank] = (t, bench.whole_job_rate(1e9, world, 5, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time_and_rate():
    world = 2
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world,
                           start_method="spawn", join=True)
        res = dict(out)
    assert res[0] == res[1] == (2.0, world * 1e9 * 5 / 2.0)


def test_single_process_is_its_own_job():
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.whole_job_rate(4.0, 1, 2, 8.0) == 1.0


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(SimpleNamespace(cpu_stride=0, warmup=0, steps=1))
    assert buf.getvalue() == ""
