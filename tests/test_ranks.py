"""The several-rank path of the benchmark (replicas only: independent frames, timing combined
with a max over ranks), run as two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [3.0, 5.0][rank]
    t_max = bench.max_over_ranks(local_ms, dist, "cpu")
    value = bench.whole_job_mdisp(10, world, 1280, 720, 128, t_max)
    q.put((rank, t_max, value, bench.rank_seed(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
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
    (r0, t0, v0, s0), (r1, t1, v1, s1) = out
    assert t0 == t1 == 5.0                       # the slowest rank bounds the job
    assert v0 == v1 == pytest.approx(10 * 2 * 1280 * 720 * 128 / 5e-3 / 1e6)
    assert s0 != s1                              # every rank processes its own frame


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(4.0, None, "cpu") == 4.0
    assert bench.whole_job_mdisp(2, 1, 100, 10, 32, 1.0) == pytest.approx(2 * 100 * 10 * 32 / 1e-3 / 1e6)
