"""The N > 1 path of bench.py on CPU: two gloo ranks (one process each, as
torchrun launches them) agree on the max-over-ranks time and on the whole-job
rate, which counts every rank's batch (replicas, weak scaling)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    local = 1.0 + 0.5 * rank  # rank r's timed region took 1 + r/2 s
    t = bench.max_over_ranks(local, dist)
    out[rank] = (t, bench.job_rate(10_000 * 20, world, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for r in (0, 1):
        t, rate = res[r]
        assert t == pytest.approx(1.5)  # the slower rank's time on every rank
        assert rate == pytest.approx(2 * 10_000 * 20 / 1.5)  # both ranks' queries over that time


def test_single_process_is_unchanged():
    sys.path.insert(0, ROOT)
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    assert bench.max_over_ranks(2.5, None) == 2.5
    assert bench.job_rate(1000, 1, 0.5) == 2000.0
