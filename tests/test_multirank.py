"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): every rank
runs its own solve (replicas) and the job's step time is the maximum over
ranks, taken after a barrier, as bench.py does on GPUs with NCCL."""
import importlib.util
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod",
                                                  os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench = _bench()
        dist.barrier()
        t = bench.job_seconds(0.25 + rank, dist, "cpu")
        dist.barrier()
        out.put((rank, t))
    finally:
        dist.destroy_process_group()


def test_job_time_is_max_over_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 1.25), (1, 1.25)]


def test_job_time_single_rank_is_local():
    assert _bench().job_seconds(0.5) == 0.5
