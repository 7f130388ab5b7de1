"""The N > 1 path of bench.py on CPU with the gloo backend (world size 2): each
rank runs an independent replica of the workload (its own seed, no data-path
collective), the step time is the slowest rank's, and the job's throughput is
the units of all ranks over that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ns = type("A", (), {"M": 4096, "intervals": 20})()
    wl = bench.workload(ns, rank)
    ms_local = 100.0 + 50.0 * rank               # rank 1 is the slower one
    ms = bench.max_over_ranks(ms_local, "cpu")
    units = bench.node_samples_per_interval(wl, 0)
    out.put((rank, wl.seed, ms, units, bench.job_throughput(units, world, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_max_time_and_job_throughput():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (r0, s0, ms0, u0, v0), (r1, s1, ms1, u1, v1) = res
    assert (r0, r1) == (0, 1)
    assert s0 != s1                      # independent replicas: different random streams
    assert u0 == u1                      # the same work per rank (weak scaling)
    assert ms0 == ms1 == 150.0           # both ranks report the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * u0 / 0.150)
