"""The node-sharded iteration's host logic on CPU with two gloo ranks: each
rank computes eps for its share of the pairs (here with the oracle, which needs
no GPU), the zero-filled buffers are summed by the all-reduce of
paper_2608_22190_b300.sharded, and the result equals the unsharded eps bit for
bit.  The GPU side (spmc_iterate_shard / spmc_apply_eps) is tested against
spmc_iterate in test_gpu_parity.py."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def test_shard_ranges_partition_the_pairs():
    from paper_2608_22190_b300.sharded import shard_range
    for n in (1, 7, 30, 8640, 10 ** 6 + 3):
        for world in (1, 2, 3, 8):
            got = [shard_range(n, r, world) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
            assert max(h - l for l, h in got) - min(h - l for l, h in got) <= 1
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def _problem():
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    from oracle import oracle as O
    O.build()
    spec = O.Spec(dim=1, n_space=6, time_family=0, M=96, n_ref=12, f_coef=(0, 0, 0, -1.0), ex_kind=O.EX_SIN,
                  ex_beta=1.0, n_threads=1)
    Mt, h = 5, 0.5
    pts = O.space_nodes_grid(spec)
    U = np.tile(np.sin(np.pi * pts[:, 0]), (Mt + 1, 1))
    cu, ct = O.reconstruct(spec, Mt, h, U)
    return O, spec, Mt, h, cu, ct


def _eps_of_pairs(lo, hi):
    O, spec, Mt, h, cu, ct = _problem()
    S = spec.n_space
    out = np.zeros(Mt * S)
    for i in range(lo, hi):
        ti, j = divmod(i, S)
        out[i] = O.node_eps(spec, Mt, 0.0, h, cu, ct, j, ti + 1, interval=0, iteration=1)
    return out


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2608_22190_b300.sharded import assemble, shard_range
    n = 5 * 6
    lo, hi = shard_range(n, rank, world)
    eps = torch.from_numpy(_eps_of_pairs(lo, hi))
    assemble(eps)
    q.put((rank, eps.numpy().copy()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharded_eps_equals_unsharded():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    full = _eps_of_pairs(0, 30)
    assert np.array_equal(res[0], full) and np.array_equal(res[1], full)
