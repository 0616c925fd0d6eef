"""The N > 1 path of bench.py on CPU: two gloo ranks (127.0.0.1) with different
timed regions must both see the slower one, the whole-job rate counts every
rank's units over that time (weak scaling: replicas on different pairs, no
data-path collective), and the batched configurations give every rank its own
block of generator pairs."""
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


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        mine = 100.0 + 50.0 * rank  # rank 1 is the slow one
        slowest = bench.max_over_ranks(mine, world, device="cpu")
        ids = bench.rank_pair_ids(2, rank)
        q.put((rank, slowest, bench.job_rate(10, world, slowest), ids[0], ids[-1], len(ids)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_split_the_pairs():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, v0, a0, b0, n0), (r1, s1, v1, a1, b1, n1) = out
    assert s0 == s1 == 150.0
    assert v0 == v1 == pytest.approx(2 * 10 / 0.150)
    assert (a0, b0, n0) == (0, 255, 256) and (a1, b1, n1) == (256, 511, 256)
