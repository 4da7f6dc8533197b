"""The bench's multi-rank host logic on CPU with the gloo backend (world size
2): each rank works on its own image, the job time is the slowest rank's, and
the value counts every rank's pixels (weak scaling, no collective on the data
path)."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import synth
    # per-rank work: the image of this rank's seed
    img = synth.rects_noise(64, 96, rank)
    my_ms = 10.0 * (rank + 1)           # rank 1 is the slow one
    slowest = bench.max_over_ranks(my_ms, world, device="cpu")
    value = bench.weak_scaling_value(img.size, 5, world, slowest)
    dist.barrier()
    out.put((rank, slowest, value, int(img.sum())))
    dist.destroy_process_group()


def test_two_rank_weak_scaling_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, v0, sum0), (r1, s1, v1, sum1) = res
    assert s0 == s1 == 20.0                       # max over ranks
    assert v0 == v1 == pytest.approx(2 * 64 * 96 * 5 / 20e-3 / 1e9)
    assert sum0 != sum1                           # each rank had its own image
