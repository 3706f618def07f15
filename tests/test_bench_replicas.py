"""bench.py's multi-GPU path on CPU: two gloo ranks stand in for two GPU replicas.

The aggregation / disaggregation of one problem needs no exchange between GPUs, so
`bench.py --gpus N` runs N independent replicas; what crosses ranks is only the
timing: the job takes as long as its slowest rank, and its ms per matvec is that
time over steps x ranks.
"""
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


def _rank_main(rank, world, port, totals, steps, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, loc = bench.dist_env()
        assert (w, r, loc) == (world, rank, rank)
        total, value = bench.whole_job_ms(totals[rank], steps, world, device="cpu")
        out[rank] = (total, value)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("totals", [(120.0, 100.0), (80.0, 95.5)])
def test_replicas_report_the_slowest_rank(totals):
    world, steps = 2, 10
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, totals, steps, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    slow = max(totals)
    for r in range(world):
        assert res[r] == (slow, slow / (steps * world))


def test_single_replica_needs_no_process_group():
    import bench
    assert bench.whole_job_ms(42.0, 7, 1) == (42.0, 6.0)
