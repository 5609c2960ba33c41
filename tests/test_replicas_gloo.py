"""Replica bookkeeping of bench.py on 2 CPU ranks (gloo): each rank draws its
own batch, the job's time is the maximum over ranks and its work the sum, so
`value` is whole-job throughput under weak scaling.  No GPU, no collective on
the data path: the only exchange is these two scalars."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    from paper_2310_05037_gb300 import synth as S

    w_, r, _ = bench.dist_init(0)
    try:
        assert (w_, r) == (world, rank)

        class A:
            workload = "batched"
            reads = 40

        w = bench.make_workload(S, A, rank)
        cells = float(w.read_lengths().sum())
        t = 1.0 + rank  # rank 1 is the slow one
        bench.barrier(world)
        out[rank] = (bench.max_over_ranks(t, world), bench.sum_over_ranks(cells, world), cells,
                     float(w.events[:4].sum()))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_rank_replicas():
    world = 2
    port = 29500 + (os.getpid() % 2000)
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    tmax = [res[r][0] for r in range(world)]
    total = [res[r][1] for r in range(world)]
    assert tmax == [2.0, 2.0]
    assert total[0] == total[1] == res[0][2] + res[1][2]
    # each replica draws its own batch
    assert res[0][3] != res[1][3]
