"""Multi-process host logic on CPU (gloo, world size 2): the batched path shards over
processes with no data-path collective.  Every rank computes the same
longest-processing-time split from the shapes alone, plans its own share, and the
ranks only agree on the split and gather timings (max over ranks), as bench.py
does for N > 1."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads as wl


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import paper_2012_00706_gb300 as gid
        shapes = wl.config4_shapes(512, 4)
        dims = [(m, n) for m, n, _ in shapes]
        ranks = [r for _, _, r in shapes]
        rank_of, work = gid.shard_batch(dims, ranks, world)
        mine = [i for i, r in enumerate(rank_of) if r == rank]
        # each rank plans its own share on the host (no GPU needed for planning)
        plan = gid.BatchPlan([dims[i] for i in mine], [ranks[i] for i in mine], precision="mixed_bf16x3",
                             device="cpu")
        j_total = plan.j_off[-1]
        # the only exchanges: the split (to check agreement) and per-rank numbers
        splits = [None] * world
        dist.all_gather_object(splits, rank_of)
        t = torch.tensor([float(rank + 1)], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot = torch.tensor([len(mine), j_total], dtype=torch.int64)
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
        q.put((rank, splits, work, float(t.item()), tot.tolist(), len(mine)))
    finally:
        dist.destroy_process_group()


def test_batch_shard_gloo_world2():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    shapes = wl.config4_shapes(512, 4)
    # every rank computed the same split
    assert out[0][1][0] == out[0][1][1] == out[1][1][0]
    rank_of = out[0][1][0]
    assert set(rank_of) == {0, 1}
    # the shares partition the batch
    assert sum(o[5] for o in out) == len(shapes)
    assert out[0][4] == [len(shapes), sum(n for _, n, _ in shapes)]
    # max over ranks, as the bench takes it
    assert out[0][3] == out[1][3] == 2.0
    # longest-processing-time balance: the spread is below the largest single matrix
    work = out[0][2]
    biggest = max(2.0 * min(r + 10, m) * m * n for m, n, r in shapes)
    assert abs(work[0] - work[1]) <= biggest


@pytest.mark.parametrize("world", [1, 3, 8])
def test_batch_shard_partition(world):
    import paper_2012_00706_gb300 as gid
    shapes = wl.config4_shapes(200, 7)
    rank_of, work = gid.shard_batch([(m, n) for m, n, _ in shapes], [r for _, _, r in shapes], world)
    assert len(rank_of) == len(shapes) and min(rank_of) >= 0 and max(rank_of) < world
    assert len(work) == world
    if world > 1:
        biggest = max(2.0 * min(r + 10, m) * m * n for m, n, r in shapes)
        assert max(work) - min(work) <= 2 * biggest
