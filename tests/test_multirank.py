"""The multi-GPU path of bench.py on CPU ranks (gloo, world size 2): each rank
decodes a batch of its own (weak scaling, no collective on the data path), the
device time is the maximum over ranks and the work is their sum."""
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


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        insts, ps = bench.workload("batch128", rank, count=2)
        t, steps = bench.combine_ranks([10.0 + rank, 100.0 * (rank + 1)], "cpu", ["max", "sum"])
        out[rank] = (t, steps, [p.seed for p in ps], [i.n for i in insts],
                     [float(i.coords.sum()) for i in insts])
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_instances_and_combine_timing():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        r0, r1 = out[0], out[1]
    assert r0[0] == r1[0] == 11.0                   # slowest rank's device time
    assert r0[1] == r1[1] == 300.0                  # work of both ranks
    assert r0[2] == [1000, 1001] and r1[2] == [101000, 101001]   # disjoint instance seeds
    assert r0[4] != r1[4]                           # so the ranks decode different instances
    import bench
    from paper_2601_19041_gb300 import synth
    insts, ps = synth.workload("batch128", count=2)
    assert [p.seed for p in ps] == r0[2] and [i.n for i in insts] == r0[3]   # rank 0 = the 1-GPU batch


def test_combine_without_a_group_is_identity():
    import bench
    assert bench.combine_ranks([3.5, 7.0], "cpu", ["max", "sum"]) == [3.5, 7.0]


def _decode_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import dataclasses

        import bench
        from oracle import oracle as orc
        insts, ps = bench.workload("batch128", rank, count=1)
        p = dataclasses.replace(ps[0], m=8, iterations=2)
        o = orc.Oracle(insts[0], p).iterate(2)
        mine = (p.seed, float(o.scalars()["L_gb"]))
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)      # host-side gather of (seed, L_gb) per rank
        out[rank] = gathered
    finally:
        dist.destroy_process_group()


def test_each_rank_decodes_its_own_shard():
    """Two gloo ranks each decode their own instance (the CPU oracle stands in
    for the GPU decode here); the gathered results equal decoding the same
    instances in one process, so the shards are independent."""
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_decode_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        g0, g1 = list(out[0]), list(out[1])
    assert g0 == g1
    import dataclasses

    import bench
    from oracle import oracle as orc
    for rank, (seed, L) in enumerate(g0):
        insts, ps = bench.workload("batch128", rank, count=1)
        assert ps[0].seed == seed
        p = dataclasses.replace(ps[0], m=8, iterations=2)
        assert orc.Oracle(insts[0], p).iterate(2).scalars()["L_gb"] == L
