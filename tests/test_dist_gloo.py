"""Multi-process host logic on CPU (gloo, world size 2): units are dealt to
ranks exactly once, and timings combine as the maximum over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2303_12166_gb300.dist import max_over_ranks, shard, sum_over_ranks
    mine = shard(257, world, rank)
    # every rank reports its own timing; the combined value is the maximum
    t = max_over_ranks(1.0 + rank)
    total = sum_over_ranks(len(mine))
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    out.put((rank, t, total, gathered))
    dist.destroy_process_group()


def test_shard_and_reduce_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, total, gathered in res:
        assert t == 2.0
        assert total == 257
        units = sorted(u for g in gathered for u in g)
        assert units == list(range(257))


def test_shard_single_process():
    from paper_2303_12166_gb300.dist import max_over_ranks, shard
    assert shard(5, 1, 0) == [0, 1, 2, 3, 4]
    assert shard(5, 2, 1) == [1, 3]
    assert max_over_ranks(3.5) == 3.5
    with pytest.raises(ValueError):
        shard(5, 2, 2)


def test_workload_recipes():
    import synth
    sw = synth.sweep_systems(256, seed=0)
    ns = [s["n_donor"] + s["n_accretor"] for s in sw]
    assert len(sw) == 256 and min(ns) >= 2048 and max(ns) <= 65536
    assert all(0.1 <= s["q"] <= 1.0 for s in sw)
    tr = synth.served_trace(64, seed=0, steps_div=100)
    ts = [r["t_arrival"] for r in tr]
    assert ts == sorted(ts) and ts[0] == 0.0
    assert all(10 <= r["nsteps"] <= 200 for r in tr)
    # mean arrival gap close to 1/20 s
    assert 0.03 < (ts[-1] / (len(ts) - 1)) < 0.08
