"""Multi-process host logic on CPU (gloo, world size 2): units are dealt to
ranks exactly once, timings combine as the maximum over ranks, and a single
system split by element rows (each rank advancing its rows, positions and
velocities all-gathered once per step) reproduces the one-process FP64
reference trajectory bitwise."""
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


def test_row_range_covers_every_row_once():
    from paper_2303_12166_gb300.dist import row_range
    for n in (0, 1, 5, 61, 1024):
        for world in (1, 2, 3, 8):
            spans = [row_range(n, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[r][1] == spans[r + 1][0] for r in range(world - 1))
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        row_range(5, 2, 2)


# a 61-element binary (ragged split over 2 or 3 ranks) with contacts and
# donor growth, 6 steps
ROWS_IC = dict(n_donor=40, n_accretor=21, q=0.5, f_donor=0.9, f_accretor=0.6, sigma_v=1e-2,
               seed=5)
ROWS_P = dict(G=1.0, eps=0.01, beta=0.4, dt=2e-3)
ROWS_GROW = dict(f0=0.9, rate=2e-3, cap=4)
ROWS_STEPS = 6


def _rows_worker(rank, world, port, out):
    import numpy as np
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as orc
    from paper_2303_12166_gb300.dist import row_range
    x, v, m, R0, gam = orc.make_ic(**ROWS_IC)
    n, nd = x.shape[0], ROWS_IC["n_donor"]
    lo, hi = row_range(n, world, rank)
    rows = np.arange(lo, hi)
    dt = ROWS_P["dt"]

    def radii(k):
        s = orc.donor_scale(k, ROWS_GROW["f0"], ROWS_GROW["rate"], ROWS_GROW["cap"])
        return np.where(np.arange(n) < nd, R0 * s, R0)

    def acc(k):
        return orc.forces_rows(rows, x, v, m, radii(k), gam, G=ROWS_P["G"], eps=ROWS_P["eps"],
                               beta=ROWS_P["beta"])

    def gather(a):
        parts = [None] * world
        dist.all_gather_object(parts, a[lo:hi].copy())
        return np.concatenate(parts)

    a = acc(0)
    for k in range(ROWS_STEPS):
        v[lo:hi] += 0.5 * dt * a
        x[lo:hi] += dt * v[lo:hi]
        x, v = gather(x), gather(v)  # the one exchange of the step
        a = acc(k + 1)
        v[lo:hi] += 0.5 * dt * a
    out.put((rank, gather(x), gather(v)))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_row_split_system_matches_one_process(orc, world):
    import numpy as np
    import torch.multiprocessing as mp
    x, v, m, R0, gam = orc.make_ic(**ROWS_IC)
    rx, rv, _ = orc.run(x, v, m, R0, gam, nsteps=ROWS_STEPS, n_donor=ROWS_IC["n_donor"],
                        grow_f0=ROWS_GROW["f0"], grow_rate=ROWS_GROW["rate"],
                        grow_cap=ROWS_GROW["cap"], **ROWS_P)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rows_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gx, gv in res:
        assert np.array_equal(gx, rx), f"rank {rank}: positions differ"
        assert np.array_equal(gv, rv), f"rank {rank}: velocities differ"
