"""Multi-process (world_size 2, gloo, CPU) checks of the row sharding and the measurement
reductions used by bench.py under torchrun (not gpu)."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

from paper_2105_13611_gb300.sharding import reduce_scalar, rows_for_rank


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rows = rows_for_rank(1425, rank, world)
    t = 1.5 + rank          # per-rank elapsed time
    ev = 1000 * (rank + 1)  # per-rank evaluation count
    q.put((rank, rows.tolist(), reduce_scalar(t, "max"), reduce_scalar(ev, "sum")))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_disjoint_rows_and_reductions():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    rows = {r: set(x) for r, x, _, _ in res}
    assert rows[0].isdisjoint(rows[1])
    assert rows[0] | rows[1] == set(range(1425))
    assert abs(len(rows[0]) - len(rows[1])) <= 1
    for _, _, tmax, evsum in res:
        assert tmax == 2.5 and evsum == 3000


def test_single_process_identity():
    assert reduce_scalar(3.0, "max") == 3.0
    assert np.array_equal(rows_for_rank(5, 0, 1), np.arange(5))


def test_bench_rows_per_rank_are_disjoint_and_same_mix():
    # bench.py's rows under torchrun come from rows_for_rank: disjoint across ranks, rank 0
    # keeps the single-GPU rows, and every rank takes one row of each cost class (a
    # temperature neighbour of the same pressure)
    import bench
    for world in (1, 2, 4, 8):
        per = [bench.batch_points(r, 8, world) for r in range(world)]
        flat = np.concatenate(per)
        assert len(set(flat.tolist())) == len(flat) and np.all((flat >= 0) & (flat < 1425))
        assert np.array_equal(per[0], bench.TABLE_ROWS)
        for rows in per:
            assert np.array_equal(rows % 25, np.array(bench.TABLE_ROWS) % 25)
            assert np.all(np.abs(rows // 25 - np.array(bench.TABLE_ROWS) // 25) < world)
