"""The multi-rank host logic of bench.py on CPU: world size 2 over gloo.  Each rank runs
its own ensemble (no collective on the data path); the only collectives are the barrier
around the timed region and the max over ranks of the elapsed time."""
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist()
    try:
        d.barrier()
        ms = d.max(10.0 + 5.0 * rank)  # the slower rank decides the job's time
        seeds = bench.rank_seeds([{"seed": 13}, {"seed": 14}], d.rank)
        q.put((d.rank, d.world, ms, seeds, bench.aggregate(1000, 20, d.world, ms)))
    finally:
        d.close()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, ms0, s0, v0), (r1, w1, ms1, s1, v1) = out
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert ms0 == ms1 == 15.0
    assert v0 == v1 == pytest.approx(2 * 1000 * 20 / 0.015)
    assert s0 == [13, 14] and len(set(s0) | set(s1)) == 4   # no shared Philox key
