"""The multi-process host logic (independent problems per rank, max-over-ranks timing) with two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, items, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    from paper_1602_05700_gb300 import multi

    multi.init("gloo")
    r, w, lr = multi.env_ranks()
    mine = multi.shard(items, r, w)
    multi.barrier()
    t = multi.max_over_ranks(10.0 + r)
    out.put((r, w, lr, mine, t))
    multi.finalize()


def test_two_gloo_ranks_share_problems_and_report_the_slowest():
    world, port = 2, _free_port()
    items = list(range(7))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, items, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = sorted(x for _, _, _, mine, _ in res for x in mine)
    assert got == items  # every independent problem exactly once
    assert all(t == 11.0 for *_, t in res)  # the max over ranks
    assert [r[:3] for r in res] == [(0, 2, 0), (1, 2, 1)]
