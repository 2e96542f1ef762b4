"""The multi-GPU path of bench.py is replicas (one index per GPU, no data
collective): its host logic -- the job time as the maximum over ranks and the
distinct query batch each rank answers -- checked with two gloo ranks on the
CPU."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        b = _bench()
        t = b.max_over_ranks(1.0 + rank, ws)          # rank 1 is the slower one
        batches = [b.rank_batch(i, rank, 10) for i in range(3)]
        out.put((rank, t, batches))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slower_rank_and_distinct_batches():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    got = dict()
    for _ in range(ws):
        rank, t, batches = q.get(timeout=120)
        got[rank] = (t, batches)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got[0][0] == got[1][0] == 2.0
    assert got[0][1] == [0, 1, 2] and got[1][1] == [1, 2, 3]


def test_single_process_is_its_own_job():
    b = _bench()
    assert b.max_over_ranks(3.5, 1) == 3.5
    assert [b.rank_batch(i, 0, 4) for i in range(6)] == [0, 1, 2, 3, 0, 1]
