"""The N > 1 path on CPU: world-size-2 gloo ranks run the rank logic bench.py uses on GPUs —
process-group start from the torchrun environment, distinct replica seeds, the round-robin
deal of independent films (disjoint, complete), the barrier and the max / sum over ranks of the
timing."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    from paper_1205_5588_gb300 import distributed as D
    r = D.init("gloo")
    films = D.shard(11, r.rank, r.world)
    seed = D.replica_seed(7, r.rank)
    D.barrier(r)
    t_max = D.max_over_ranks(1.0 + r.rank, r)
    att = D.sum_over_ranks(100 * (r.rank + 1), r)
    out.put((r.rank, r.world, films, seed, t_max, att, r.is_root))
    D.finish(r)


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(k, world, port, q)) for k in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ranks = [r[0] for r in res]
    assert ranks == [0, 1] and all(r[1] == world for r in res)
    dealt = sorted(i for r in res for i in r[2])
    assert dealt == list(range(11))                                  # every film once
    assert set(res[0][2]).isdisjoint(res[1][2])
    assert res[0][3] == 7 and res[1][3] != res[0][3]                 # rank 0 keeps the base seed
    assert all(r[4] == 2.0 for r in res)                             # max over ranks
    assert all(r[5] == 300.0 for r in res)                           # sum over ranks
    assert [r[6] for r in res] == [True, False]


def test_single_process_defaults(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    from paper_1205_5588_gb300 import distributed as D
    r = D.init("gloo")
    assert (r.rank, r.world, r.is_root) == (0, 1, True)
    assert D.max_over_ranks(3.5, r) == 3.5 and D.shard(4, 0, 1) == [0, 1, 2, 3]
