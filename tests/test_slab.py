"""Row-slab decomposition of one film, host side (no GPU): the slab partition, the neighbour
map, the whole-film series from slab traces, the host fold of a series into step records
(checked against the oracle's own records of the same chain), and the halo exchange between
world-size 2 and 3 gloo ranks on host buffers (the code path NCCL takes between GPUs)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp

from paper_1205_5588_gb300 import slab as S
from paper_1205_5588_gb300 import workloads as W


@pytest.mark.parametrize("rows,world", [(2, 1), (9, 1), (10, 2), (11, 2), (17, 3), (64, 5), (6, 3), (256, 8)])
def test_slab_bounds_partition(rows, world):
    b = S.slab_bounds(rows, world)
    assert len(b) == world and b[0][0] == 0 and b[-1][1] == rows
    for (y0, y1), (z0, _) in zip(b, b[1:]):
        assert y1 == z0
    for y0, y1 in b:
        assert y0 % 2 == 0 and y1 - y0 >= 2
        assert y1 % 2 == 0 or y1 == rows
    sizes = [y1 - y0 for y0, y1 in b[:-1]]
    assert max(sizes, default=2) - min(sizes, default=2) <= 2            # even split


@pytest.mark.parametrize("rows,world", [(3, 2), (4, 3), (1, 1), (10, 0)])
def test_slab_bounds_refuses(rows, world):
    with pytest.raises(ValueError):
        S.slab_bounds(rows, world)


def test_neighbours():
    assert S.neighbours(0, 1, False) == (None, None)
    assert S.neighbours(0, 1, True) == (0, 0)
    assert S.neighbours(0, 3, False) == (None, 1)
    assert S.neighbours(2, 3, False) == (1, None)
    assert S.neighbours(0, 3, True) == (2, 1)
    assert S.neighbours(2, 3, True) == (1, 0)
    assert S.neighbours(1, 2, True) == (0, 0)


def test_whole_film_series():
    t1 = np.array([[1, -2], [3, 4]], dtype=np.int64)
    t2 = np.array([[-5, 6], [0, 1]], dtype=np.int64)
    M, B, n = S.whole_film_series([t1, t2], [(10, 7, 3), (-4, 9, 5)])
    assert M.tolist() == [10 - 4 + 1 - 5, 10 - 4 + 3 + 0]
    assert B.tolist() == [8 - 2 + 6, 8 + 4 + 1] and n == 8
    with pytest.raises(ValueError):
        S.whole_film_series([t1], [(0, 3, 1)])                          # odd total 2B


def _lib_or_skip():
    try:
        from paper_1205_5588_gb300 import isingfilm as I
    except ImportError as e:          # the library is built by build(); no GPU is needed here
        pytest.skip(f"library not built: {e}")
    return I


@pytest.mark.parametrize("case", ["flat_periodic", "fractal_gate_free"])
def test_fold_series_equals_oracle_records(olib, case):
    """isf_fold_series on the oracle's own per-sweep series gives the oracle's step records: the
    exact sums bit for bit, the derived averages to the last bit (same FP64 formulas)."""
    I = _lib_or_skip()
    from oracle import oracle
    if case == "flat_periodic":
        H, L, flags = np.full((8, 8), 3, dtype=np.uint8), 3, 3
        sched = W.schedule([2.0, 5.0, 3.5], [0.5, 0.0, -1.0], [2, 0, 1], [5, 7, 3])
    else:
        H, L, flags = W.fractal_heights(12, 18, 0.7, 1, 4, seed=3), 4, 0
        sched = W.schedule(np.linspace(1.0, 9.0, 5), 0.3, 1, 4)
    f = oracle.Film(H, L, flags=flags, seed=9, lib=olib)
    n_occ = f.info()["n_occ"]
    recs, ser = f.run(sched["T"], sched["h"], sched["eq"], sched["meas"], series=True)
    got = I.fold_series(sched["T"], sched["h"], sched["eq"], sched["meas"], n_occ, ser[:, 0], ser[:, 1])
    assert len(got) == len(recs)
    for g, w in zip(got, recs):
        for k in ("M_last", "B_last", "n_meas", "sumM", "sumAbsM", "sumB", "sumM2", "sumB2", "sumMB"):
            assert g[k] == w[k], (k, g[k], w[k])
        for k in ("m", "abs_m", "e", "chi", "chi_abs", "C"):
            assert g[k] == pytest.approx(w[k], rel=1e-12, abs=1e-300), k


class FakeSlab:
    """Host stand-in for a slab film: colour-rows [colour][row] of `width` bytes, own rows
    filled with (rank, colour, row) codes, halo rows zero."""

    def __init__(self, rank, nrows, width=6):
        self.rank, self.nrows, self.width = rank, nrows, width
        self.rows = np.zeros((4, nrows + 2, width), dtype=np.int16)
        for c in range(4):
            for j in range(1, nrows + 1):
                self.rows[c, j] = 1000 * (rank + 1) + 100 * c + j

    def empty_rows(self):
        return torch.zeros(self.width, dtype=torch.int16)

    def export_rows(self, colour, side):
        j = 1 if side == S.LOW else self.nrows
        return torch.from_numpy(self.rows[colour, j].copy())

    def import_rows(self, colour, side, t):
        j = 0 if side == S.LOW else self.nrows + 1
        self.rows[colour, j] = t.numpy()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _exchange_rank(rank, world, port, periodic, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    from paper_1205_5588_gb300 import distributed as D
    r = D.init("gloo")
    fake = FakeSlab(rank, nrows=3 + rank)
    ex = S.DistExchange(fake, r.rank, r.world, periodic)
    for c in (2, 0, 3):                 # only the colour just updated moves
        ex(c)
    out.put((rank, fake.rows.tolist()))
    D.finish(r)


@pytest.mark.parametrize("world,periodic", [(2, False), (2, True), (3, False), (3, True)])
def test_halo_exchange_over_gloo(world, periodic):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_exchange_rank, args=(k, world, port, periodic, q)) for k in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    nrows = {r: 3 + r for r in range(world)}
    for r in range(world):
        rows = np.array(res[r])
        lo, hi = S.neighbours(r, world, periodic)
        for c in range(4):
            moved = c in (2, 0, 3)
            want_lo = 1000 * (lo + 1) + 100 * c + nrows[lo] if (lo is not None and moved) else 0
            want_hi = 1000 * (hi + 1) + 100 * c + 1 if (hi is not None and moved) else 0
            assert (rows[c, 0] == want_lo).all(), (r, c, rows[c, 0])
            assert (rows[c, nrows[r] + 1] == want_hi).all(), (r, c, rows[c, -1])
            for j in range(1, nrows[r] + 1):                            # own rows untouched
                assert (rows[c, j] == 1000 * (r + 1) + 100 * c + j).all()


def test_local_exchange_single_rank_periodic():
    a = FakeSlab(0, nrows=4)
    S.LocalExchange([a], periodic_y=True)(1)
    assert (a.rows[1, 0] == 1000 + 100 + 4).all() and (a.rows[1, 5] == 1000 + 100 + 1).all()
    assert (a.rows[0, 0] == 0).all()
