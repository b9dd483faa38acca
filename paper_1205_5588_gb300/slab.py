"""Row-slab decomposition of one film over several GPUs.

Sec. 3 splits the film between processes by rows of the image: each process updates its own
rows and, between updates, exchanges the rows next to its neighbours' slabs.  Here a rank holds
whole-film rows [y0, y1) as a slab film (isf_lattice_create_slab) with one halo row pair on each
side.  A sweep is four colour passes (Sec. 3's checkerboard, four colours for z = 12); after
pass c every rank sends its two boundary colour-rows of colour c (all layers) to its neighbours,
which copy them into their halos, before anyone starts pass c + 1.  The slabs carry the whole
film's Philox counters, so the decomposed run is the whole film's trajectory, bit for bit.

Observables: each slab's trace holds the change of its own M and B after every sweep; the whole
film's series is the sum over ranks (an int64 all-reduce) plus the sum of the slabs' creation
shares, and isf_fold_series turns it into the step records.

The exchange is written against two operations, `export_rows(colour, side)` -> tensor and
`import_rows(colour, side, tensor)`, so the same code moves halos between GPUs over NCCL
(DistExchange), between slabs in one process (LocalExchange), or between host buffers over gloo.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

LOW, HIGH = 0, 1


def slab_bounds(rows: int, world: int) -> list[tuple[int, int]]:
    """Rows [y0, y1) of each rank: contiguous, y0 even (the colour of a site depends on the
    parity of y), at least two rows each, the last slab ending at `rows`."""
    pairs = rows // 2
    if world < 1 or pairs < world:
        raise ValueError(f"{rows} rows cannot be split into {world} slabs of at least two rows")
    base, extra = divmod(pairs, world)
    out, y = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        y1 = y + 2 * n
        out.append((y, rows if r == world - 1 else y1))
        y = y1
    return out


def neighbours(rank: int, world: int, periodic_y: bool) -> tuple[int | None, int | None]:
    """Ranks holding the rows just below (low y) and just above (high y) this rank's slab; None
    at an open edge of the film.  A periodic film wraps (a single rank is its own neighbour)."""
    lo = rank - 1 if rank > 0 else (world - 1 if periodic_y else None)
    hi = rank + 1 if rank < world - 1 else (0 if periodic_y else None)
    return lo, hi


class LocalExchange:
    """Halo exchange between slab films held by one process (one device): after colour pass c
    each slab's boundary rows are copied into its neighbours' halos."""

    def __init__(self, slabs, periodic_y: bool):
        self.slabs = list(slabs)
        self.periodic_y = periodic_y

    def __call__(self, colour: int):
        world = len(self.slabs)
        out = [(s.export_rows(colour, LOW), s.export_rows(colour, HIGH)) for s in self.slabs]
        for r, s in enumerate(self.slabs):
            lo, hi = neighbours(r, world, self.periodic_y)
            if lo is not None:
                s.import_rows(colour, LOW, out[lo][HIGH])
            if hi is not None:
                s.import_rows(colour, HIGH, out[hi][LOW])


class DistExchange:
    """Halo exchange between ranks of a torch.distributed process group (NCCL on GPUs, gloo on
    host buffers): every rank sends its low boundary rows to the rank below and its high ones to
    the rank above, and receives the matching halos.  The order of the point-to-point operations
    is the same on every rank, so with two ranks on a periodic film (both neighbours are the
    same rank) the two messages still land in the right halos."""

    def __init__(self, slab, rank: int, world: int, periodic_y: bool):
        self.slab, self.rank, self.world = slab, rank, world
        self.lo, self.hi = neighbours(rank, world, periodic_y)

    def __call__(self, colour: int):
        import torch.distributed as dist
        s = self.slab
        if self.world == 1:
            if self.lo is not None:         # periodic film on one rank: its own rows wrap
                low, high = s.export_rows(colour, LOW), s.export_rows(colour, HIGH)
                s.import_rows(colour, LOW, high)
                s.import_rows(colour, HIGH, low)
            return
        ops, into = [], []
        if self.lo is not None:
            ops.append(dist.P2POp(dist.isend, s.export_rows(colour, LOW), self.lo))
        if self.hi is not None:
            ops.append(dist.P2POp(dist.isend, s.export_rows(colour, HIGH), self.hi))
        if self.hi is not None:
            t = s.empty_rows()
            ops.append(dist.P2POp(dist.irecv, t, self.hi))
            into.append((HIGH, t))
        if self.lo is not None:
            t = s.empty_rows()
            ops.append(dist.P2POp(dist.irecv, t, self.lo))
            into.append((LOW, t))
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        for side, t in into:
            s.import_rows(colour, side, t)


class SlabFilm:
    """A rank's slab of one film on the current CUDA device."""

    def __init__(self, heights, layers, y0, y1, *, periodic_x=False, periodic_y=False, packed=False, seed=1,
                 init="random", stream=None):
        import torch
        from . import isingfilm as I
        self.lat = I.Lattice.slab(heights, layers, y0, y1, periodic_x=periodic_x, periodic_y=periodic_y,
                                  packed=packed, seed=seed, init=init, stream=stream)
        self.info = self.lat.slab_info()
        self.stream = stream
        n = self.info["halo_bytes"]
        self._out = {side: torch.empty(n, dtype=torch.uint8, device="cuda") for side in (LOW, HIGH)}

    def empty_rows(self):
        import torch
        return torch.empty(self.info["halo_bytes"], dtype=torch.uint8, device="cuda")

    def export_rows(self, colour, side):
        buf = self._out[side]
        self.lat.slab_export(colour, side, buf.data_ptr(), self.stream)
        return buf

    def import_rows(self, colour, side, buf):
        self.lat.slab_import(colour, side, buf.data_ptr(), self.stream)

    def close(self):
        self.lat.close()


@dataclass
class SlabRun:
    records: list          # step records of the whole film
    M: np.ndarray          # whole-film M after every sweep
    B: np.ndarray          # whole-film B after every sweep
    n_occ: int


def whole_film_series(traces, shares):
    """Whole-film (M, B) per sweep from every slab's trace of its own change (rows: sweeps,
    columns: dM, dB) and creation shares (M0, 2B0, n_occ) of every slab."""
    dm = sum(np.asarray(t[:, 0], dtype=np.int64) for t in traces)
    db = sum(np.asarray(t[:, 1], dtype=np.int64) for t in traces)
    m0 = sum(int(s[0]) for s in shares)
    b2 = sum(int(s[1]) for s in shares)
    if b2 % 2:
        raise ValueError("the slabs' shares of 2B do not add up to an even number")
    return m0 + dm, b2 // 2 + db, sum(int(s[2]) for s in shares)


def run_local(heights, layers, sched, world, *, periodic_x=False, periodic_y=False, packed=False, seed=1,
              init="random", J=1.0):
    """The whole schedule on `world` slabs of one film held by this process (one device), with
    halos exchanged after every colour pass; returns the whole film's records, series and the
    slab films (spins readable per slab)."""
    from . import isingfilm as I
    R = np.asarray(heights).shape[0]
    total = int(np.sum(sched["eq"]) + np.sum(sched["meas"]))
    slabs = [SlabFilm(heights, layers, y0, y1, periodic_x=periodic_x, periodic_y=periodic_y, packed=packed,
                      seed=seed, init=init) for (y0, y1) in slab_bounds(R, world)]
    for s in slabs:
        s.lat.enable_trace(total)
        s.lat.set_schedule(sched["T"], sched["h"], sched["eq"], sched["meas"], J=J)
    exchange = LocalExchange(slabs, periodic_y)
    for _ in range(total):
        for c in range(4):
            for s in slabs:
                s.lat.run_pass(c)
            exchange(c)
    traces = [s.lat.trace() for s in slabs]
    shares = [(s.info["M0"], s.info["B2_0"], s.info["n_occ"]) for s in slabs]
    M, B, n_occ = whole_film_series(traces, shares)
    recs = I.fold_series(sched["T"], sched["h"], sched["eq"], sched["meas"], n_occ, M, B, J=J)
    return SlabRun(recs, M, B, n_occ), slabs


def run_dist(heights, layers, sched, *, periodic_x=False, periodic_y=False, packed=False, seed=1, init="random",
             J=1.0):
    """The whole schedule on this rank's slab of one film, one slab per rank of the initialised
    torch.distributed group (NCCL between GPUs): halos exchanged after every colour pass, the
    slabs' traces summed by an int64 all-reduce.  Every rank returns the whole film's records
    and series, and its slab film."""
    import torch
    import torch.distributed as dist
    from . import isingfilm as I
    rank, world = dist.get_rank(), dist.get_world_size()
    R = np.asarray(heights).shape[0]
    y0, y1 = slab_bounds(R, world)[rank]
    total = int(np.sum(sched["eq"]) + np.sum(sched["meas"]))
    s = SlabFilm(heights, layers, y0, y1, periodic_x=periodic_x, periodic_y=periodic_y, packed=packed, seed=seed,
                 init=init)
    s.lat.enable_trace(total)
    s.lat.set_schedule(sched["T"], sched["h"], sched["eq"], sched["meas"], J=J)
    exchange = DistExchange(s, rank, world, periodic_y)
    for _ in range(total):
        for c in range(4):
            s.lat.run_pass(c)
            exchange(c)
    tr = torch.from_numpy(s.lat.trace()).cuda()
    sh = torch.tensor([s.info["M0"], s.info["B2_0"], s.info["n_occ"]], dtype=torch.int64, device="cuda")
    dist.all_reduce(tr)
    dist.all_reduce(sh)
    M, B, n_occ = whole_film_series([tr.cpu().numpy()], [tuple(int(v) for v in sh.cpu().tolist())])
    recs = I.fold_series(sched["T"], sched["h"], sched["eq"], sched["meas"], n_occ, M, B, J=J)
    return SlabRun(recs, M, B, n_occ), s


def whole_spins(slabs, rows):
    """The whole film's spins [z][y][x] from every slab's own rows."""
    parts = []
    for s in slabs:
        sp = s.lat.spins()                      # the slab's local rows, halos included
        y0, y1, ya = s.info["y0"], s.info["y1"], s.info["ya"]
        parts.append(sp[:, y0 - ya:y1 - ya, :])
    out = np.concatenate(parts, axis=1)
    assert out.shape[1] == rows
    return out
