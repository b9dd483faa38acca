"""Benchmark: Metropolis spin-flip attempts/s of the CUDA path on one GB300 (or N replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload fractal256|flat16|fractal2048]
    python bench.py --impl reference ...      # the CPU oracle on a bounded sample, same metric

One step = one pass of the whole hot path over one film: the full temperature scan (or
hysteresis loop) of the workload, every sweep of every schedule step, with the spins resident
in device memory.  Synthetic seeded inputs (fractal height maps) stand in for the paper's STM
images.  Timing: CUDA events on the launching stream around each step; L2 is flushed between
steps (outside the events); W untimed warm-up steps; max over ranks.  Under torchrun every rank
runs its own replica of the film (the single-film path has no exchange step).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "spin-flip attempts/s and % roofline on 1 GB300, batched/served vs plain"
UNIT = "attempts/s"
# Integer operations the method needs per attempt, counted at source level: a quarter of a
# Philox4x32-10 block (10 rounds x (2 32x32->64 multiplies + 4 XORs + 2 key adds) / 4 = 25), the
# 12-neighbour sum (12) and the acceptance test and update (5).
OPS_PER_ATTEMPT = 40
SMS, LANES_PER_SM, SM_MAX_MHZ = 152, 128, 2070.0
ALU_PEAK_TOPS = SMS * LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12    # 40.3 T int32 lane-ops/s


def workload(name: str):
    from paper_1205_5588_gb300 import workloads as W
    if name == "fractal256":
        return W.fractal256_tscan()
    if name == "flat16":
        return W.flat16_hysteresis()
    if name == "fractal2048":
        return W.fractal2048_hysteresis()
    raise SystemExit(f"unknown workload {name}")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fp:
            for line in fp:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def flush_l2(buf):
    buf.fill_(1)     # 256 MiB write: larger than the 129 MB L2


def attempts_of(spec, n_occ):
    s = spec["schedule"]
    return int(n_occ) * int(s["eq"].sum() + s["meas"].sum())


def run_impl(args):
    import torch
    from paper_1205_5588_gb300 import distributed as D
    ranks = D.env_ranks()
    torch.cuda.set_device(ranks.local if ranks.world > 1 else 0)
    ranks = D.init("nccl")
    ws, rank = ranks.world, ranks.rank
    dev = torch.cuda.current_device()
    from paper_1205_5588_gb300 import build as B
    B.build()
    from paper_1205_5588_gb300 import isingfilm as I

    spec = workload(args.workload)
    sched = spec["schedule"]
    seed = D.replica_seed(spec["seed"], rank)   # a single film does not shard: one replica per rank
    stream = torch.cuda.current_stream()
    lat = I.Lattice(spec["heights"], spec["layers"], periodic_x=spec["periodic_x"], periodic_y=spec["periodic_y"],
                    packed=spec["packed"], seed=seed, init=spec["init"], stream=stream)
    if args.ctas or args.threads:
        lat.set_launch(args.ctas, args.threads)
    n_occ = lat.info()["n_occ"]
    per_step = attempts_of(spec, n_occ)
    l2buf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def one_step():
        lat.set_schedule(sched["T"], sched["h"], sched["eq"], sched["meas"], J=spec["J"])
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        lat.run(-1, stream=stream)
        b.record(stream)
        return a, b

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    D.barrier(ranks)
    clocks = Clocks(dev) if rank == 0 else None
    times = []
    for _ in range(args.steps):
        flush_l2(l2buf)
        a, b = one_step()
        b.synchronize()
        times.append(a.elapsed_time(b) / 1e3)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    total = D.max_over_ranks(sum(times), ranks, device="cuda")
    D.barrier(ranks)
    recs = lat.observables()
    shape = lat.launch_info()
    lat.close()
    value = per_step * args.steps * ws / total

    # end to end through the public API with host buffers: create from the host height map,
    # upload the schedule, run, read the observables back, every step
    e2e_times = []
    h2d = int(spec["heights"].nbytes) + int(sched["T"].nbytes + sched["h"].nbytes + sched["eq"].nbytes
                                             + sched["meas"].nbytes) + len(sched["T"]) * 52 * 4
    d2h = len(sched["T"]) * 96 + 4          # exact per-step records + the kernel status word
    heights_pinned = torch.from_numpy(spec["heights"]).pin_memory().numpy()
    for i in range(args.e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L2 = I.Lattice(heights_pinned, spec["layers"], periodic_x=spec["periodic_x"],
                       periodic_y=spec["periodic_y"], packed=spec["packed"], seed=seed, init=spec["init"],
                       stream=stream)
        L2.set_schedule(sched["T"], sched["h"], sched["eq"], sched["meas"], J=spec["J"])
        L2.run(-1, stream=stream)
        out = L2.observables()
        t1 = time.perf_counter()
        L2.close()
        assert len(out) == len(sched["T"])
        if i > 0:                      # first one warms the path
            e2e_times.append(t1 - t0)
    e2e_value = per_step * ws / statistics.mean(e2e_times)

    ms = total / args.steps * 1e3
    achieved_tops = OPS_PER_ATTEMPT * per_step / (total / args.steps) / 1e12
    traffic = load_traffic(args.workload)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int8" if not spec["packed"] else "u32 (1 bit/spin)",
        "data": "synthetic (seeded fractal height map stands in for the STM image)",
        "config": {"workload": spec["name"], "rows": int(spec["heights"].shape[0]),
                   "cols": int(spec["heights"].shape[1]), "layers": spec["layers"], "occupied_sites": n_occ,
                   "schedule_steps": int(len(sched["T"])), "sweeps_per_step_of_bench": int(sched["eq"].sum() + sched["meas"].sum()),
                   "attempts_per_step": per_step, "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU",
                   "final_abs_m_at_lowest_T": recs[0]["abs_m"] if recs else None},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "what": "isf_lattice_create from host heights + isf_set_schedule + isf_run_sweeps + isf_read_observables"},
        "gpu_launches": args.steps,
        "roofline": {"bound": "alu", "achieved": achieved_tops, "peak": ALU_PEAK_TOPS, "unit": "Tops/s",
                     "frac": achieved_tops / ALU_PEAK_TOPS, "traffic": traffic,
                     "kernel": ("k_resident (film in one cluster's shared memory)" if shape["path"] == "resident"
                                else "k_sweep (global-memory persistent kernel)"),
                     "launch": shape,
                     "sms_usable": shape["ctas"] if shape["path"] == "resident" else 152,
                     "peak_from": "152 SMs x 128 int32 lanes x 2070 MHz (issue-rate ceiling)",
                     "ops_per_attempt": OPS_PER_ATTEMPT},
        "clocks": clk,
    }
    if not args.no_multispin and args.workload != "fractal2048":
        m = measure_multispin(I, ranks)
        if rank == 0:
            line["multispin"] = m
    if not args.no_batched:
        # independent films: each rank runs its own share of the list (weak scaling)
        b = measure_batched(I, n_films=args.batch_films, sweeps_per_step=args.batch_sweeps, ranks=ranks,
                            plain=ranks.world == 1)
        bp = measure_batched(I, n_films=args.batch_films, sweeps_per_step=args.batch_sweeps, ranks=ranks,
                             plain=ranks.world == 1, packed=True)
        if rank == 0:
            line["batched"] = b
            line["batched_packed"] = bp
    if rank == 0 and not args.no_served:
        line["served"] = measure_served(I, rate=args.serve_rate, duration=args.serve_seconds)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(spec, budget_s=args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    D.finish(ranks)


def measure_multispin(I, ranks, steps=2, warmup=1):
    """The bit-packed multispin sweep on the 2048x2048x(2..6) film: one timed step is the whole
    hysteresis loop (641 field steps x 200 sweeps at T = 2), one k_sweep launch, L2 flushed
    between steps.  Under several ranks each rank runs its own replica."""
    import torch
    from paper_1205_5588_gb300 import distributed as D
    spec = workload("fractal2048")
    sched = spec["schedule"]
    lat = I.Lattice(spec["heights"], spec["layers"], packed=True, seed=D.replica_seed(spec["seed"], ranks.rank),
                    init=spec["init"])
    n_occ = lat.info()["n_occ"]
    per_step = attempts_of(spec, n_occ)
    l2buf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    times = []
    for i in range(warmup + steps):
        lat.set_schedule(sched["T"], sched["h"], sched["eq"], sched["meas"], J=spec["J"])
        flush_l2(l2buf)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        lat.run(-1, stream=stream)
        b.record(stream)
        b.synchronize()
        if i >= warmup:
            times.append(a.elapsed_time(b) / 1e3)
    shape = lat.launch_info()
    recs = lat.observables()
    lat.close()
    del l2buf
    total = D.max_over_ranks(sum(times), ranks, device="cuda")
    t_launch = sum(times) / len(times)
    achieved = OPS_PER_ATTEMPT * per_step / t_launch / 1e12
    return {"workload": spec["name"], "value": per_step * steps * ranks.world / total, "unit": UNIT,
            "dtype": "u32 (1 bit/spin)", "occupied_sites": n_occ, "attempts_per_step": per_step,
            "seconds_per_step": t_launch, "steps": steps, "warmup": warmup,
            "final_m": recs[-1]["m"] if recs else None,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": ALU_PEAK_TOPS, "unit": "Tops/s",
                         "frac": achieved / ALU_PEAK_TOPS, "traffic": load_traffic("fractal2048"),
                         "kernel": "k_sweep<packed> (global-memory persistent kernel)", "launch": shape,
                         "ops_per_attempt": OPS_PER_ATTEMPT}}


def measure_batched(I, n_films=128, sweeps_per_step=20, seed=4, plain=True, ranks=None, packed=False):
    """Batched films (ragged sizes 64..1024, 1..8 layers, own T and field loop each) advanced to
    the end of their schedules by isf_batch_run, against the same films run one per launch; int8
    or bit-packed spins.  Under several ranks each rank runs its round-robin share of the films."""
    import torch
    from paper_1205_5588_gb300 import distributed as D
    from paper_1205_5588_gb300 import workloads as W
    ranks = ranks or D.env_ranks()
    films = W.batch_films(n_films, seed=seed, sweeps_per_step=sweeps_per_step)
    films = [films[i] for i in D.shard(len(films), ranks.rank, ranks.world)]
    lats = []
    for f in films:
        L = I.Lattice(f["heights"], f["layers"], seed=f["seed"], packed=packed)
        lats.append(L)
    att = sum(L.info()["n_occ"] * int(f["schedule"]["eq"].sum() + f["schedule"]["meas"].sum())
              for L, f in zip(lats, films))

    def reset():
        for L, f in zip(lats, films):
            sc = f["schedule"]
            L.set_schedule(sc["T"], sc["h"], sc["eq"], sc["meas"])

    reset()
    b = I.Batch(lats, graph=True)
    b.tune()
    b.run()                       # warm: kernels loaded, graph captured
    torch.cuda.synchronize()
    reset()
    D.barrier(ranks)
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    b.run()
    e.record()
    e.synchronize()
    t_batch = D.max_over_ranks(a.elapsed_time(e) / 1e3, ranks, device="cuda")
    att_all = int(D.sum_over_ranks(att, ranks, device="cuda"))
    out = {"value": att_all / t_batch, "unit": UNIT, "films": n_films, "attempts": att_all, "seconds": t_batch,
           "spins": "u32 (1 bit/spin)" if packed else "int8",
           "sweeps_per_step": sweeps_per_step, "launch": b.info(), "graph": True,
           "ranks": ranks.world, "scaling": "weak (films dealt out across ranks)"}
    b.close()
    if plain:
        reset()
        torch.cuda.synchronize()
        a.record()
        for L in lats:
            L.run(-1)
        e.record()
        e.synchronize()
        t_plain = a.elapsed_time(e) / 1e3
        out["plain_one_film_per_launch"] = {"value": att / t_plain, "unit": UNIT, "seconds": t_plain}
        out["speedup_vs_plain"] = t_plain / t_batch
    for L in lats:
        L.close()
    return out


def measure_served(I, rate=200.0, duration=5.0, seed=5, pool=24, budget_gb=40.0, sweeps_per_tick=50, packed=True):
    """Poisson stream of hysteresis-loop and temperature-scan jobs (50/50) on films with
    log-normal side length (median 256, 64..2048) and 1..8 layers, bit-packed spins, served with
    continuous batching; latency is submit -> completion."""
    import torch
    from paper_1205_5588_gb300 import workloads as W
    rng = np.random.Generator(np.random.PCG64(seed))
    maps = []
    for i in range(pool):
        R, Cc = W.lognormal_side(rng), W.lognormal_side(rng)
        L = int(rng.integers(1, 9))
        maps.append((W.fractal_heights(R, Cc, float(rng.uniform(0.5, 0.9)), 1, L, seed=5000 + i), L))
    hyst_h = W.loop_fields(40, 10)                         # +4 -> -4 -> +4 by 0.1, 161 steps
    arrivals = W.poisson_arrivals(rate, duration, seed=seed)
    jobs = []
    for k in range(len(arrivals)):
        H, L = maps[int(rng.integers(0, pool))]
        if rng.random() < 0.5:
            sc = W.schedule(float(rng.uniform(1.0, 10.0)), hyst_h, 0, 50)
        else:
            sc = W.schedule(np.linspace(0.5, 12.0, 24), 0.0, 200, 200)
        jobs.append((H, L, sc, 10000 + k))
    srv = I.Server(int(budget_gb * (1 << 30)), sweeps_per_tick=sweeps_per_tick)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ids = []
    for (H, L, sc, sd), t_arr in zip(jobs, arrivals):
        dt = t0 + t_arr - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        ids.append(srv.submit(H, L, sc["T"], sc["h"], sc["eq"], sc["meas"], seed=sd, packed=packed))
    lat = []
    for jid in ids:
        state = srv.wait(jid, timeout=600.0)
        if state != "done":
            raise RuntimeError(f"served job {jid} ended {state}")
        _, _, l = srv.result(jid)
        lat.append(l)
        srv.release(jid)
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    lat = np.array(lat)
    return {"value": st["attempts_done"] / wall, "unit": UNIT, "jobs": len(ids), "rate_per_s": rate,
            "arrival_window_s": duration, "wall_s": wall,
            "offered": st["attempts_done"] / duration, "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)), "ticks": st["ticks"], "sweeps_per_tick": sweeps_per_tick,
            "gpu_busy_s": st["busy_s"], "peak_device_bytes": st["peak_bytes"],
            "spins": "u32 (1 bit/spin)" if packed else "int8"}


# dram__bytes_read.sum + dram__bytes_write.sum of one bench launch of the dominant kernel, from
# the ncu captures summarised in profiles/, valid while the kernel's sources hash to the
# recorded value (None: not captured for the current sources).
NCU_TRAFFIC = {
    "fractal256": {"sources": ["kernels_resident.cu", "sweep_core.cuh", "device_common.cuh"],
                   "sources_sha256": "f36ebbab1af1299b3c47ee70d982d7ff64c27ea00cc75d4b1f52033a3fddf4b6",
                   "bytes_per_launch": 1309952.0},
    "fractal2048": {"sources": ["kernels_sweep.cu", "sweep_core.cuh", "device_common.cuh"],
                    "sources_sha256": "1eaef32c6540c29532335150a443768566022045f45b69e381857ffcc1ad8d5d",
                    "bytes_per_launch": 21053440.0 + 2549504.0},
}


def kernel_sources_sha256(names) -> str:
    import hashlib
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_1205_5588_gb300", "csrc", name), "rb") as fp:
            h.update(fp.read())
    return h.hexdigest()


def load_traffic(workload_name):
    rec = NCU_TRAFFIC.get(workload_name)
    if not rec or rec["sources_sha256"] != kernel_sources_sha256(rec["sources"]):
        return None
    return rec["bytes_per_launch"]


def cpu_baseline(spec, budget_s=15.0, max_sweeps=None):
    """The oracle as it stands, single-threaded, on a bounded sample of the same film: sweeps of
    the first schedule step until the time budget is used."""
    from oracle import oracle
    init = {"random": oracle.INIT_RANDOM, "up": oracle.INIT_UP, "down": oracle.INIT_DOWN}[spec["init"]]
    flags = (1 if spec["periodic_x"] else 0) | (2 if spec["periodic_y"] else 0)
    f = oracle.Film(spec["heights"], spec["layers"], flags=flags, seed=spec["seed"], init=init)
    n_occ = f.info()["n_occ"]
    s = spec["schedule"]
    T0, h0 = float(s["T"][0]), float(s["h"][0])
    done = 0
    chunk = 1
    t0 = time.perf_counter()
    while True:
        f.run([T0], [h0], [0], [chunk])
        done += chunk
        el = time.perf_counter() - t0
        if el >= budget_s or (max_sweeps and done >= max_sweeps):
            break
        chunk = max(1, min(chunk * 2, int(done * (budget_s - el) / max(el, 1e-6)) or 1))
    el = time.perf_counter() - t0
    f.close()
    return {"value": n_occ * done / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} sweeps of the first schedule step (T={T0}, h={h0}) on the full {spec['name']} film, "
                      f"{n_occ} occupied sites, {el:.1f} s single-threaded"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    spec = workload(args.workload)
    from oracle import oracle
    oracle.load()
    init = {"random": oracle.INIT_RANDOM, "up": oracle.INIT_UP, "down": oracle.INIT_DOWN}[spec["init"]]
    flags = (1 if spec["periodic_x"] else 0) | (2 if spec["periodic_y"] else 0)
    f = oracle.Film(spec["heights"], spec["layers"], flags=flags, seed=spec["seed"], init=init)
    n_occ = f.info()["n_occ"]
    s = spec["schedule"]
    sweeps = args.ref_sweeps or max(1, int(2.0e7 // max(n_occ, 1)))    # ~ a few seconds per step
    for _ in range(args.warmup):
        f.run([float(s["T"][0])], [float(s["h"][0])], [0], [1])
    times = []
    for k in range(args.steps):
        kk = k % len(s["T"])
        t0 = time.perf_counter()
        f.run([float(s["T"][kk])], [float(s["h"][kk])], [0], [sweeps])
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = n_occ * sweeps * args.steps / total
    sample = (f"{sweeps} sweeps per step at the workload's schedule temperatures/fields, full {spec['name']} "
              f"film ({n_occ} occupied sites), single-threaded CPU oracle")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int8", "data": "synthetic",
        "config": {"workload": spec["name"], "occupied_sites": n_occ, "sweeps_per_step": sweeps},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)
    f.close()


def profile_case(args):
    """Small case for ncu captures of the sweep kernel: the workload's film, one launch of
    --profile-sweeps sweeps at the first schedule step."""
    import torch
    torch.cuda.set_device(0)
    from paper_1205_5588_gb300 import build as B
    B.build()
    from paper_1205_5588_gb300 import isingfilm as I
    spec = workload(args.workload)
    s = spec["schedule"]
    lat = I.Lattice(spec["heights"], spec["layers"], periodic_x=spec["periodic_x"], periodic_y=spec["periodic_y"],
                    packed=spec["packed"], seed=spec["seed"], init=spec["init"])
    if args.path != "auto":
        lat.set_path(args.path)
    if args.ctas or args.threads:
        lat.set_launch(args.ctas, args.threads)
    lat.set_schedule(s["T"][:1], s["h"][:1], [0], [args.profile_sweeps], J=spec["J"])
    lat.run(-1)
    print("profile case done, M_last =", lat.observables()[0]["M_last"], "launch", lat.launch_info())
    lat.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--workload", default="fractal256", choices=["fractal256", "flat16", "fractal2048"])
    ap.add_argument("--ctas", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=2, help="end-to-end steps (at least 1)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-multispin", action="store_true", help="skip the bit-packed 2048^2 loop leg")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--batch-films", type=int, default=128)
    ap.add_argument("--batch-sweeps", type=int, default=20, help="sweeps per schedule step of the batched films")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-seconds", type=float, default=5.0)
    ap.add_argument("--ref-sweeps", type=int, default=0)
    ap.add_argument("--path", default="auto", choices=["auto", "global", "resident", "slabs"],
                    help="sweep kernel of the profiling case")
    ap.add_argument("--profile-sweeps", type=int, default=0,
                    help="profiling case: one launch of this many sweeps at the first schedule step, no JSON")
    args = ap.parse_args()
    args.e2e_steps = max(1, args.e2e_steps)
    if args.profile_sweeps:
        profile_case(args)
        return
    if args.warmup < 3 and args.impl == "cuda":
        print("note: warm-up raised to 3 steps", file=sys.stderr)
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_impl(args)


if __name__ == "__main__":
    main()
