"""Benchmark: Metropolis spin-flip attempts/s of the CUDA path on one GB300 (or N replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload fractal2048|fractal256|flat16]
    python bench.py --impl reference ...      # the CPU oracle on a bounded sample, same metric

Headline (`value`): the 2048 x 2048 x (2..6) fractal film with bit-packed spins (one bit per
spin, 32 spins per uint32 word), hysteresis loop at T = 2 with h = +8 -> -8 -> +8 in steps of 0.05
(641 field steps x 200 sweeps).  One step = one pass of the whole hot path over that film: every
sweep of every field step, spins resident in device memory, one persistent launch.  Synthetic
seeded inputs (fractal height maps) stand in for the paper's STM images.

Timing: CUDA events on the launching stream around each step; L2 is flushed between steps
(256 MiB write, outside the events); W >= 3 untimed warm-up steps; max over ranks.  Under
torchrun every rank runs its own replica of the film (the single-film path has no exchange
step).  Further legs in the same JSON line: the 256^2 int8 temperature scan (one film in one
cluster's shared memory), batched films (512 ragged films, int8 and bit-packed) against the same
films one per launch, a served Poisson job stream at a sustainable and at the stated rate, and
the integer-issue ceilings the rooflines divide by, measured in the same run.
"""
from __future__ import annotations

import argparse
import hashlib
import json
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
LANES_PER_SM = 128          # dispatch: 4 sub-partitions x one 32-lane warp instruction per clock


def workload(name: str, schedule_steps: int = 0):
    """The named workload; schedule_steps > 0 keeps only the first steps of its schedule (quick
    timings of the same kernel on the same film; not a bench value)."""
    from paper_1205_5588_gb300 import workloads as W
    if name == "fractal2048":
        spec = W.fractal2048_hysteresis()
    elif name == "fractal256":
        spec = W.fractal256_tscan()
    elif name == "flat16":
        spec = W.flat16_hysteresis()
    else:
        raise SystemExit(f"unknown workload {name}")
    if schedule_steps > 0:
        spec["schedule"] = {k: v[:schedule_steps].copy() for k, v in spec["schedule"].items()}
        spec["name"] += f"_first{schedule_steps}steps"
    return spec


KERNEL_OF_PATH = {("global", True): "k_words (bit-packed word lists, persistent kernel on all SMs)",
                  ("global", False): "k_sweep<int8> (global-memory persistent kernel)",
                  ("resident", False): "k_resident (film in one cluster's shared memory)",
                  ("resident", True): "k_resident (film in one cluster's shared memory)",
                  ("slabs", True): "k_slabs (row bands in shared memory)"}


def kernel_of(shape, packed):
    return KERNEL_OF_PATH.get((shape["path"], bool(packed)), shape["path"])


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


def events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


# ---------------------------------------------------------------- integer-issue ceilings ----
def probe_peaks(I, stream, target_s=0.05, reps=3) -> dict:
    """The integer-issue ceilings of this GPU (isf_peak_probe), each the best of `reps` timed
    launches (CUDA events on `stream`) of about target_s seconds, after a warm-up launch."""
    import torch
    out = {}
    for mode, threads, key, unit in ((I.PEAK_LOP3, 1024, "lop3_lane_ops_per_s", "lane-ops"),
                                     (I.PEAK_MIX, 1024, "mix_lane_ops_per_s", "lane-ops"),
                                     (I.PEAK_PHILOX, 512, "philox_blocks_per_s", "blocks"),
                                     (I.PEAK_ATTEMPT, 512, "attempts_per_s_arithmetic", "attempts")):
        iters = 64
        best = 0.0
        for rep in range(reps + 8):
            a, b = events()
            a.record(stream)
            units = I.peak_probe(mode, 0, threads, iters, stream=stream)
            b.record(stream)
            b.synchronize()
            dt = a.elapsed_time(b) / 1e3
            if dt < 0.5 * target_s and rep < 8:        # grow the launch until it runs ~target_s
                iters = int(iters * min(64.0, max(2.0, target_s / max(dt, 1e-6))))
                continue
            best = max(best, units / dt)
        out[key] = best
    torch.cuda.synchronize()
    return out


def roofline(attempts_per_launch, t_launch, peaks, sms, sm_max_mhz, kernel, shape, traffic, inst_per_attempt,
             pipes=None):
    """ALU roofline of one sweep launch, both sides in the algorithmic unit (40 int-ops per
    attempt): achieved = 40 x attempts / launch time; peak = 40 x the attempts/s this GPU reaches
    on the per-attempt arithmetic alone (isf_peak_probe ISF_PEAK_ATTEMPT, measured in this run)."""
    rate = attempts_per_launch / t_launch
    achieved = OPS_PER_ATTEMPT * rate / 1e12
    peak = OPS_PER_ATTEMPT * peaks["attempts_per_s_arithmetic"] / 1e12
    derived = sms * LANES_PER_SM * sm_max_mhz * 1e6 if sm_max_mhz else None
    ceil = {
        "sms": sms, "sm_max_mhz": sm_max_mhz,
        "lane_issue_lop3_Tops": peaks["lop3_lane_ops_per_s"] / 1e12,
        "lane_issue_mix_Tops": peaks["mix_lane_ops_per_s"] / 1e12,
        "lane_issue_derived_Tops": derived / 1e12 if derived else None,
        "philox_blocks_per_s": peaks["philox_blocks_per_s"],
        "attempts_per_s_if_every_attempt_draws_a_word": 4.0 * peaks["philox_blocks_per_s"],
        "attempts_per_s_arithmetic": peaks["attempts_per_s_arithmetic"],
        "frac_of_philox_ceiling": rate / (4.0 * peaks["philox_blocks_per_s"]),
        "frac_of_arithmetic_ceiling": rate / peaks["attempts_per_s_arithmetic"],
        "inst_per_attempt": inst_per_attempt,
        "frac_of_lop3_issue_by_instructions": (inst_per_attempt * rate / peaks["lop3_lane_ops_per_s"]
                                               if inst_per_attempt else None),
        "frac_of_dispatch_by_instructions": (inst_per_attempt * rate / derived if inst_per_attempt and derived
                                             else None),
    }
    if pipes:
        # from the committed ncu capture of the kernel's small case: how busy its issue slots and its
        # integer ALU pipe were, and the attempts/s its own ALU work would allow at a full ALU pipe
        ceil["ncu_issue_active"] = pipes["issue_active"]
        ceil["ncu_alu_pipe_busy"] = pipes["alu_pipe"]
        ceil["attempts_per_s_at_full_alu_pipe"] = rate / pipes["alu_pipe"]
        ceil["frac_of_own_alu_pipe_ceiling"] = pipes["alu_pipe"]
    # a film held by one cluster runs on that cluster's SMs only: its share of their ceiling
    used = shape.get("ctas") if shape.get("path") == "resident" else sms
    if used and used < sms:
        ceil["sms_in_use"] = used
        ceil["frac_of_arithmetic_ceiling_of_sms_in_use"] = rate / (peaks["attempts_per_s_arithmetic"] * used / sms)
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": kernel, "launch": shape, "ops_per_attempt": OPS_PER_ATTEMPT,
            "peak_from": "measured in this run on this GPU: 40 x the attempts/s of the per-attempt integer "
                         "arithmetic alone (a 32-site word's 8 Philox4x32-10 blocks, bit-sliced neighbour count, "
                         "table lookups and compares; registers only, all SMs, no film loads, no barriers; "
                         "isf_peak_probe ISF_PEAK_ATTEMPT), CUDA events, best of 3",
            "ceilings": ceil}


# ---------------------------------------------------------------- one film, timed ----
def time_film(I, spec, seed, steps, warmup, stream, l2buf, path="auto", launch=(0, 0)):
    """W warm-up and K timed passes of the whole schedule of one film; returns per-step seconds
    (CUDA events on `stream`), attempts per step, launch shape, records and a sweep-kernel launch
    count of the timed region."""
    import torch
    sched = spec["schedule"]
    lat = I.Lattice(spec["heights"], spec["layers"], periodic_x=spec["periodic_x"], periodic_y=spec["periodic_y"],
                    packed=spec["packed"], seed=seed, init=spec["init"], stream=stream)
    if path != "auto":
        lat.set_path(path)
    if launch[0] or launch[1]:
        lat.set_launch(*launch)
    n_occ = lat.info()["n_occ"]
    per_step = attempts_of(spec, n_occ)
    times = []
    for i in range(warmup + steps):
        lat.set_schedule(sched["T"], sched["h"], sched["eq"], sched["meas"], J=spec["J"])
        if i >= warmup:
            flush_l2(l2buf)
        a, b = events()
        a.record(stream)
        lat.run(-1, stream=stream)
        b.record(stream)
        b.synchronize()
        if i >= warmup:
            times.append(a.elapsed_time(b) / 1e3)
    torch.cuda.synchronize()
    shape = lat.launch_info()
    recs = lat.observables()
    lat.close()
    return {"times": times, "per_step": per_step, "n_occ": n_occ, "shape": shape, "recs": recs}


def e2e_film(I, spec, seed, steps, stream):
    """End to end through the public C ABI from host buffers, every step: isf_lattice_create
    from the pinned host height map, isf_set_schedule from host arrays, isf_run_sweeps,
    isf_read_observables back to the host.  The first pass warms the path."""
    import torch
    sched = spec["schedule"]
    heights_pinned = torch.from_numpy(spec["heights"]).pin_memory().numpy()
    ts = []
    for i in range(steps + 1):
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
        if i > 0:
            ts.append(t1 - t0)
    h2d = int(spec["heights"].nbytes) + len(sched["T"]) * (52 * 4 + 8)    # heights; per step: table, eq, total
    d2h = len(sched["T"]) * 96 + 4                                        # per-step records + status word
    return {"seconds": ts, "h2d": h2d, "d2h": d2h}


# dram__bytes_read.sum + dram__bytes_write.sum of one bench launch of the dominant kernel, and
# its thread-instructions per attempt (smsp__inst_executed.sum x threads per instruction /
# attempts), from the ncu captures summarised in profiles/; each valid while the kernel's sources
# hash to the recorded value (None: not captured for the current sources).
NCU_RECORDS = {
    "fractal256": {"sources": ["kernels_resident.cu", "sweep_core.cuh", "device_common.cuh"],
                   "sources_sha256": "7eb0ceb4c157983f4913e350a6e95a2ee2a8151005e81e97642390bfe346bf67",
                   "bytes_per_launch": 1785344.0 + 0.0, "inst_per_attempt": None,
                   "pipes": {"issue_active": 0.491, "alu_pipe": 0.381}},
    "fractal2048": {"sources": ["kernels_words.cu", "sweep_core.cuh", "device_common.cuh", "grid_sync.cuh"],
                    "sources_sha256": "03fa43aa3b5ac631b510b1dab797589a2e3e49d1af96b5f1c0b3c544ee1b47ef",
                    "bytes_per_launch": 21731584.0 + 781824.0, "inst_per_attempt": 25.86,
                    "pipes": {"issue_active": 0.513, "alu_pipe": 0.477}},
}


def kernel_sources_sha256(names) -> str:
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_1205_5588_gb300", "csrc", name), "rb") as fp:
            h.update(fp.read())
    return h.hexdigest()


def ncu_record(workload_name, key):
    rec = NCU_RECORDS.get(workload_name)
    if not rec or rec["sources_sha256"] != kernel_sources_sha256(rec["sources"]):
        return None
    return rec[key]


def load_traffic(workload_name):
    return ncu_record(workload_name, "bytes_per_launch")


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

    spec = workload(args.workload, args.schedule_steps)
    sched = spec["schedule"]
    seed = D.replica_seed(spec["seed"], rank)   # a single film does not shard: one replica per rank
    stream = torch.cuda.current_stream()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    l2buf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    peaks = probe_peaks(I, stream)

    D.barrier(ranks)
    clocks = Clocks(dev) if rank == 0 else None
    leg = time_film(I, spec, seed, args.steps, args.warmup, stream, l2buf, path=args.path,
                    launch=(args.ctas, args.threads))
    clk = clocks.stop() if clocks else None
    total = D.max_over_ranks(sum(leg["times"]), ranks, device="cuda")
    D.barrier(ranks)
    per_step = leg["per_step"]
    value = per_step * args.steps * ws / total
    t_launch = sum(leg["times"]) / len(leg["times"])
    shape = leg["shape"]
    sm_max = (clk or {}).get("sm_max_mhz")
    e2e = e2e_film(I, spec, seed, args.e2e_steps, stream)
    e2e_value = per_step * ws / statistics.mean(e2e["seconds"])

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "u32 (1 bit/spin, 32 spins per word)" if spec["packed"] else "int8",
        "data": "synthetic (seeded fractal height map stands in for the STM image)",
        "config": {"workload": spec["name"], "rows": int(spec["heights"].shape[0]),
                   "cols": int(spec["heights"].shape[1]), "layers": spec["layers"], "occupied_sites": leg["n_occ"],
                   "schedule_steps": int(len(sched["T"])),
                   "sweeps_per_step_of_bench": int(sched["eq"].sum() + sched["meas"].sum()),
                   "attempts_per_step": per_step, "spins": "bit-packed" if spec["packed"] else "int8",
                   "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU",
                   "final_m": leg["recs"][-1]["m"] if leg["recs"] else None},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"],
                "steps": args.e2e_steps,
                "what": "isf_lattice_create from pinned host heights + isf_set_schedule + isf_run_sweeps + "
                        "isf_read_observables, every step"},
        "gpu_launches": args.steps,
        "roofline": roofline(per_step, t_launch, peaks, sms, sm_max, kernel_of(shape, spec["packed"]),
                             shape, load_traffic(args.workload), ncu_record(args.workload, "inst_per_attempt"),
                             ncu_record(args.workload, "pipes")),
        "clocks": clk,
    }
    if not args.no_tscan and args.workload != "fractal256":
        t = time_film(I, workload("fractal256"), D.replica_seed(1, rank), args.leg_steps, 3, stream, l2buf)
        tl = sum(t["times"]) / len(t["times"])
        tot = D.max_over_ranks(sum(t["times"]), ranks, device="cuda")
        if rank == 0:
            line["tscan256"] = {
                "workload": "fractal256x256x6_tscan", "value": t["per_step"] * len(t["times"]) * ws / tot,
                "unit": UNIT, "dtype": "int8", "occupied_sites": t["n_occ"], "attempts_per_step": t["per_step"],
                "seconds_per_step": tl, "steps": len(t["times"]), "warmup": 3,
                "roofline": roofline(t["per_step"], tl, peaks, sms, sm_max,
                                     kernel_of(t["shape"], False), t["shape"],
                                     load_traffic("fractal256"), ncu_record("fractal256", "inst_per_attempt"),
                                     ncu_record("fractal256", "pipes"))}
    del l2buf
    if not args.no_batched:
        # independent films: each rank runs its own share of the list (weak scaling)
        b = measure_batched(I, n_films=args.batch_films, sweeps_per_step=args.batch_sweeps, ranks=ranks,
                            plain=ranks.world == 1)
        bp = measure_batched(I, n_films=args.batch_films, sweeps_per_step=args.batch_sweeps, ranks=ranks,
                             plain=ranks.world == 1, packed=True)
        if rank == 0:
            # the whole GPU's share of the per-attempt arithmetic ceiling measured above (the packed
            # word's form; an int8 attempt costs more instructions)
            for leg in (b, bp):
                leg["frac_of_arithmetic_ceiling"] = leg["value"] / (ws * peaks["attempts_per_s_arithmetic"])
            line["batched"] = b
            line["batched_packed"] = bp
    if rank == 0 and not args.no_served:
        line["served"] = measure_served(I, rate=args.serve_rate, duration=args.serve_seconds)
        line["served_sustainable"] = measure_served(I, rate=args.serve_rate_sustainable,
                                                    duration=args.serve_seconds_sustainable)
        if args.serve_rate_over > 0:
            # twice the stated stream: offered load above what the GPU serves, so the achieved
            # rate is the server's capacity and the latencies include the backlog
            line["served_over_capacity"] = measure_served(I, rate=args.serve_rate_over,
                                                          duration=args.serve_seconds_over)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(spec, budget_s=args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    D.finish(ranks)


def measure_batched(I, n_films=512, sweeps_per_step=100, seed=4, plain=True, ranks=None, packed=False,
                    plain_every=8):
    """Batched films (ragged sizes 64..1024, 1..8 layers, own T and field loop each) advanced to
    the end of their schedules by isf_batch_run, int8 or bit-packed spins, against the same films
    run one per launch on every `plain_every`-th film (a sample, to bound the time).  Under several
    ranks each rank runs its round-robin share of the films."""
    import torch
    from paper_1205_5588_gb300 import distributed as D
    from paper_1205_5588_gb300 import workloads as W
    ranks = ranks or D.env_ranks()
    films = W.batch_films(n_films, seed=seed, sweeps_per_step=sweeps_per_step)
    films = [films[i] for i in D.shard(len(films), ranks.rank, ranks.world)]
    lats = [I.Lattice(f["heights"], f["layers"], seed=f["seed"], packed=packed) for f in films]
    atts = [L.info()["n_occ"] * int(f["schedule"]["eq"].sum() + f["schedule"]["meas"].sum())
            for L, f in zip(lats, films)]
    att = sum(atts)

    def reset(sel=None):
        for i, (L, f) in enumerate(zip(lats, films)):
            if sel is None or i in sel:
                sc = f["schedule"]
                L.set_schedule(sc["T"], sc["h"], sc["eq"], sc["meas"])

    reset()
    b = I.Batch(lats, graph=True)
    b.tune()
    b.run(max_sweeps=sweeps_per_step)     # warm: kernels loaded, graph captured (one step's sweeps)
    torch.cuda.synchronize()
    reset()
    D.barrier(ranks)
    a, e = events()
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
        sel = set(range(0, len(films), plain_every))
        reset(sel)
        torch.cuda.synchronize()
        a.record()
        for i in sorted(sel):
            lats[i].run(-1)
        e.record()
        e.synchronize()
        t_plain = a.elapsed_time(e) / 1e3
        att_plain = sum(atts[i] for i in sel)
        out["plain_one_film_per_launch"] = {"value": att_plain / t_plain, "unit": UNIT, "seconds": t_plain,
                                            "films": len(sel), "attempts": att_plain,
                                            "sample": f"every {plain_every}th film of the batch"}
        out["speedup_vs_plain"] = out["value"] / (att_plain / t_plain)
    for L in lats:
        L.close()
    return out


def measure_served(I, rate=200.0, duration=60.0, seed=5, pool=128, budget_gb=40.0, sweeps_per_tick=50, packed=True):
    """Poisson stream of hysteresis-loop and temperature-scan jobs (50/50) on films with
    log-normal side length (median 256, 64..2048) and 1..8 layers, bit-packed spins, served with
    continuous batching; latency is submit -> completion.  Films come from a pool of `pool`
    seeded maps (each job with its own seed, temperature and schedule)."""
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
    offered = 0
    for H, L, sc, _ in jobs:
        n_sites = int(np.minimum(H, L).sum())
        offered += n_sites * int(sc["eq"].sum() + sc["meas"].sum())
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
        state = srv.wait(jid, timeout=900.0)
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
            "offered": offered / duration, "sustained": bool(wall < duration * 1.1 + 2.0),
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "ticks": st["ticks"], "sweeps_per_tick": sweeps_per_tick,
            "gpu_busy_s": st["busy_s"], "peak_device_bytes": st["peak_bytes"], "map_pool": pool,
            "spins": "u32 (1 bit/spin)" if packed else "int8"}


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
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
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
    sweeps = args.ref_sweeps or max(1, int(2.0e7 // max(n_occ, 1)))    # ~ a second per step
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
    sample = (f"{sweeps} sweep(s) per step at the workload's schedule temperatures/fields in order, full "
              f"{spec['name']} film ({n_occ} occupied sites), single-threaded CPU oracle")
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
    --profile-sweeps sweeps at schedule step --profile-step (default the first)."""
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
    k = args.profile_step
    lat.set_schedule(s["T"][k:k + 1], s["h"][k:k + 1], [0], [args.profile_sweeps], J=spec["J"])
    lat.run(-1)
    print("profile case done, M_last =", lat.observables()[0]["M_last"], "launch", lat.launch_info())
    lat.close()


def sizes_case(args):
    """The bit-packed film of the headline's kind (fractal map, Hurst 0.8, layers 2..6, all up) at
    several sizes, on the global-memory word kernel and on the row-slab kernel: microseconds per
    sweep over the loop's first 3 field steps (200 sweeps each), best of 3 after a warm-up, CUDA
    events; one JSON line per film and path."""
    import torch
    torch.cuda.set_device(0)
    from paper_1205_5588_gb300 import build as B
    B.build()
    from paper_1205_5588_gb300 import isingfilm as I
    from paper_1205_5588_gb300 import workloads as W
    spec = W.fractal2048_hysteresis()
    s = spec["schedule"]
    T, h, eq, me = (s[k][:3] for k in ("T", "h", "eq", "meas"))
    sweeps = int(eq.sum() + me.sum())
    stream = torch.cuda.current_stream()
    for n in [int(x) for x in args.sizes.split(",")]:
        H = W.fractal_heights(n, n, 0.8, 2, 6, seed=3)
        for path in ("global", "slabs"):
            lat = I.Lattice(H, 6, packed=True, seed=1, init="up", stream=stream)
            lat.set_path(path)
            ts = []
            for rep in range(4):
                lat.set_schedule(T, h, eq, me, J=spec["J"])
                a, b = events()
                a.record(stream)
                lat.run(-1, stream=stream)
                b.record(stream)
                b.synchronize()
                ts.append(a.elapsed_time(b) / 1e3)
            print(json.dumps({"size": n, "path": path, "us_per_sweep": min(ts[1:]) / sweeps * 1e6,
                              "occupied_sites": lat.info()["n_occ"], "launch": lat.launch_info()}), flush=True)
            lat.close()


def probe_case(args):
    """The integer-issue probes alone: the ceilings as the bench measures them, or (with
    --probe-iters) one launch of each probe of that many iterations, for ncu captures."""
    import torch
    torch.cuda.set_device(0)
    from paper_1205_5588_gb300 import build as B
    B.build()
    from paper_1205_5588_gb300 import isingfilm as I
    stream = torch.cuda.current_stream()
    if not args.probe_iters:
        print(json.dumps(probe_peaks(I, stream)))
        return
    out = {}
    for mode, threads in ((I.PEAK_LOP3, 1024), (I.PEAK_MIX, 1024), (I.PEAK_PHILOX, 512), (I.PEAK_ATTEMPT, 512)):
        a, b = events()
        a.record(stream)
        units = I.peak_probe(mode, 0, threads, args.probe_iters, stream=stream)
        b.record(stream)
        b.synchronize()
        out[mode] = {"units": units, "seconds": a.elapsed_time(b) / 1e3}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--workload", default="fractal2048", choices=["fractal2048", "fractal256", "flat16"])
    ap.add_argument("--path", default="auto", choices=["auto", "global", "resident", "slabs"],
                    help="sweep kernel (auto = the library's choice)")
    ap.add_argument("--ctas", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=2, help="end-to-end steps (at least 1)")
    ap.add_argument("--leg-steps", type=int, default=3, help="timed steps of the 256^2 scan leg")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-tscan", action="store_true", help="skip the 256^2 int8 scan leg")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--batch-films", type=int, default=512)
    ap.add_argument("--batch-sweeps", type=int, default=100, help="sweeps per schedule step of the batched films")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-rate-sustainable", type=float, default=100.0)
    ap.add_argument("--serve-seconds-sustainable", type=float, default=20.0)
    ap.add_argument("--serve-rate-over", type=float, default=400.0, help="0 = no over-capacity serving leg")
    ap.add_argument("--serve-seconds-over", type=float, default=20.0)
    ap.add_argument("--ref-sweeps", type=int, default=0)
    ap.add_argument("--schedule-steps", type=int, default=0,
                    help="time only the first N steps of the workload's schedule (quick kernel timings)")
    ap.add_argument("--profile-step", type=int, default=0, help="schedule step of the --profile-sweeps case")
    ap.add_argument("--profile-sweeps", type=int, default=0,
                    help="profiling case: one launch of this many sweeps at the first schedule step, no JSON")
    ap.add_argument("--sizes", default="", help="comma-separated film sides: time the packed film on both paths")
    ap.add_argument("--probe", action="store_true", help="print the integer-issue ceilings only")
    ap.add_argument("--probe-iters", type=int, default=0,
                    help="with --probe: one launch of each probe of this many iterations per thread")
    args = ap.parse_args()
    args.e2e_steps = max(1, args.e2e_steps)
    if args.profile_sweeps:
        profile_case(args)
        return
    if args.sizes:
        sizes_case(args)
        return
    if args.probe or args.probe_iters:
        probe_case(args)
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
