"""Serving: jobs submitted at any time are admitted by device memory, run overlapped with the
jobs already on the GPU, and each result equals the same job run alone (bit for bit)."""
import time

import numpy as np
import pytest

from paper_1205_5588_gb300 import workloads as W
from tests.gpu_common import assert_records_equal, gpu_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def I():
    return gpu_lib()


def jobs():
    rng = np.random.Generator(np.random.PCG64(5))
    out = []
    for i in range(10):
        side = W.lognormal_side(rng, median=96, sigma=0.6, lo=24, hi=300)
        L = int(rng.integers(1, 7))
        H = W.fractal_heights(side, int(side * rng.uniform(0.7, 1.3)), 0.7, 1, L, seed=700 + i)
        if i % 2:      # hysteresis loop
            h = W.loop_fields(int(rng.integers(4, 9)), 4)
            sched = W.schedule(float(rng.uniform(1.5, 6.0)), h, 0, 3)
        else:          # temperature scan
            sched = W.schedule(np.linspace(1.0, 9.0, 6), 0.0, 4, 4)
        out.append({"heights": H, "layers": L, "seed": 40 + i, "schedule": sched, "packed": i % 3 == 0})
    return out


def solo(I, j):
    lat = I.Lattice(j["heights"], j["layers"], seed=j["seed"], packed=j["packed"])
    s = j["schedule"]
    lat.set_schedule(s["T"], s["h"], s["eq"], s["meas"])
    lat.run(-1)
    r = lat.observables()
    lat.close()
    return r


def test_served_results_equal_solo_runs(I):
    js = jobs()
    one = max(I.lattice_bytes(j["heights"].shape[0], j["heights"].shape[1], j["layers"], 8 if j["packed"] else 0)
              for j in js)
    budget = 3 * one + 3 * 4096 * 4
    srv = I.Server(budget, sweeps_per_tick=5)
    ids = []
    for k, j in enumerate(js):
        s = j["schedule"]
        ids.append(srv.submit(j["heights"], j["layers"], s["T"], s["h"], s["eq"], s["meas"], seed=j["seed"],
                              packed=j["packed"]))
        if k == 4:
            time.sleep(0.05)          # later jobs arrive while the first ones run
    for jid in ids:
        assert srv.wait(jid, timeout=120) == "done"
    for j, jid in zip(js, ids):
        state, recs, latency = srv.result(jid)
        assert state == "done" and latency > 0
        assert_records_equal(recs, solo(I, j))
        srv.release(jid)
    st = srv.stats()
    assert st["completed"] == len(js) and st["failed"] == 0
    assert st["peak_bytes"] <= budget
    assert st["ticks"] > 1
    srv.close()


def test_served_jobs_overlap_on_the_device(I):
    """Continuous batching, not a queue: a job submitted while another is on the GPU is admitted
    into the running ticks, so the two films are advanced by the same batched launches (their
    tick ranges intersect), and each still ends with its solo result."""
    rng = np.random.Generator(np.random.PCG64(8))
    mk = lambda side, L, s: W.fractal_heights(side, side, 0.7, 1, L, seed=s)
    long_job = {"heights": mk(160, 4, 81), "layers": 4, "seed": 81, "packed": True,
                "schedule": W.schedule(2.5, W.loop_fields(8, 4), 0, 40)}
    late_jobs = [{"heights": mk(int(rng.integers(40, 90)), 3, 90 + i), "layers": 3, "seed": 90 + i,
                  "packed": bool(i % 2), "schedule": W.schedule([3.0, 5.0], [0.5, -0.5], 2, 6)} for i in range(4)]
    srv = I.Server(1 << 30, sweeps_per_tick=4)
    s = long_job["schedule"]
    first = srv.submit(long_job["heights"], 4, s["T"], s["h"], s["eq"], s["meas"], seed=81, packed=True)
    t0 = time.time()
    while srv.job_ticks(first)["count"] < 2 and time.time() - t0 < 60:
        time.sleep(0.002)                       # the long job is running
    assert srv.job_ticks(first)["count"] >= 2
    late = []
    for j in late_jobs:
        sj = j["schedule"]
        late.append(srv.submit(j["heights"], j["layers"], sj["T"], sj["h"], sj["eq"], sj["meas"], seed=j["seed"],
                               packed=j["packed"]))
    for jid in [first] + late:
        assert srv.wait(jid, timeout=120) == "done"
    tf = srv.job_ticks(first)
    overlapped = 0
    for jid, j in zip(late, late_jobs):
        tl = srv.job_ticks(jid)
        assert tl["first"] > tf["first"]                      # admitted after the long job started
        if tl["first"] <= tf["last"]:                         # ... and advanced in the same launches
            overlapped += 1
        assert_records_equal(srv.result(jid)[1], solo(I, j))
        srv.release(jid)
    assert overlapped >= 1
    assert_records_equal(srv.result(first)[1], solo(I, long_job))
    srv.close()


def test_job_larger_than_budget_fails(I):
    srv = I.Server(1 << 14, sweeps_per_tick=10)        # the film needs about 57 KB
    H = np.full((64, 64), 4, dtype=np.uint8)
    jid = srv.submit(H, 4, [2.0], [0.0], [1], [1])
    assert srv.wait(jid, timeout=30) == "failed"
    with pytest.raises(I.IsfError) as e:
        srv.result(jid)
    assert e.value.code == -2
    srv.close()
