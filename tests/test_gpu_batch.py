"""Batched films on the GPU: every film of a mixed batch (single-CTA and cluster resident films,
one-CTA and one-cluster global-memory films; int8 and packed, open and periodic, different seeds
and schedules) ends exactly where the oracle and where the film run alone end, with and without
graph replay and autotuning."""
import numpy as np
import pytest

from paper_1205_5588_gb300 import workloads as W
from tests.gpu_common import assert_records_equal, gpu_lib, oracle_flags, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def I():
    return gpu_lib()


def mixed_films():
    rng = np.random.Generator(np.random.PCG64(77))
    films = []
    shapes = [(40, 52, 3, {}), (64, 64, 2, {}), (17, 23, 5, {}), (96, 130, 4, {}),
              (200, 256, 4, {}),                     # needs a cluster
              (150, 310, 5, {}),                     # needs a cluster
              (48, 64, 3, {"packed": True}),         # global memory: one CTA or a cluster by its share of the work
              (16, 16, 3, {"periodic_x": True, "periodic_y": True}),   # one CTA, global memory (a tiny share)
              (8, 12, 2, {}), (33, 65, 6, {}),
              (96, 200, 5, {"packed": True}),        # global memory: one CTA or a cluster by its share of the work
              (512, 1024, 3, {"packed": True, "short": True}),   # over 2^20 sites: a cluster, global memory
              (2000, 2000, 1, {"short": True})]      # int8, too large for a cluster's shared memory
    for i, (R, Cc, L, extra) in enumerate(shapes):
        if extra.get("periodic_x"):
            H = np.full((R, Cc), L, dtype=np.uint8)
        else:
            H = W.fractal_heights(R, Cc, float(rng.uniform(0.5, 0.9)), 1, L, seed=500 + i)
        nst = int(rng.integers(2, 5))
        T = rng.uniform(1.0, 8.0, size=nst)
        h = rng.uniform(-2.0, 2.0, size=nst)
        eq = rng.integers(0, 3, size=nst)
        me = rng.integers(2, 7, size=nst)
        if extra.pop("short", False):       # keep the oracle's share of the test short
            eq, me = np.zeros(nst, dtype=int), np.full(nst, 2)
        f = {"heights": H, "layers": L, "seed": 900 + i, "init": "random", "schedule": W.schedule(T, h, eq, me)}
        f.update(extra)
        films.append(f)
    return films


def make(I, f):
    lat = I.Lattice(f["heights"], f["layers"], seed=f["seed"], init=f["init"], packed=f.get("packed", False),
                    periodic_x=f.get("periodic_x", False), periodic_y=f.get("periodic_y", False))
    s = f["schedule"]
    lat.set_schedule(s["T"], s["h"], s["eq"], s["meas"])
    return lat


@pytest.mark.parametrize("graph,tune", [(False, False), (True, False), (False, True)])
def test_batch_matches_oracle_and_solo(I, graph, tune):
    films = mixed_films()
    lats = [make(I, f) for f in films]
    b = I.Batch(lats, graph=graph)
    if tune:
        b.tune()
    b.run()
    info = b.info()
    # the batch has films for the cluster global-memory kernel, so the two films that fit a
    # cluster's shared memory join its queue (the resident cluster kernel is covered by
    # test_batch_launch_shapes, whose films fit)
    assert info["single_cta_films"] >= 5 and info["cluster_films"] == 0, info
    # a global-memory film takes one CTA only if its work is at most an even share of the batch's
    # per CTA (here the two largest films hold most of the work): one CTA or a cluster each
    assert info["global_cta_films"] >= 1 and info["global_cta_films"] + info["global_cluster_films"] == 7, info
    for f, lat in zip(films, lats):
        o = run_oracle(f, f["schedule"])
        assert_records_equal(lat.observables(), o["recs"])
        assert np.array_equal(lat.spins(), o["spins"])
        st = lat.state(recompute=True)
        assert st["M"] == st["M_full"] and st["B"] == st["B_full"]
    # replay: new schedules for every film, same batch (graph replay when enabled)
    for f, lat in zip(films, lats):
        s = f["schedule"]
        lat.set_schedule(s["T"][::-1].copy(), s["h"], s["eq"], s["meas"])
    b.run()
    for f, lat in zip(films, lats):
        solo = make(I, f)
        solo.run(-1)
        s = f["schedule"]
        solo.set_schedule(s["T"][::-1].copy(), s["h"], s["eq"], s["meas"])
        solo.run(-1)
        assert_records_equal(lat.observables(), solo.observables())
        assert np.array_equal(lat.spins(), solo.spins())
        solo.close()
    b.close()
    for lat in lats:
        lat.close()


def test_global_kernel_takes_waiting_resident_films(I):
    """More single-CTA resident films than the resident kernel holds at once, beside one tiny
    global-memory film: the one-CTA global-memory kernel, done with its own film, takes resident
    films that have not started and runs them in global memory; every film ends exactly where it
    ends alone."""
    rng = np.random.Generator(np.random.PCG64(78))
    films = []
    for i in range(800):
        H = W.fractal_heights(16, 16, 0.7, 1, 2, seed=3000 + i)
        sc = W.schedule(rng.uniform(1.0, 8.0, size=2), rng.uniform(-2.0, 2.0, size=2), [0, 0], [20, 20])
        films.append({"heights": H, "layers": 2, "seed": 5000 + i, "init": "random", "schedule": sc})
    films.append({"heights": np.full((16, 16), 2, dtype=np.uint8), "layers": 2, "seed": 77, "init": "random",
                  "packed": True, "schedule": W.schedule([3.0], [0.0], [0], [1])})
    lats = [make(I, f) for f in films]
    b = I.Batch(lats)
    b.run()
    info, taken = b.info(), b.taken()
    assert info["single_cta_films"] == 800 and info["global_cta_films"] == 1, info
    assert info["ctas"] < 800, info          # films wait for a resident CTA
    assert taken["single_cta"] > 0 and taken["cluster"] == 0, taken
    for f, lat in zip(films, lats):
        solo = make(I, f)
        solo.run(-1)
        assert_records_equal(lat.observables(), solo.observables())
        assert np.array_equal(lat.spins(), solo.spins())
        solo.close()
    b.close()
    for lat in lats:
        lat.close()


def test_batch_of_one_and_empty(I):
    f = mixed_films()[0]
    lat = make(I, f)
    b = I.Batch([lat])
    b.run()
    b.run()            # nothing left: a no-op
    assert_records_equal(lat.observables(), run_oracle(f, f["schedule"])["recs"])
    b.clear()
    b.run()
    b.close()
    lat.close()


@pytest.mark.parametrize("shape", [(64, 8, 64), (512, 16, 96), (160, 2, 512)])
def test_batch_launch_shapes(I, shape):
    """Explicit launch shapes, down to one site-taking warp next to the folding warp; no film
    needs the cluster global-memory kernel, so the two large films run cluster-resident."""
    films = mixed_films()[:6]
    lats = [make(I, f) for f in films]
    b = I.Batch(lats)
    b.set_launch(*shape)
    b.run()
    assert b.info()["cluster_films"] == 2 and b.info()["global_cluster_films"] == 0, b.info()
    for f, lat in zip(films, lats):
        o = run_oracle(f, f["schedule"])
        assert_records_equal(lat.observables(), o["recs"])
        assert np.array_equal(lat.spins(), o["spins"])
    b.close()
    for lat in lats:
        lat.close()


def test_batch_launch_shape_errors(I):
    b = I.Batch([])
    for bad in ((32, 0, 0), (0, 8, 32), (544, 0, 0), (0, 17, 0), (70, 0, 0)):
        with pytest.raises(I.IsfError) as e:
            b.set_launch(*bad)
        assert e.value.code == -1
    b.close()
