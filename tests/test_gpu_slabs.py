"""The row-slab kernel (packed films split by rows over the CTAs, each band of rows in shared
memory, boundary rows exchanged between neighbouring CTAs after every colour pass): the same
trajectory as the oracle, bit for bit, on ragged films, bands of one, two and many rows, forced
CTA counts and block sizes, the Eq. 9 gate, runs longer than one launch, runs interleaved with
the global kernel, the full-size 2048 x 2048 film against the global kernel, and edge films."""
import numpy as np
import pytest

from paper_1205_5588_gb300 import workloads as W
from tests.gpu_common import assert_records_equal, assert_same_run, gpu_lib, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def I():
    return gpu_lib()


def film(heights, layers, seed=1, init="random"):
    return {"heights": np.asarray(heights, dtype=np.uint8), "layers": layers, "seed": seed, "init": init,
            "packed": True}


SCHED = W.schedule([1.5, 4.0, 9.0], [0.6, -0.3, 0.0], [3, 2, 0], [4, 5, 6])


@pytest.mark.parametrize("shape", [(37, 77, 4, 0.6, 0), (9, 130, 3, 0.7, 1), (50, 33, 8, 0.5, 0),
                                   (620, 100, 4, 0.7, 1), (1300, 70, 3, 0.8, 1)])
def test_slabs_match_oracle(I, shape):
    R, C, L, hurst, lo = shape
    spec = film(W.fractal_heights(R, C, hurst, lo, L, seed=R + 3 * C), L, seed=R * C)
    o = run_oracle(spec, SCHED)
    g = run_gpu(I, spec, SCHED, path="slabs")
    assert g["launch"]["path"] == "slabs" and g["launch"]["item_sites"] == 32
    assert_same_run(g, o)


@pytest.mark.parametrize("launch", [(1, 512), (2, 64), (7, 256), (13, 96), (40, 0), (0, 128)])
def test_slab_launch_shapes(I, launch):
    """Bands of 1 to 40 rows (one CTA: no neighbours; 40 CTAs of 80 colour rows: two each)."""
    spec = film(W.fractal_heights(160, 90, 0.7, 1, 5, seed=31), 5, seed=8)
    o = run_oracle(spec, SCHED)
    g = run_gpu(I, spec, SCHED, path="slabs", launch=launch)
    if launch[0]:
        assert g["launch"]["ctas"] == launch[0]
    assert_same_run(g, o)


def test_slab_gate_parity(I):
    spec = film(W.fractal_heights(300, 70, 0.7, 1, 4, seed=9), 4, seed=5)
    sched = W.schedule([2.0, 4.0, 6.0], [2.0, -2.0, 0.5], [2, 2, 2], [4, 4, 4])
    o = run_oracle(spec, sched, h_s=4.0)
    assert_same_run(run_gpu(I, spec, sched, h_s=4.0, path="slabs"), o)


def test_slab_runs_longer_than_one_launch(I):
    """4100 sweeps: three launches (2048 + 2048 + 4), each folded after it; and a run cut in odd
    chunks."""
    spec = film(W.fractal_heights(16, 40, 0.7, 1, 2, seed=2), 2, seed=6)
    sched = W.schedule([2.5, 3.5, 1.0], [0.4, -0.4, 0.0], [50, 0, 10], [2000, 2030, 10])
    o = run_oracle(spec, sched)
    assert_same_run(run_gpu(I, spec, sched, path="slabs"), o)
    assert_same_run(run_gpu(I, spec, sched, path="slabs", chunks=[1, 2047, 2049, 3]), o)


def test_slabs_and_global_interleave(I):
    spec = film(W.fractal_heights(64, 96, 0.7, 1, 5, seed=13), 5, seed=14)
    sched = W.schedule([2.0, 3.0, 4.0], [0.3, 0.0, -0.3], [3, 3, 3], [5, 5, 5])
    o = run_oracle(spec, sched)
    lat = I.Lattice(spec["heights"], 5, seed=14, packed=True)
    lat.enable_trace(24)
    lat.set_schedule(sched["T"], sched["h"], sched["eq"], sched["meas"])
    for n, path in ((5, "slabs"), (4, "global"), (7, "slabs"), (8, "global")):
        lat.set_path(path)
        lat.run(n)
    assert np.array_equal(lat.trace(), o["trace"])
    assert np.array_equal(lat.spins(), o["spins"])
    assert_records_equal(lat.observables(), o["recs"])
    lat.close()


@pytest.mark.parametrize("case", ["single_site", "all_vacant", "one_row", "thin_column", "tall_sparse", "down_start"])
def test_slab_edge_films(I, case):
    sched = W.schedule([2.5, 3.5], [0.3, -0.3], [1, 0], [3, 4])
    if case == "single_site":
        spec = film(np.ones((1, 1)), 1)
    elif case == "all_vacant":
        spec = film(np.zeros((5, 7)), 3)
    elif case == "one_row":
        spec = film(np.full((1, 45), 2), 2)
    elif case == "thin_column":
        spec = film(np.full((31, 1), 3), 3)
    elif case == "tall_sparse":
        rng = np.random.Generator(np.random.PCG64(4))
        spec = film(rng.integers(0, 9, size=(23, 19)), 8)
    else:
        spec = film(W.fractal_heights(17, 29, 0.7, 0, 4, seed=2), 4, init="down")
    assert_same_run(run_gpu(I, spec, sched, path="slabs"), run_oracle(spec, sched))


def test_fractal2048_slabs_equal_global(I):
    spec = W.fractal2048_hysteresis()
    s = spec["schedule"]
    sched = W.schedule(s["T"][:3], s["h"][:3], 0, 20)
    a = run_gpu(I, spec, sched, path="slabs")
    b = run_gpu(I, spec, sched, path="global")
    assert a["launch"]["path"] == "slabs"
    assert np.array_equal(a["trace"], b["trace"])
    assert np.array_equal(a["spins"], b["spins"])
    assert_records_equal(a["recs"], b["recs"])


@pytest.mark.parametrize("R,L,want", [(16, 3, "global"), (256, 6, "slabs"), (512, 6, "global"), (768, 6, "global"),
                                      (2048, 6, "global")])
def test_automatic_path_choice(I, R, L, want):
    """Packed films: the row-slab kernel while a colour pass has 513 to 4096 words (about 150^2 to
    350^2 sites per layer), where it is the faster one; the word kernel on global memory for
    smaller films (one CTA) and larger ones."""
    H = W.fractal_heights(R, R, 0.8, 2, L, seed=3)
    lat = I.Lattice(H, L, seed=1, init="up", packed=True)
    lat.set_schedule([2.0], [0.0], [0], [1])
    lat.run(-1)
    assert lat.launch_info()["path"] == want
    lat.close()


def test_slab_layer_limit(I):
    """16 layers run on the row-slab kernel; 17 are refused there, and the automatic choice then
    takes the global kernel."""
    sched = W.schedule([3.0, 5.0], [0.5, -0.5], [1, 1], [3, 3])
    spec = film(W.fractal_heights(40, 64, 0.7, 4, 16, seed=12), 16, seed=3)
    assert_same_run(run_gpu(I, spec, sched, path="slabs"), run_oracle(spec, sched))
    H = W.fractal_heights(300, 300, 0.7, 4, 17, seed=13)
    lat = I.Lattice(H, 17, packed=True)
    with pytest.raises(I.IsfError) as e:
        lat.set_path("slabs")
    assert e.value.code == -1
    lat.set_schedule([3.0], [0.0], [0], [1])
    lat.run(-1)
    assert lat.launch_info()["path"] == "global"
    lat.close()


def test_slab_path_errors(I):
    H = W.fractal_heights(12, 10, 0.7, 1, 3, seed=2)
    lat = I.Lattice(H, 3)                                    # int8
    with pytest.raises(I.IsfError) as e:
        lat.set_path("slabs")
    assert e.value.code == -1
    lat.close()
    lat = I.Lattice(H, 3, packed=True)
    lat.set_path("slabs")
    lat.set_schedule([2.0], [0.0], [0], [2])
    lat.set_launch(7, 0)                                     # more CTAs than the film's 6 colour rows
    with pytest.raises(I.IsfError) as e:
        lat.run(1)
    assert e.value.code == -1
    lat.set_launch(0, 0)
    lat.run(-1)
    lat.close()
