"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, bit for bit.

Integer state (spins, M and B after every sweep, the exact per-step sums) must be identical;
fp64 estimators derived from those sums agree to 1e-12 relative.  Sizes span several CTAs,
several 16-site chunks / 32-site words per row and ragged tails; the full-size workloads are
checked on sampled sweeps that the oracle recomputes one at a time from the GPU's own state.
"""
import numpy as np
import pytest

from paper_1205_5588_gb300 import workloads as W
from tests.gpu_common import (assert_records_equal, assert_same_run, gpu_lib, run_gpu, run_oracle)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def I():
    return gpu_lib()


def film(heights, layers, seed=1, init="random", **kw):
    d = {"heights": np.ascontiguousarray(heights, dtype=np.uint8), "layers": layers, "seed": seed, "init": init}
    d.update(kw)
    return d


def test_philox_device_matches_oracle(I):
    from oracle import oracle
    lib = oracle.load()
    rng = np.random.Generator(np.random.PCG64(99))
    for _ in range(40):
        seed = int(rng.integers(0, 2**64, dtype=np.uint64))
        stream = int(rng.integers(0, 3))
        sweep = int(rng.integers(0, 2**40))
        q0 = int(rng.integers(0, 2**32 - 600))
        got = I.philox_blocks(seed, stream, sweep, q0, 500)
        for b in range(0, 500, 7):
            want = oracle.philox([q0 + b, sweep & 0xFFFFFFFF, sweep >> 32, stream],
                                 [seed & 0xFFFFFFFF, seed >> 32], lib=lib)
            assert np.array_equal(got[b], want)


def test_flat16_hysteresis_full_run(I):
    """16x16x3 periodic film, T = 3, h = +4 -> -4 -> +4 by 0.1, 100 sweeps per step: every one
    of the 16,100 sweeps and all 161 step records bit-exact."""
    spec = W.flat16_hysteresis()
    sched = spec["schedule"]
    g = run_gpu(I, spec, sched)
    o = run_oracle(spec, sched)
    assert_same_run(g, o)
    assert g["info"]["n_occ"] == 768 and g["info"]["n_bonds"] == 3840


def test_fractal256_tscan_prefix(I):
    """256x256 fractal map, 1..6 layers, the T-scan's first steps at reduced sweep counts."""
    spec = W.fractal256_tscan()
    s = spec["schedule"]
    sched = W.schedule(s["T"][:3], s["h"][:3], 6, 8)
    assert_same_run(run_gpu(I, spec, sched), run_oracle(spec, sched))


def _spot_check(I, spec, sched, stops, packed=None):
    """Run the full schedule on the GPU, stopping at the given sweeps; at each stop the oracle
    takes the GPU's spins and sweep counter and computes the next sweep itself."""
    from oracle import oracle
    packed = spec.get("packed", False) if packed is None else packed
    lat = I.Lattice(spec["heights"], spec["layers"], packed=packed, seed=spec["seed"], init=spec["init"])
    total = int(sched["eq"].sum() + sched["meas"].sum())
    lat.enable_trace(total)
    lat.set_schedule(sched["T"], sched["h"], sched["eq"], sched["meas"])
    ends = np.cumsum(sched["eq"] + sched["meas"])
    init = {"random": oracle.INIT_RANDOM, "up": oracle.INIT_UP, "down": oracle.INIT_DOWN}[spec["init"]]
    of = oracle.Film(spec["heights"], spec["layers"], seed=spec["seed"], init=init)
    done = 0
    for t in stops:
        lat.run(t - done)
        before = lat.spins()
        lat.run(1)
        after = lat.spins()
        done = t + 1
        k = int(np.searchsorted(ends, t + 1))     # step holding sweep t+1
        of.set_spins(before)
        of.set_sweep(t)
        recs, ser = of.run([sched["T"][k]], [sched["h"][k]], [0], [1], series=True)
        assert np.array_equal(after, of.spins()), f"spins differ after sweep {t + 1}"
        tr = lat.trace()
        assert tuple(tr[t]) == tuple(ser[0]), (t, tr[t], ser[0])
    lat.run(-1)
    st = lat.state(recompute=True)
    assert st["M"] == st["M_full"] and st["B"] == st["B_full"]
    recs = lat.observables()
    tr = lat.trace()
    assert len(recs) == len(sched["T"])
    for k, r in enumerate(recs):
        assert r["M_last"] == tr[ends[k] - 1, 0] and r["B_last"] == tr[ends[k] - 1, 1]
        seg = tr[ends[k] - sched["meas"][k]: ends[k]]
        assert r["sumM"] == int(seg[:, 0].sum()) and r["sumB"] == int(seg[:, 1].sum())
        assert r["sumM2"] == sum(int(v) ** 2 for v in seg[:, 0])
    lat.close()


def test_fractal256_tscan_full_size_sampled(I):
    spec = W.fractal256_tscan()
    s = spec["schedule"]
    _spot_check(I, spec, s, stops=[0, 3999, 4000, 95999, 190000, 191998])


def test_fractal2048_hysteresis_full_size_sampled(I):
    spec = W.fractal2048_hysteresis()
    s = spec["schedule"]
    sched = W.schedule(s["T"][:4], s["h"][:4], s["eq"][:4], s["meas"][:4])
    _spot_check(I, spec, sched, stops=[0, 399, 799])


def test_packed_int8_oracle_agree_on_ragged_films(I):
    for (R, C, L, hurst, lo) in [(37, 77, 4, 0.6, 0), (64, 96, 5, 0.8, 1), (9, 130, 3, 0.7, 1), (50, 33, 8, 0.5, 0)]:
        spec = film(W.fractal_heights(R, C, hurst, lo, L, seed=R * C), L, seed=R + C)
        sched = W.schedule([1.5, 4.0, 9.0], [0.6, -0.3, 0.0], [3, 2, 0], [4, 5, 6])
        o = run_oracle(spec, sched)
        assert_same_run(run_gpu(I, spec, sched, packed=False), o)
        assert_same_run(run_gpu(I, spec, sched, packed=True), o)


def test_fractal2048_int8_and_packed_identical(I):
    spec = W.fractal2048_hysteresis()
    s = spec["schedule"]
    sched = W.schedule(s["T"][:2], s["h"][:2], 0, 25)
    a = run_gpu(I, spec, sched, packed=True, trace=True)
    b = run_gpu(I, spec, sched, packed=False, trace=True)
    assert np.array_equal(a["trace"], b["trace"])
    assert np.array_equal(a["spins"], b["spins"])
    assert_records_equal(a["recs"], b["recs"])


@pytest.mark.parametrize("packed,path,sites", [(False, "global", 0), (True, "global", 0), (False, "resident", 16),
                                               (False, "resident", 8)])
def test_launch_shape_does_not_change_the_trajectory(I, packed, path, sites):
    spec = film(W.fractal_heights(80, 120, 0.7, 1, 6, seed=5), 6, seed=11)
    sched = W.schedule([2.0, 6.0], [0.5, -0.5], [2, 2], [5, 5])
    ref = run_oracle(spec, sched)
    shapes = [(1, 256), (2, 64), (7, 128), (3, 32)] if path == "global" else \
             [(1, 512), (2, 256), (3, 128), (4, 512), (8, 64), (10, 96), (5, 0), (0, 0)]   # 40 colour rows
    if sites == 8:
        shapes += [(1, 768), (16, 0), (2, 736)]
    for launch in shapes:
        g = run_gpu(I, spec, sched, packed=packed, launch=launch, path=path, sites=sites)
        assert np.array_equal(g["trace"], ref["trace"]) and np.array_equal(g["spins"], ref["spins"]), launch
        if sites:
            assert g["launch"]["item_sites"] == sites


@pytest.mark.parametrize("h_s", [0.0, 3.0])
def test_packed_word_kernel_every_step_kind(I, h_s):
    """The packed multi-CTA kernel decides a step's lanes in two ways (the carry form when no
    threshold of the step is "never", the plain comparison otherwise, and always the plain one
    under the Eq. 9 gate) and draws a word's random blocks ahead (both halves when nearly every
    word needs them, else the second half lazily; words past the drawn-ahead slots in the pass).
    One schedule mixes all of them: T = 0.6 and 0.9 (never thresholds, lazy), T = 3, 1.4 and 2 with
    a strong field (carry, all drawn), T = inf (every flip "always": carry, lazy), T = 1.2 with
    h = 4 (never thresholds, all drawn); on launch shapes from 3 words per thread to less than
    one; bit-exact against the oracle."""
    spec = film(W.fractal_heights(64, 256, 0.7, 1, 3, seed=77), 3, seed=19)
    sched = W.schedule([0.6, 3.0, float("inf"), 1.4, 2.0, 0.9, 1.2], [0.5, -1.0, 0.0, 2.0, -6.0, 0.2, 4.0],
                       [1, 2, 0, 1, 0, 2, 1], [3, 3, 2, 4, 3, 2, 3])
    ref = run_oracle(spec, sched, h_s=h_s)
    for launch in [(4, 32), (3, 64), (8, 64), (2, 512), (0, 0)]:
        g = run_gpu(I, spec, sched, packed=True, launch=launch, path="global", h_s=h_s)
        assert_same_run(g, ref)
        if launch[0] > 1:
            assert g["launch"]["ctas"] == launch[0] and g["launch"]["path"] == "global", g["launch"]


@pytest.mark.parametrize("sites", [16, 8])
@pytest.mark.parametrize("name", ["flat16", "periodic_y_only", "periodic_x_only", "cube4", "ragged", "f256_prefix",
                                  "ragged_x9"])
def test_resident_path_matches_oracle(I, name, sites):
    sched = W.schedule([2.0, 8.0, 5.0], [1.0, 0.0, -1.0], [1, 1, 1], [4, 4, 4])
    if name == "flat16":
        spec = W.flat16_hysteresis()
        sched = W.schedule(3.0, spec["schedule"]["h"][:30], 0, 20)
    elif name == "periodic_y_only":
        spec = film(np.full((12, 9), 3), 3, seed=4, periodic_y=True)
    elif name == "periodic_x_only":
        spec = film(W.fractal_heights(9, 36, 0.7, 1, 4, seed=3), 4, seed=8, periodic_x=True)
    elif name == "cube4":
        spec = film(np.full((4, 4), 4), 4, seed=6, periodic_x=True, periodic_y=True, periodic_z=True)
    elif name == "ragged":
        spec = film(W.fractal_heights(45, 83, 0.6, 0, 5, seed=10), 5, seed=12)
    elif name == "ragged_x9":
        # 9 columns per colour row: an 8-site item and a 1-site one, periodic columns
        spec = film(W.fractal_heights(10, 18, 0.6, 1, 3, seed=15), 3, seed=16, periodic_x=True)
    else:
        spec = W.fractal256_tscan()
        s = spec["schedule"]
        sched = W.schedule(s["T"][:3], s["h"][:3], 6, 8)
    o = run_oracle(spec, sched)
    # cluster sizes the film fits: the 256x256x6 film needs at least 4 CTAs of shared memory
    launches = ([0, 0], [4, 0], [8, 512], [16, 256]) if name == "f256_prefix" else ([0, 0], [1, 0], [2, 0], [3, 64])
    for launch in launches:
        if launch[0] > (spec["heights"].shape[0] + 1) // 2:
            continue
        g = run_gpu(I, spec, sched, launch=tuple(launch), path="resident", sites=sites)
        assert g["launch"]["item_sites"] == sites
        assert_same_run(g, o)


@pytest.mark.parametrize("sites", [16, 8])
def test_resident_gate_parity(I, sites):
    spec = film(W.fractal_heights(30, 70, 0.7, 1, 4, seed=9), 4, seed=5)
    sched = W.schedule([2.0, 4.0, 6.0], [2.0, -2.0, 0.5], [2, 2, 2], [4, 4, 4])
    o = run_oracle(spec, sched, h_s=4.0)
    assert_same_run(run_gpu(I, spec, sched, h_s=4.0, path="resident", sites=sites), o)


def test_paths_interleave(I):
    """Launches of the resident and the global kernel on one film continue each other."""
    spec = film(W.fractal_heights(64, 96, 0.7, 1, 5, seed=13), 5, seed=14)
    sched = W.schedule([2.0, 3.0, 4.0], [0.3, 0.0, -0.3], [3, 3, 3], [5, 5, 5])
    o = run_oracle(spec, sched)
    lat = I.Lattice(spec["heights"], 5, seed=14)
    lat.enable_trace(24)
    lat.set_schedule(sched["T"], sched["h"], sched["eq"], sched["meas"])
    for n, path in ((5, "resident"), (4, "global"), (7, "resident"), (8, "global")):
        lat.set_path(path)
        lat.run(n)
    assert np.array_equal(lat.trace(), o["trace"])
    assert np.array_equal(lat.spins(), o["spins"])
    assert_records_equal(lat.observables(), o["recs"])
    lat.close()


def test_chunked_runs_equal_one_run(I):
    spec = film(W.fractal_heights(40, 52, 0.7, 1, 4, seed=6), 4, seed=3)
    sched = W.schedule([3.0, 2.0, 5.0], [0.0, 0.7, -0.7], [5, 0, 3], [6, 9, 4])
    o = run_oracle(spec, sched)
    for chunks in ([1, 1, 1], [7, 3, 11], [20]):      # 27 sweeps in all
        assert_same_run(run_gpu(I, spec, sched, chunks=chunks), o)


@pytest.mark.parametrize("case", ["single_site", "all_vacant", "one_row", "thin_column", "tall_sparse",
                                  "infinite_T", "zero_T", "down_start"])
def test_edge_films(I, case):
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
    elif case == "infinite_T":
        spec = film(W.fractal_heights(20, 24, 0.7, 1, 3, seed=1), 3)
        sched = W.schedule([float("inf")] * 2, [0.0, 2.0], 0, 5)
    elif case == "zero_T":
        spec = film(W.fractal_heights(20, 24, 0.7, 1, 3, seed=1), 3)
        sched = W.schedule([0.0, 0.0], [0.0, 1.0], 0, 5)
    else:
        spec = film(W.fractal_heights(17, 29, 0.7, 0, 4, seed=2), 4, init="down")
    o = run_oracle(spec, sched)
    for packed in (False, True):
        assert_same_run(run_gpu(I, spec, sched, packed=packed), o)


@pytest.mark.parametrize("shape", [(4, 4, 2, (True, True, False)), (6, 8, 3, (True, False, False)),
                                   (8, 6, 3, (False, True, False)), (4, 4, 4, (True, True, True)),
                                   (10, 12, 2, (True, True, False))])
def test_periodic_films(I, shape):
    R, C, L, (px, py, pz) = shape
    spec = film(np.full((R, C), L), L, seed=R * 7 + C, periodic_x=px, periodic_y=py, periodic_z=pz)
    sched = W.schedule([2.0, 8.0, 5.0], [1.0, 0.0, -1.0], [1, 1, 1], [4, 4, 4])
    assert_same_run(run_gpu(I, spec, sched), run_oracle(spec, sched))


@pytest.mark.parametrize("packed,periodic", [(False, False), (True, False), (False, True)])
def test_switching_gate_parity(I, packed, periodic):
    if periodic:
        spec = film(np.full((8, 8), 3), 3, periodic_x=True, periodic_y=True)
    else:
        spec = film(W.fractal_heights(30, 70, 0.7, 1, 4, seed=9), 4, seed=5)
    sched = W.schedule([2.0, 4.0, 6.0], [2.0, -2.0, 0.5], [2, 2, 2], [4, 4, 4])
    o = run_oracle(spec, sched, h_s=4.0)
    assert_same_run(run_gpu(I, spec, sched, packed=packed, h_s=4.0), o)


def test_write_spins_resume_and_save_load(I, tmp_path):
    spec = film(W.fractal_heights(24, 40, 0.7, 1, 4, seed=8), 4, seed=21)
    sched = W.schedule([2.0, 3.0], [0.4, -0.4], [0, 0], [6, 7])
    full = run_gpu(I, spec, sched, trace=False)
    lat = I.Lattice(spec["heights"], 4, seed=21)
    lat.set_schedule(sched["T"][:1], sched["h"][:1], [0], [6])
    lat.run(-1)
    path = tmp_path / "film.isf"
    lat.save(path)
    lat.close()
    lat2 = I.Lattice.load(path)
    assert lat2.info()["sweep"] == 6
    lat2.set_schedule(sched["T"][1:], sched["h"][1:], [0], [7])
    lat2.run(-1)
    assert np.array_equal(lat2.spins(), full["spins"])
    assert lat2.observables()[0]["sumM"] == full["recs"][1]["sumM"]
    lat2.close()


def test_errors_are_reported(I):
    lat = I.Lattice(np.full((6, 6), 2), 2)
    with pytest.raises(I.IsfError) as e:
        lat.run(1)
    assert e.value.code == -7
    lat.set_schedule([2.0], [0.0], [0], [3])
    with pytest.raises(I.IsfError) as e:
        lat.run(4)
    assert e.value.code == -5
    with pytest.raises(I.IsfError) as e:
        lat.write_spins(np.full((2, 6, 6), 3, dtype=np.int8), 0)
    assert e.value.code == -1
    with pytest.raises(I.IsfError) as e:
        lat.set_schedule([2.0], [0.0], [0], [0])
    assert e.value.code == -5
    for bad in (4, 12, 32, -8):
        with pytest.raises(I.IsfError) as e:
            lat.set_item_sites(bad)
        assert e.value.code == -1
    lat.close()


def test_runs_on_a_side_stream(I):
    import torch
    spec = film(W.fractal_heights(32, 48, 0.7, 1, 3, seed=3), 3, seed=2)
    sched = W.schedule([2.0], [0.1], [2], [5])
    s = torch.cuda.Stream()
    lat = I.Lattice(spec["heights"], 3, seed=2, stream=s)
    lat.set_schedule(sched["T"], sched["h"], sched["eq"], sched["meas"])
    lat.run(-1, stream=s)
    assert_records_equal(lat.observables(), run_oracle(spec, sched)["recs"])
    lat.close()


@pytest.mark.parametrize("packed", [False, True])
def test_surface_image_and_stats_match_oracle(I, packed):
    """PMOKE frames (Sec. 6) along a hysteresis loop and the Table 1 statistics (Sec. 4)."""
    from oracle import oracle
    spec = film(W.fractal_heights(37, 61, 0.7, 0, 4, seed=17), 4, seed=23)
    lat = I.Lattice(spec["heights"], 4, seed=23, packed=packed)
    of = oracle.Film(spec["heights"], 4, seed=23)
    h = W.loop_fields(8, 4)
    lat.set_schedule(np.full(len(h), 2.5), h, np.zeros(len(h), np.int32), np.full(len(h), 3, np.int32))
    for k in range(len(h)):
        lat.run(3)
        of.run([2.5], [h[k]], [0], [3])
        img = lat.surface_image()
        oimg = of.surface_image()
        assert np.array_equal(img, oimg), k
        assert lat.surface_domains() == oracle.domain_stats(oimg), k
    st = lat.stats()
    info = of.info()
    assert st["zbar"] == 2 * info["n_bonds"] / info["n_occ"]
    assert st["p_c"] == 2.0 / st["zbar"]
    assert st["p"] == info["n_occ"] / (37 * 61 * 4)
    lat.close()


def test_curie_estimate_of_a_scan(I):
    """T_c of a scan (Sec. 4, Table 1): isf_estimate_tc on the GPU's records picks the same step
    as the oracle's or_estimate_tc on the oracle's records of the same scan (the records are
    identical), and the susceptibility peak of a thick periodic film sits below the bulk FCC T_c."""
    from oracle import oracle
    spec = film(np.full((16, 16), 8), 8, seed=3, periodic_x=True, periodic_y=True)
    T = np.linspace(6.0, 12.0, 13)
    lat = I.Lattice(spec["heights"], 8, seed=3, periodic_x=True, periodic_y=True)
    sc = W.schedule(T, 0.0, 300, 600)
    lat.set_schedule(sc["T"], sc["h"], sc["eq"], sc["meas"])
    lat.run(-1)
    recs = lat.observables()
    lat.close()
    tc, k = I.estimate_tc(recs, with_index=True)
    of = oracle.Film(spec["heights"], 8, flags=3, seed=3)
    orecs, _ = of.run(sc["T"], sc["h"], sc["eq"], sc["meas"])
    of.close()
    assert (tc, k) == oracle.estimate_tc(orecs)
    assert 7.0 <= tc <= 10.0


def test_curie_estimate_of_the_fractal_scan(I):
    """The same on a fractal int8 film (open edges, 1..4 layers), a scan like the 256^2 workload's
    at reduced size: GPU and oracle pick the same temperature."""
    from oracle import oracle
    H = W.fractal_heights(40, 44, 0.7, 1, 4, seed=2)
    T = np.array([0.5 + k * 11.5 / 23.0 for k in range(24)])
    sc = W.schedule(T, 0.0, 60, 120)
    lat = I.Lattice(H, 4, seed=1)
    lat.set_schedule(sc["T"], sc["h"], sc["eq"], sc["meas"])
    lat.run(-1)
    recs = lat.observables()
    lat.close()
    of = oracle.Film(H, 4, seed=1)
    orecs, _ = of.run(sc["T"], sc["h"], sc["eq"], sc["meas"])
    of.close()
    assert I.estimate_tc(recs, with_index=True) == oracle.estimate_tc(orecs)


@pytest.mark.parametrize("shape,periodic", [((64, 96), False), ((48, 48), True), ((300, 257), False)])
def test_surface_domains_match_oracle(I, shape, periodic):
    """Domain counts and largest domains of the PMOKE image (Sec. 6, Fig. 5) on films with many
    domains: a high-temperature state on open and periodic films, and a large open film."""
    from oracle import oracle
    R, C = shape
    if periodic:
        spec = film(np.full((R, C), 2), 2, seed=5, periodic_x=True, periodic_y=True)
    else:
        spec = film(W.fractal_heights(R, C, 0.6, 0, 3, seed=R + C), 3, seed=9)
    lat = I.Lattice(spec["heights"], spec["layers"], seed=spec["seed"], periodic_x=periodic, periodic_y=periodic)
    of = oracle.Film(spec["heights"], spec["layers"], flags=3 if periodic else 0, seed=spec["seed"])
    lat.set_schedule([6.0, 3.0], [0.0, 0.2], [0, 0], [2, 2])
    lat.run(-1)
    of.run([6.0, 3.0], [0.0, 0.2], [0, 0], [2, 2])
    oimg = of.surface_image()
    assert np.array_equal(lat.surface_image(), oimg)
    want = oracle.domain_stats(oimg, periodic_x=periodic, periodic_y=periodic)
    assert want["white"] > 3 and want["black"] > 3
    assert lat.surface_domains() == want
    lat.close()
