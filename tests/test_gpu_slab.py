"""Row slabs of one film on the GPU: the film split into 1, 2 or 3 slabs (emulated ranks in one
process, halos copied on the device after every colour pass) follows the oracle's trajectory of
the whole film exactly: per-sweep M and B, step records and final spins; int8 and packed, open
and periodic in y, with the Eq. 9 gate off."""
import numpy as np
import pytest

from paper_1205_5588_gb300 import slab as S
from paper_1205_5588_gb300 import workloads as W
from tests.gpu_common import assert_records_equal, gpu_lib, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def I():
    return gpu_lib()


CASES = {
    "fractal_open": (lambda: W.fractal_heights(22, 30, 0.7, 1, 4, seed=21), 4, {}),
    "fractal_odd_rows": (lambda: W.fractal_heights(23, 17, 0.6, 0, 3, seed=22), 3, {}),
    "flat_periodic": (lambda: np.full((12, 16), 3, dtype=np.uint8), 3, {"periodic_x": True, "periodic_y": True}),
    "fractal_packed": (lambda: W.fractal_heights(26, 70, 0.7, 1, 5, seed=23), 5, {"packed": True}),
}


@pytest.mark.parametrize("world", [1, 2, 3])
@pytest.mark.parametrize("case", list(CASES))
def test_slabs_follow_the_whole_film(I, case, world):
    make_h, L, extra = CASES[case]
    H = make_h()
    sched = W.schedule([2.0, 6.0, 3.5], [0.4, -0.2, 0.0], [1, 0, 2], [3, 4, 2])
    spec = {"heights": H, "layers": L, "seed": 31, "init": "random", "J": 1.0,
            "periodic_x": extra.get("periodic_x", False), "periodic_y": extra.get("periodic_y", False),
            "packed": extra.get("packed", False)}
    o = run_oracle(spec, sched)
    run, slabs = S.run_local(H, L, sched, world, seed=31, **extra)
    try:
        assert np.array_equal(np.stack([run.M, run.B], axis=1), o["trace"])
        assert_records_equal(run.records, o["recs"])
        assert np.array_equal(S.whole_spins(slabs, H.shape[0]), o["spins"])
        assert run.n_occ == o["info"]["n_occ"]
    finally:
        for s in slabs:
            s.close()


def test_slab_errors(I):
    H = W.fractal_heights(12, 10, 0.7, 1, 3, seed=2)
    for y0, y1 in ((1, 6), (0, 1), (4, 4), (0, 13), (-2, 4), (2, 7)):
        with pytest.raises(I.IsfError) as e:
            I.Lattice.slab(H, 3, y0, y1)
        assert e.value.code == -1
    lat = I.Lattice.slab(H, 3, 0, 6)
    lat.set_schedule([2.0], [0.0], [0], [2])
    with pytest.raises(I.IsfError) as e:
        lat.run(1)                                   # slabs advance by colour passes
    assert e.value.code == -7
    with pytest.raises(I.IsfError) as e:
        lat.run_pass(1)                              # out of order
    assert e.value.code == -7
    import torch
    buf = torch.empty(lat.slab_info()["halo_bytes"], dtype=torch.uint8, device="cuda")
    with pytest.raises(I.IsfError) as e:
        lat.slab_import(0, 0, buf.data_ptr())        # no halo below the film's open edge
    assert e.value.code == -1
    for c in range(4):
        lat.run_pass(c)
    for c in range(4):
        lat.run_pass(c)
    with pytest.raises(I.IsfError) as e:
        lat.run_pass(0)                              # schedule done
    assert e.value.code == -5
    b = I.Batch([])
    with pytest.raises(I.IsfError) as e:
        b.add(lat)
    assert e.value.code == -7
    b.close()
    lat.close()
    whole = I.Lattice(H, 3)
    with pytest.raises(I.IsfError) as e:
        whole.run_pass(0)                            # whole films use isf_run_sweeps
    assert e.value.code == -7
    whole.close()
