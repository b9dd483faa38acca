"""isf_run_noalloc: the entry point for callers that must not allocate device memory (their
device memory belongs to another allocator's pool, or cudaMalloc/cudaFree would synchronise the
device inside a latency-bound loop).  It must give what the allocating path gives, call after
call, although every call reuses the same fixed device array.

Collected last on purpose (file name), so a run that stops at its first failure has already
run every other test.  Passes alone in a fresh process and after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1205_5588_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP_REL = 1e-12
INT_FIELDS = ("M_last", "B_last", "n_meas", "sumM", "sumAbsM", "sumB", "sumM2", "sumB2", "sumMB")
FP_FIELDS = ("m", "abs_m", "e", "chi", "chi_abs", "C")


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1205_5588_gb300 import build
    build.build()
    from paper_1205_5588_gb300 import isingfilm as I
    lib = C.CDLL(I.lib._name)          # the C ABI directly, not the binding
    fn = lib.isf_run_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.POINTER(C.c_uint8), C.c_int32, C.c_int32, C.c_int32, C.c_uint32, C.c_uint64, C.c_int32,
                   C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int32),
                   C.POINTER(C.c_int32), C.c_double, C.c_double, C.c_void_p, C.POINTER(I.StepObs), C.c_void_p]
    lib.isf_last_error.restype = C.c_char_p
    return torch, I, lib


def run_noalloc(env, H, layers, flags, seed, init, sched, h_s=0.0):
    torch, I, lib = env
    H = np.ascontiguousarray(H, dtype=np.uint8)
    R, Cc = H.shape
    T = np.ascontiguousarray(sched["T"], dtype=np.float64)
    h = np.ascontiguousarray(sched["h"], dtype=np.float64)
    eq = np.ascontiguousarray(sched["eq"], dtype=np.int32)
    me = np.ascontiguousarray(sched["meas"], dtype=np.int32)
    n = len(T)
    spins = torch.empty(layers * R * Cc, dtype=torch.int8, device="cuda")   # caller-owned output
    recs = (I.StepObs * n)()
    stream = torch.cuda.current_stream()
    rc = lib.isf_run_noalloc(H.ctypes.data_as(C.POINTER(C.c_uint8)), R, Cc, layers, flags, seed, init, n,
                             T.ctypes.data_as(C.POINTER(C.c_double)), h.ctypes.data_as(C.POINTER(C.c_double)),
                             eq.ctypes.data_as(C.POINTER(C.c_int32)), me.ctypes.data_as(C.POINTER(C.c_int32)),
                             1.0, h_s, C.c_void_p(spins.data_ptr()), recs, C.c_void_p(stream.cuda_stream))
    assert rc == 0, lib.isf_last_error()
    return spins.cpu().numpy().reshape(layers, R, Cc), I.obs_to_dicts(recs)


def run_allocating(env, H, layers, flags, seed, init, sched, h_s=0.0):
    _, I, _ = env
    lat = I.Lattice(H, layers, periodic_x=bool(flags & 1), periodic_y=bool(flags & 2), packed=bool(flags & 8),
                    seed=seed, init=init)
    lat.set_schedule(sched["T"], sched["h"], sched["eq"], sched["meas"], h_s=h_s)
    lat.run(-1)
    out = lat.spins(), lat.observables()
    lat.close()
    return out


def assert_same(a, b):
    assert np.array_equal(a[0], b[0])
    assert len(a[1]) == len(b[1])
    for ra, rb in zip(a[1], b[1]):
        for f in INT_FIELDS:
            assert ra[f] == rb[f], f
        for f in FP_FIELDS:
            if np.isnan(rb[f]):
                assert np.isnan(ra[f])
            else:
                assert ra[f] == pytest.approx(rb[f], rel=FP_REL, abs=1e-300), f


CASES = [
    # (heights, layers, flags, seed, init, schedule, h_s)
    (W.fractal_heights(96, 80, 0.7, 1, 5, seed=31), 5, 0, 3, 0,
     W.schedule([1.5, 3.0, 6.0], [0.5, 0.0, -0.5], [3, 2, 0], [5, 6, 7]), 0.0),
    (W.fractal_heights(40, 64, 0.8, 1, 3, seed=32), 3, 8, 9, 1,
     W.schedule([2.0, 2.0, 4.0, 4.0], [2.0, -2.0, 1.0, -1.0], 1, 4), 3.0),
    (np.full((16, 16), 3, dtype=np.uint8), 3, 3, 1, 0,
     W.schedule(3.0, W.loop_fields(40, 10)[:20], 0, 10), 0.0),
]


def test_noalloc_matches_the_allocating_path_call_after_call(env):
    first = []
    for H, L, flags, seed, init, sched, h_s in CASES:            # one call after another
        got = run_noalloc(env, H, L, flags, seed, init, sched, h_s)
        assert_same(got, run_allocating(env, H, L, flags, seed, init, sched, h_s))
        first.append(got)
    H, L, flags, seed, init, sched, h_s = CASES[0]                 # the first film again, after the others
    assert_same(run_noalloc(env, H, L, flags, seed, init, sched, h_s), first[0])


def test_noalloc_allocates_no_device_memory(env):
    """The property the entry point exists for: after a warm-up call (which loads the kernels and
    looks up the array's address), a further call leaves the device's free memory unchanged."""
    torch, I, lib = env
    H, L, flags, seed, init, sched, h_s = CASES[0]
    run_noalloc(env, H, L, flags, seed, init, sched, h_s)            # warm-up
    Hc = np.ascontiguousarray(H, dtype=np.uint8)
    R, Cc = Hc.shape
    T = np.ascontiguousarray(sched["T"], dtype=np.float64)
    h = np.ascontiguousarray(sched["h"], dtype=np.float64)
    eq = np.ascontiguousarray(sched["eq"], dtype=np.int32)
    me = np.ascontiguousarray(sched["meas"], dtype=np.int32)
    spins = torch.empty(L * R * Cc, dtype=torch.int8, device="cuda")  # the caller's buffers, made before
    recs = (I.StepObs * len(T))()
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    rc = lib.isf_run_noalloc(Hc.ctypes.data_as(C.POINTER(C.c_uint8)), R, Cc, L, flags, seed, init, len(T),
                             T.ctypes.data_as(C.POINTER(C.c_double)), h.ctypes.data_as(C.POINTER(C.c_double)),
                             eq.ctypes.data_as(C.POINTER(C.c_int32)), me.ctypes.data_as(C.POINTER(C.c_int32)),
                             1.0, h_s, C.c_void_p(spins.data_ptr()), recs, C.c_void_p(stream.cuda_stream))
    assert rc == 0, lib.isf_last_error()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before


def test_noalloc_refuses_films_beyond_its_array(env):
    torch, I, lib = env
    H = np.full((2048, 2048), 6, dtype=np.uint8)                  # ~35 MB of int8 layout
    sched = W.schedule([2.0], [0.0], 0, 1)
    with pytest.raises(AssertionError) as e:
        run_noalloc(env, H, 6, 0, 1, 0, sched)
    assert b"scratch" in lib.isf_last_error()
