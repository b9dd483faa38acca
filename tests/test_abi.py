"""The C-ABI library builds for sm_103a, loads, and exports every function include/*.h declares
(the method's boundary in isingfilm.h, the tuning and test hooks in isingfilm_tuning.h);
host-side argument checks and host-only calls answer without touching a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")
HEADER = os.path.join(INCLUDE, "isingfilm.h")


def declared_functions(path=None):
    paths = [path] if path else [os.path.join(INCLUDE, n) for n in sorted(os.listdir(INCLUDE)) if n.endswith(".h")]
    names = set()
    for p in paths:
        text = re.sub(r"/\*.*?\*/", "", open(p).read(), flags=re.S)
        names |= set(re.findall(r"\b(isf_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1205_5588_gb300 import build
    path = build.build()
    from paper_1205_5588_gb300 import isingfilm
    assert isingfilm.lib._name == path
    return isingfilm.lib


def test_header_declares_the_boundary():
    names = declared_functions(HEADER)
    for must in ("isf_lattice_create", "isf_set_schedule", "isf_run_sweeps", "isf_read_observables",
                 "isf_read_spins", "isf_lattice_destroy", "isf_last_error", "isf_estimate_tc"):
        assert must in names
    # tuning and test hooks live in their own header, not in the method's boundary
    hooks = declared_functions(os.path.join(INCLUDE, "isingfilm_tuning.h"))
    for hook in ("isf_set_launch", "isf_set_path", "isf_set_item_sites", "isf_debug_checks", "isf_debug_item_lists",
                 "isf_debug_slab_partition", "isf_philox_blocks", "isf_peak_probe", "isf_batch_taken",
                 "isf_debug_wait_timeout"):
        assert hook in hooks and hook not in names


def test_every_declared_symbol_is_exported(lib):
    raw = C.CDLL(lib._name)
    missing = [n for n in declared_functions() if not hasattr(raw, n)]
    assert not missing, missing


def test_lattice_bytes(lib):
    from paper_1205_5588_gb300 import isingfilm as I
    assert I.lattice_bytes(256, 256, 6, 0) > 4 * 6 * 128 * 128        # four colour arrays of int8
    assert I.lattice_bytes(2048, 2048, 6, I.PACKED) > 0
    # two bit-planes per colour instead of a byte per site (the height map is stored in both); the
    # packed film also keeps its occupied-word lists and 16 bytes of vacant-neighbour counts per
    # 32-site word position, and still takes less than the int8 one
    assert I.lattice_bytes(2048, 2048, 6, I.PACKED) < I.lattice_bytes(2048, 2048, 6, 0)
    assert I.lattice_bytes(2048, 2048, 6, I.PACKED) > I.lattice_bytes(2048, 2048, 6, 0) / 4
    for bad in [(0, 4, 1, 0), (4, 0, 1, 0), (4, 4, 0, 0), (4, 4, 256, 0), (5, 4, 2, I.PERIODIC_Y),
                (4, 6, 2, I.PERIODIC_X | I.PACKED), (4, 4, 3, I.PERIODIC_Z), (4, 4, 2, 64)]:
        assert I.lattice_bytes(*bad) == 0, bad


@pytest.mark.parametrize("R,C_,L,flags,H,code", [
    (6, 7, 3, 1, 3, -4),        # periodic x with odd extent
    (2, 8, 3, 2, 3, -4),        # periodic y with extent 2
    (4, 4, 3, 0, 4, -1),        # a height above the number of layers
    (4, 6, 2, 1 | 8, 2, -1),    # packed with a periodic axis
    (4, 4, 300, 0, 0, -1),      # too many layers
])
def test_create_rejects_bad_films_before_any_device_work(lib, R, C_, L, flags, H, code):
    heights = np.full((R, C_), H, dtype=np.uint8)
    out = C.c_void_p()
    rc = lib.isf_lattice_create(heights.ctypes.data_as(C.POINTER(C.c_uint8)), R, C_, L, flags, 1, 0, None,
                                C.byref(out))
    assert rc == code
    assert out.value is None
    assert len(lib.isf_last_error()) > 0


def test_null_arguments(lib):
    assert lib.isf_run_sweeps(None, 1, None) == -1
    assert lib.isf_set_schedule(None, 1, None, None, None, None, 1.0, 0.0) == -1
    got = C.c_int32()
    assert lib.isf_read_observables(None, None, 0, C.byref(got)) == -1
    assert lib.isf_lattice_info(None, None, None, None, None) == -1
    assert lib.isf_lattice_create(None, 4, 4, 1, 0, 1, 0, None, None) == -1
    lib.isf_lattice_destroy(None)


def test_peak_probe_rejects_bad_arguments_without_a_gpu(lib):
    from paper_1205_5588_gb300 import isingfilm as I
    for mode, threads, iters in ((9, 256, 10), (I.PEAK_LOP3, 33, 10), (I.PEAK_ATTEMPT, 1024, 10), (I.PEAK_MIX, 256, 0)):
        with pytest.raises(I.IsfError) as e:
            I.peak_probe(mode, 0, threads, iters, stream=0)
        assert e.value.code == -1


def test_wait_probe_argument_errors(lib):
    from paper_1205_5588_gb300 import isingfilm as I
    for ctas in (-1, 0, 1):
        with pytest.raises(I.IsfError):
            I.debug_wait_timeout(ctas)
