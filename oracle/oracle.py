"""ctypes wrapper of the CPU oracle (isf_oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's CPU-baseline
leg use this module; the product library never does.  It imports nothing from the product
package.  `build()` compiles the C source with gcc into oracle/_build/.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "isf_oracle.c")
HDR = os.path.join(HERE, "isf_oracle.h")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libisf_oracle.so")

ALWAYS = 0xFFFFFFFF
PERIODIC_X, PERIODIC_Y, PERIODIC_Z = 1, 2, 4
INIT_RANDOM, INIT_UP, INIT_DOWN = 0, 1, 2
STREAM_METROPOLIS, STREAM_GATE, STREAM_INIT = 0, 1, 2


class StepObs(C.Structure):
    _fields_ = [
        ("T", C.c_double), ("h", C.c_double),
        ("M_last", C.c_int64), ("B_last", C.c_int64), ("n_meas", C.c_int64),
        ("sumM", C.c_int64), ("sumAbsM", C.c_int64),
        ("sumM2", C.c_uint64 * 2), ("sumB2", C.c_uint64 * 2), ("sumMB", C.c_uint64 * 2),
        ("sumB", C.c_int64),
        ("m", C.c_double), ("abs_m", C.c_double), ("e", C.c_double),
        ("chi", C.c_double), ("chi_abs", C.c_double), ("C", C.c_double),
    ]


_lock = threading.Lock()
_lib = None


def build(src: str = SRC, out: str = LIB_PATH, extra_flags=()) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math: libm exp must be the one used)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
           *extra_flags, "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _stale(path: str) -> bool:
    if not os.path.exists(path):
        return True
    t = os.path.getmtime(path)
    return any(os.path.getmtime(p) > t for p in (SRC, HDR))


def load(path: str | None = None):
    """Load (building first if needed) the oracle shared library."""
    global _lib
    with _lock:
        if path is None and _lib is not None:
            return _lib
        p = path or LIB_PATH
        if path is None and _stale(p):
            build()
        lib = C.CDLL(p)
        _declare(lib)
        if path is None:
            _lib = lib
        return lib


def _declare(lib):
    u8p, i8p = C.POINTER(C.c_uint8), C.POINTER(C.c_int8)
    i64p, dp, ip = C.POINTER(C.c_int64), C.POINTER(C.c_double), C.POINTER(C.c_int)
    u32p = C.POINTER(C.c_uint32)
    lib.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
    lib.or_philox4x32_10.restype = None
    lib.or_colour.argtypes = [C.c_int] * 3
    lib.or_colour.restype = C.c_int
    lib.or_site_word.argtypes = [C.c_void_p, C.c_uint32, C.c_uint64, C.c_int, C.c_int, C.c_int]
    lib.or_site_word.restype = C.c_uint32
    lib.or_threshold.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, C.c_int]
    lib.or_threshold.restype = C.c_uint32
    lib.or_gate_threshold.argtypes = [C.c_double, C.c_double]
    lib.or_gate_threshold.restype = C.c_uint32
    lib.or_film_create.argtypes = [u8p, C.c_int, C.c_int, C.c_int, C.c_uint, C.c_uint64, C.c_int,
                                   C.POINTER(C.c_void_p)]
    lib.or_film_create.restype = C.c_int
    lib.or_film_destroy.argtypes = [C.c_void_p]
    lib.or_film_destroy.restype = None
    lib.or_film_info.argtypes = [C.c_void_p, i64p, i64p, i64p, i64p, i64p]
    lib.or_film_info.restype = C.c_int
    lib.or_neighbours.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, ip]
    lib.or_neighbours.restype = C.c_int
    lib.or_check_colouring.argtypes = [C.c_void_p]
    lib.or_check_colouring.restype = C.c_int
    lib.or_get_spins.argtypes = [C.c_void_p, i8p]
    lib.or_get_spins.restype = C.c_int
    lib.or_set_spins.argtypes = [C.c_void_p, i8p]
    lib.or_set_spins.restype = C.c_int
    lib.or_set_sweep.argtypes = [C.c_void_p, C.c_int64]
    lib.or_set_sweep.restype = C.c_int
    lib.or_recompute.argtypes = [C.c_void_p, i64p, i64p]
    lib.or_recompute.restype = C.c_int
    lib.or_run.argtypes = [C.c_void_p, C.c_int, dp, dp, ip, ip, C.c_double, C.c_double,
                           C.POINTER(StepObs), i64p]
    lib.or_run.restype = C.c_int
    lib.or_derive.argtypes = [C.POINTER(StepObs), C.c_int64, C.c_double]
    lib.or_derive.restype = None
    lib.or_exact.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, dp]
    lib.or_exact.restype = C.c_int
    lib.or_estimate_tc.argtypes = [C.POINTER(StepObs), C.c_int, dp]
    lib.or_estimate_tc.restype = C.c_int
    lib.or_surface_image.argtypes = [C.c_void_p, C.POINTER(C.c_uint8)]
    lib.or_surface_image.restype = C.c_int64


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


def philox(ctr, key, lib=None) -> np.ndarray:
    lib = lib or load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.or_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def threshold(T, h, J, n, s, lib=None) -> int:
    lib = lib or load()
    return int(lib.or_threshold(T, h, J, n, s))


def gate_threshold(T, h_s, lib=None) -> int:
    """Eq. 9 gate threshold: the gate word g passes iff g < it (or it is ALWAYS)."""
    lib = lib or load()
    return int(lib.or_gate_threshold(T, h_s))


def threshold_table(T, h, J=1.0, lib=None) -> np.ndarray:
    """thr[n + 12][s'] (s' = 0 for s = -1, 1 for s = +1), as the oracle builds it."""
    lib = lib or load()
    t = np.zeros((25, 2), dtype=np.uint32)
    for n in range(-12, 13):
        t[n + 12, 0] = lib.or_threshold(T, h, J, n, -1)
        t[n + 12, 1] = lib.or_threshold(T, h, J, n, 1)
    return t


def records_to_dicts(recs) -> list[dict]:
    out = []
    for r in recs:
        d = {f: getattr(r, f) for f, _ in StepObs._fields_}
        for f in ("sumM2", "sumB2", "sumMB"):
            w = list(d[f])
            v = w[0] | (w[1] << 64)
            if f == "sumMB" and v >= 1 << 127:
                v -= 1 << 128
            d[f] = v
        out.append(d)
    return out


def dicts_to_records(recs):
    """Step records (dicts, as records_to_dicts makes them) back into an or_step_obs array."""
    out = (StepObs * max(len(recs), 1))()
    for i, d in enumerate(recs):
        for f, _ in StepObs._fields_:
            v = d[f]
            if f in ("sumM2", "sumB2", "sumMB"):
                v = int(v) & ((1 << 128) - 1)
                getattr(out[i], f)[0] = v & ((1 << 64) - 1)
                getattr(out[i], f)[1] = v >> 64
            else:
                setattr(out[i], f, v)
    return out


def estimate_tc(recs, lib=None):
    """(T_c, index) of a scan's records by the oracle's or_estimate_tc; (None, -1) if none qualifies."""
    lib = lib or load()
    arr = dicts_to_records(recs)
    t = C.c_double()
    k = int(lib.or_estimate_tc(arr, len(recs), C.byref(t)))
    return (t.value if k >= 0 else None), k


# In-plane neighbours of a pixel (dx, dy): the film's 6 in-plane bonds (Sec. 2).
PIXEL_NEIGHBOURS = ((1, 0), (-1, 0), (0, 1), (0, -1), (1, -1), (-1, 1))


def domain_stats(img, periodic_x=False, periodic_y=False) -> dict:
    """Domains of a PMOKE image (Sec. 6, Fig. 5): connected sets of white (255) or of black (0)
    pixels, two pixels touching when their columns are in-plane neighbours; 128 (no atom)
    belongs to none.  Plain breadth-first search, one pixel at a time."""
    img = np.asarray(img)
    R, C = img.shape
    seen = np.zeros((R, C), dtype=bool)
    out = {"white": 0, "black": 0, "largest_white": 0, "largest_black": 0}
    for y0 in range(R):
        for x0 in range(C):
            v = int(img[y0, x0])
            if v == 128 or seen[y0, x0]:
                continue
            seen[y0, x0] = True
            queue, size = [(x0, y0)], 0
            while queue:
                x, y = queue.pop()
                size += 1
                for dx, dy in PIXEL_NEIGHBOURS:
                    xx, yy = x + dx, y + dy
                    if not 0 <= xx < C:
                        if not periodic_x:
                            continue
                        xx %= C
                    if not 0 <= yy < R:
                        if not periodic_y:
                            continue
                        yy %= R
                    if not seen[yy, xx] and int(img[yy, xx]) == v:
                        seen[yy, xx] = True
                        queue.append((xx, yy))
            key = "white" if v == 255 else "black"
            out[key] += 1
            out["largest_" + key] = max(out["largest_" + key], size)
    return out


class Film:
    """One film in the oracle: heights (rows x cols uint8), layers, flags, seed, init."""

    def __init__(self, heights, layers, flags=0, seed=1, init=INIT_RANDOM, lib=None):
        self.lib = lib or load()
        H = np.ascontiguousarray(heights, dtype=np.uint8)
        if H.ndim != 2:
            raise ValueError("heights must be 2-D (rows, cols)")
        self.rows, self.cols = H.shape
        self.layers = int(layers)
        self.flags = int(flags)
        self.seed = int(seed)
        h = C.c_void_p()
        rc = self.lib.or_film_create(_ptr(H, C.c_uint8), self.rows, self.cols, self.layers,
                                     self.flags, self.seed, int(init), C.byref(h))
        if rc != 0:
            raise OracleError(rc, "film_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self.lib.or_film_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        v = [C.c_int64() for _ in range(5)]
        self.lib.or_film_info(self._h, *[C.byref(x) for x in v])
        return dict(zip(("n_occ", "n_bonds", "M", "B", "sweep"), (x.value for x in v)))

    def neighbours(self, x, y, z) -> list[tuple[int, int, int]]:
        buf = np.zeros(36, dtype=np.int32)
        n = self.lib.or_neighbours(self._h, x, y, z, _ptr(buf, C.c_int))
        if n < 0:
            raise OracleError(n, "neighbours")
        return [tuple(int(v) for v in buf[3 * k:3 * k + 3]) for k in range(n)]

    def check_colouring(self) -> int:
        return int(self.lib.or_check_colouring(self._h))

    def site_word(self, stream, sweep, x, y, z) -> int:
        return int(self.lib.or_site_word(self._h, stream, sweep, x, y, z))

    def spins(self) -> np.ndarray:
        out = np.zeros((self.layers, self.rows, self.cols), dtype=np.int8)
        self.lib.or_get_spins(self._h, _ptr(out, C.c_int8))
        return out

    def set_spins(self, s):
        s = np.ascontiguousarray(s, dtype=np.int8)
        rc = self.lib.or_set_spins(self._h, _ptr(s, C.c_int8))
        if rc != 0:
            raise OracleError(rc, "set_spins")

    def set_sweep(self, sweep):
        rc = self.lib.or_set_sweep(self._h, int(sweep))
        if rc != 0:
            raise OracleError(rc, "set_sweep")

    def recompute(self) -> tuple[int, int]:
        M, B = C.c_int64(), C.c_int64()
        self.lib.or_recompute(self._h, C.byref(M), C.byref(B))
        return M.value, B.value

    def run(self, T, h, sweeps_eq, sweeps_meas, J=1.0, h_s=0.0, series=False):
        """Run whole steps; returns (records as dicts, series (n_sweeps, 2) or None)."""
        T = np.ascontiguousarray(T, dtype=np.float64)
        h = np.ascontiguousarray(h, dtype=np.float64)
        eq = np.ascontiguousarray(sweeps_eq, dtype=np.int32)
        me = np.ascontiguousarray(sweeps_meas, dtype=np.int32)
        n = len(T)
        if not (len(h) == len(eq) == len(me) == n):
            raise ValueError("schedule arrays differ in length")
        recs = (StepObs * max(n, 1))()
        ser = None
        serp = None
        if series:
            ser = np.zeros((int(eq.sum() + me.sum()), 2), dtype=np.int64)
            serp = _ptr(ser, C.c_int64)
        rc = self.lib.or_run(self._h, n, _ptr(T, C.c_double), _ptr(h, C.c_double),
                             _ptr(eq, C.c_int), _ptr(me, C.c_int), float(J), float(h_s),
                             recs, serp)
        if rc != 0:
            raise OracleError(rc, "run")
        return records_to_dicts(recs[:n]), ser

    def surface_image(self) -> np.ndarray:
        out = np.zeros((self.rows, self.cols), dtype=np.uint8)
        self.lib.or_surface_image(self._h, _ptr(out, C.c_uint8))
        return out

    def exact(self, T, h, J=1.0) -> dict:
        out = np.zeros(6, dtype=np.float64)
        rc = self.lib.or_exact(self._h, float(T), float(h), float(J), _ptr(out, C.c_double))
        if rc != 0:
            raise OracleError(rc, "exact")
        return dict(zip(("M", "absM", "M2", "E", "E2", "B"), out.tolist()))
