"""Thin Python binding of libisingfilm.so (include/isingfilm.h): argument marshalling only.

Every step of the sweep runs in the library's CUDA kernels.  PyTorch supplies device memory
(the film lives in a torch uint8 tensor handed to isf_lattice_create_in) and CUDA streams.
Importing this module fails loudly if the library has not been built; there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

PERIODIC_X, PERIODIC_Y, PERIODIC_Z, PACKED = 1, 2, 4, 8
PATHS = {"auto": 0, "global": 1, "resident": 2, "slabs": 3}
INIT = {"random": 0, "up": 1, "down": 2}
STATUS = {0: "ISF_OK", -1: "ISF_ERR_ARG", -2: "ISF_ERR_OOM", -3: "ISF_ERR_CUDA", -4: "ISF_ERR_COLOURING",
          -5: "ISF_ERR_SCHEDULE", -6: "ISF_ERR_TIMEOUT", -7: "ISF_ERR_STATE"}


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


class IsfJob(C.Structure):
    _fields_ = [
        ("heights", C.POINTER(C.c_uint8)), ("rows", C.c_int32), ("cols", C.c_int32), ("layers", C.c_int32),
        ("flags", C.c_uint32), ("seed", C.c_uint64), ("init", C.c_int32), ("nsteps", C.c_int32),
        ("T", C.POINTER(C.c_double)), ("h", C.POINTER(C.c_double)),
        ("sweeps_eq", C.POINTER(C.c_int32)), ("sweeps_meas", C.POINTER(C.c_int32)),
        ("J", C.c_double), ("h_s", C.c_double),
    ]


class IsfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def _declare(lib):
    vp, u8p, i8p, i64p, dp = C.c_void_p, C.POINTER(C.c_uint8), C.POINTER(C.c_int8), C.POINTER(C.c_int64), C.POINTER(C.c_double)
    i32p, u32p = C.POINTER(C.c_int32), C.POINTER(C.c_uint32)
    sig = {
        "isf_lattice_bytes": (C.c_size_t, [C.c_int32, C.c_int32, C.c_int32, C.c_uint32]),
        "isf_lattice_create": (C.c_int, [u8p, C.c_int32, C.c_int32, C.c_int32, C.c_uint32, C.c_uint64, C.c_int32, vp,
                                         C.POINTER(vp)]),
        "isf_lattice_create_in": (C.c_int, [u8p, C.c_int32, C.c_int32, C.c_int32, C.c_uint32, C.c_uint64, C.c_int32,
                                            vp, vp, C.c_size_t, C.POINTER(vp)]),
        "isf_set_schedule": (C.c_int, [vp, C.c_int32, dp, dp, i32p, i32p, C.c_double, C.c_double]),
        "isf_run_sweeps": (C.c_int, [vp, C.c_int64, vp]),
        "isf_read_observables": (C.c_int, [vp, C.POINTER(StepObs), C.c_int32, i32p]),
        "isf_read_spins": (C.c_int, [vp, i8p]),
        "isf_write_spins": (C.c_int, [vp, i8p, C.c_int64]),
        "isf_lattice_info": (C.c_int, [vp, i64p, i64p, dp, i64p]),
        "isf_read_state": (C.c_int, [vp, i64p, i64p, C.c_int32, i64p, i64p]),
        "isf_enable_trace": (C.c_int, [vp, C.c_int64]),
        "isf_read_trace": (C.c_int, [vp, i64p, C.c_int64, i64p]),
        "isf_set_launch": (C.c_int, [vp, C.c_int32, C.c_int32]),
        "isf_set_path": (C.c_int, [vp, C.c_int32]),
        "isf_read_surface_image": (C.c_int, [vp, u8p, i64p]),
        "isf_lattice_stats": (C.c_int, [vp, dp, dp, dp]),
        "isf_surface_domains": (C.c_int, [vp, i64p]),
        "isf_launch_info": (C.c_int, [vp, i32p, i32p, i32p]),
        "isf_set_item_sites": (C.c_int, [vp, C.c_int32]),
        "isf_debug_item_lists": (C.c_int, [u8p, C.c_int32, C.c_int32, C.c_int32, C.c_uint32, i32p,
                                           C.POINTER(C.c_uint32), C.c_int64, i32p]),
        "isf_debug_slab_partition": (C.c_int, [u8p, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, i32p]),
        "isf_lattice_create_slab": (C.c_int, [u8p, C.c_int32, C.c_int32, C.c_int32, C.c_uint32, C.c_uint64,
                                              C.c_int32, C.c_int32, C.c_int32, vp, C.POINTER(vp)]),
        "isf_slab_info": (C.c_int, [vp, i32p, C.POINTER(C.c_size_t), i64p]),
        "isf_slab_export": (C.c_int, [vp, C.c_int32, C.c_int32, vp, vp]),
        "isf_slab_import": (C.c_int, [vp, C.c_int32, C.c_int32, vp, vp]),
        "isf_run_pass": (C.c_int, [vp, C.c_int32, vp]),
        "isf_fold_series": (C.c_int, [C.c_int32, dp, dp, i32p, i32p, C.c_double, C.c_int64, i64p, i64p,
                                      C.POINTER(StepObs)]),
        "isf_launch_item_sites": (C.c_int, [vp, i32p]),
        "isf_save": (C.c_int, [vp, C.c_char_p]),
        "isf_load": (C.c_int, [C.c_char_p, vp, C.POINTER(vp)]),
        "isf_lattice_destroy": (None, [vp]),
        "isf_last_error": (C.c_char_p, []),
        "isf_philox_blocks": (C.c_int, [C.c_uint64, C.c_uint32, C.c_uint64, C.c_uint32, C.c_int64, u32p]),
        "isf_peak_probe": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int64, vp, dp]),
        "isf_estimate_tc": (C.c_int, [C.POINTER(StepObs), C.c_int32, dp, i32p]),
        "isf_server_job_ticks": (C.c_int, [vp, C.c_int64, i64p]),
        "isf_batch_create": (C.c_int, [C.POINTER(vp)]),
        "isf_batch_add": (C.c_int, [vp, vp]),
        "isf_batch_clear": (C.c_int, [vp]),
        "isf_batch_set_launch": (C.c_int, [vp, C.c_int32, C.c_int32, C.c_int32]),
        "isf_batch_set_graph": (C.c_int, [vp, C.c_int32]),
        "isf_batch_tune": (C.c_int, [vp, vp]),
        "isf_batch_run": (C.c_int, [vp, vp]),
        "isf_batch_info": (C.c_int, [vp, i32p]),
        "isf_batch_taken": (C.c_int, [vp, i32p]),
        "isf_debug_wait_timeout": (C.c_int, [C.c_int32, i32p, i32p]),
        "isf_batch_destroy": (None, [vp]),
        "isf_batch_run_sweeps": (C.c_int, [vp, C.c_int64, vp]),
        "isf_server_create": (C.c_int, [C.c_size_t, C.c_int64, C.POINTER(vp)]),
        "isf_server_submit": (C.c_int, [vp, C.POINTER(IsfJob), i64p]),
        "isf_server_wait": (C.c_int, [vp, C.c_int64, C.c_double, i32p]),
        "isf_server_poll": (C.c_int, [vp, C.c_int64, i32p, C.POINTER(StepObs), C.c_int32, i32p, dp]),
        "isf_server_release": (C.c_int, [vp, C.c_int64]),
        "isf_server_stats": (C.c_int, [vp, i64p, dp]),
        "isf_server_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def _load():
    path = _build.LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"{path} is not built; run `python -m paper_1205_5588_gb300.build` "
                          "(the library has no CPU fallback)")
    return _declare(C.CDLL(path))


lib = _load()


def _check(rc: int, what: str):
    if rc != 0:
        raise IsfError(rc, f"{what}: {lib.isf_last_error().decode(errors='replace')}")


def _stream_handle(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def obs_to_dicts(recs) -> list[dict]:
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


def flags_of(periodic_x=False, periodic_y=False, periodic_z=False, packed=False) -> int:
    return (PERIODIC_X if periodic_x else 0) | (PERIODIC_Y if periodic_y else 0) | \
           (PERIODIC_Z if periodic_z else 0) | (PACKED if packed else 0)


def lattice_bytes(rows, cols, layers, flags) -> int:
    return int(lib.isf_lattice_bytes(rows, cols, layers, flags))


def item_lists(heights, layers, flags=0) -> tuple[list[np.ndarray], int, int]:
    """The occupied-item lists the library keeps for a film (host only): per colour an array of
    entries (z << (jbits + wbits)) | (j << wbits) | w, and (wbits, jbits)."""
    h = np.ascontiguousarray(heights, dtype=np.uint8)
    rows, cols = h.shape
    per_row = -(-(-(-cols // 2)) // (32 if flags & PACKED else 16))
    cap = layers * ((rows + 1) // 2) * per_row
    n = (C.c_int32 * 4)()
    out = np.zeros(4 * max(cap, 1), dtype=np.uint32)
    bits = (C.c_int32 * 2)()
    _check(lib.isf_debug_item_lists(h.ctypes.data_as(C.POINTER(C.c_uint8)), rows, cols, layers, flags, n,
                                    out.ctypes.data_as(C.POINTER(C.c_uint32)), cap, bits), "debug_item_lists")
    return [out[c * cap:c * cap + n[c]].copy() for c in range(4)], bits[0], bits[1]


def slab_partition(heights, layers, bands, max_rows) -> np.ndarray:
    """The row bands the row-slab kernel would use for a packed film (host only): bands + 1
    colour-row boundaries."""
    h = np.ascontiguousarray(heights, dtype=np.uint8)
    out = np.zeros(bands + 1, dtype=np.int32)
    _check(lib.isf_debug_slab_partition(h.ctypes.data_as(C.POINTER(C.c_uint8)), h.shape[0], h.shape[1], layers, bands,
                                        max_rows, out.ctypes.data_as(C.POINTER(C.c_int32))), "debug_slab_partition")
    return out


def fold_series(T, h, sweeps_eq, sweeps_meas, n_occ, M, B, J=1.0) -> list[dict]:
    """Step records of a whole film's per-sweep M, B series under a schedule (isf_fold_series;
    host only)."""
    T = np.ascontiguousarray(T, dtype=np.float64)
    h = np.ascontiguousarray(h, dtype=np.float64)
    eq = np.ascontiguousarray(sweeps_eq, dtype=np.int32)
    me = np.ascontiguousarray(sweeps_meas, dtype=np.int32)
    M = np.ascontiguousarray(M, dtype=np.int64)
    B = np.ascontiguousarray(B, dtype=np.int64)
    n = len(T)
    if not (len(h) == len(eq) == len(me) == n) or len(M) != len(B) or len(M) < int(eq.sum() + me.sum()):
        raise ValueError("schedule arrays differ in length, or the series is shorter than the schedule")
    out = (StepObs * n)()
    _check(lib.isf_fold_series(n, _ptr(T, C.c_double), _ptr(h, C.c_double), _ptr(eq, C.c_int32),
                               _ptr(me, C.c_int32), float(J), int(n_occ), _ptr(M, C.c_int64), _ptr(B, C.c_int64),
                               out), "fold_series")
    return obs_to_dicts(out)


class Lattice:
    """One film on the current CUDA device (isf_lattice_create / isf_lattice_create_in)."""

    def __init__(self, heights, layers, *, periodic_x=False, periodic_y=False, periodic_z=False,
                 packed=False, seed=1, init="random", stream=None, torch_buffer=True):
        H = np.ascontiguousarray(heights, dtype=np.uint8)
        if H.ndim != 2:
            raise ValueError("heights must be 2-D (rows, cols)")
        self.rows, self.cols = H.shape
        self.layers = int(layers)
        self.flags = flags_of(periodic_x, periodic_y, periodic_z, packed)
        self.heights = H
        self._buf = None
        h = C.c_void_p()
        s = _stream_handle(stream)
        initv = INIT[init] if isinstance(init, str) else int(init)
        if torch_buffer:
            import torch
            nbytes = lattice_bytes(self.rows, self.cols, self.layers, self.flags)
            if nbytes == 0:
                # let the library report the reason
                _check(lib.isf_lattice_create(_ptr(H, C.c_uint8), self.rows, self.cols, self.layers, self.flags,
                                              int(seed), initv, s, C.byref(h)), "lattice_create")
            self._buf = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            base = self._buf.data_ptr()
            aligned = (base + 255) & ~255
            rc = lib.isf_lattice_create_in(_ptr(H, C.c_uint8), self.rows, self.cols, self.layers, self.flags,
                                           int(seed), initv, s, C.c_void_p(aligned), nbytes, C.byref(h))
        else:
            rc = lib.isf_lattice_create(_ptr(H, C.c_uint8), self.rows, self.cols, self.layers, self.flags,
                                        int(seed), initv, s, C.byref(h))
        _check(rc, "lattice_create")
        self._h = h

    @classmethod
    def slab(cls, heights, layers, y0, y1, *, periodic_x=False, periodic_y=False, packed=False, seed=1,
             init="random", stream=None):
        """Rows [y0, y1) of the whole film `heights` (isf_lattice_create_slab)."""
        H = np.ascontiguousarray(heights, dtype=np.uint8)
        flags = flags_of(periodic_x, periodic_y, False, packed)
        h = C.c_void_p()
        initv = INIT[init] if isinstance(init, str) else int(init)
        _check(lib.isf_lattice_create_slab(_ptr(H, C.c_uint8), H.shape[0], H.shape[1], int(layers), flags, int(seed),
                                           initv, int(y0), int(y1), _stream_handle(stream), C.byref(h)),
               "lattice_create_slab")
        self = cls._wrap(h, None, H.shape[1], int(layers), flags, H)
        info = self.slab_info()
        self.rows = info["local_rows"]
        return self

    def slab_info(self) -> dict:
        v = (C.c_int32 * 6)()
        nb = C.c_size_t()
        w = (C.c_int64 * 3)()
        _check(lib.isf_slab_info(self._h, v, C.byref(nb), w), "slab_info")
        return {"y0": v[0], "y1": v[1], "ya": v[2], "local_rows": v[3], "jlo": v[4], "jhi": v[5],
                "halo_bytes": nb.value, "M0": w[0], "B2_0": w[1], "n_occ": w[2]}

    def slab_export(self, colour, side, dev_ptr, stream=None):
        _check(lib.isf_slab_export(self._h, int(colour), int(side), C.c_void_p(dev_ptr), _stream_handle(stream)),
               "slab_export")

    def slab_import(self, colour, side, dev_ptr, stream=None):
        _check(lib.isf_slab_import(self._h, int(colour), int(side), C.c_void_p(dev_ptr), _stream_handle(stream)),
               "slab_import")

    def run_pass(self, colour, stream=None):
        _check(lib.isf_run_pass(self._h, int(colour), _stream_handle(stream)), "run_pass")

    @classmethod
    def _wrap(cls, handle, rows, cols, layers, flags, heights):
        self = cls.__new__(cls)
        self._h, self.rows, self.cols, self.layers, self.flags = handle, rows, cols, layers, flags
        self.heights, self._buf = heights, None
        return self

    def close(self):
        if getattr(self, "_h", None):
            lib.isf_lattice_destroy(self._h)
            self._h = None
        self._buf = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_schedule(self, T, h, sweeps_eq, sweeps_meas, J=1.0, h_s=0.0):
        T = np.ascontiguousarray(T, dtype=np.float64)
        h = np.ascontiguousarray(h, dtype=np.float64)
        eq = np.ascontiguousarray(sweeps_eq, dtype=np.int32)
        me = np.ascontiguousarray(sweeps_meas, dtype=np.int32)
        n = len(T)
        if not (len(h) == len(eq) == len(me) == n):
            raise ValueError("schedule arrays differ in length")
        self._nsteps = n
        _check(lib.isf_set_schedule(self._h, n, _ptr(T, C.c_double), _ptr(h, C.c_double), _ptr(eq, C.c_int32),
                                    _ptr(me, C.c_int32), float(J), float(h_s)), "set_schedule")

    def run(self, nsweeps=-1, stream=None):
        _check(lib.isf_run_sweeps(self._h, int(nsweeps), _stream_handle(stream)), "run_sweeps")

    def observables(self, max_steps=None) -> list[dict]:
        n = max_steps if max_steps is not None else getattr(self, "_nsteps", 0)
        recs = (StepObs * max(n, 1))()
        got = C.c_int32()
        _check(lib.isf_read_observables(self._h, recs, n, C.byref(got)), "read_observables")
        return obs_to_dicts(recs[:got.value])

    def spins(self) -> np.ndarray:
        out = np.zeros((self.layers, self.rows, self.cols), dtype=np.int8)
        _check(lib.isf_read_spins(self._h, _ptr(out, C.c_int8)), "read_spins")
        return out

    def surface_domains(self) -> dict:
        """Domains of the PMOKE image: counts and largest sizes, white (up) and black (down)."""
        v = (C.c_int64 * 4)()
        _check(lib.isf_surface_domains(self._h, v), "surface_domains")
        return {"white": v[0], "black": v[1], "largest_white": v[2], "largest_black": v[3]}

    def surface_image(self) -> np.ndarray:
        """Simulated PMOKE image (255 up, 0 down, 128 no atom), rows x cols uint8."""
        out = np.zeros((self.rows, self.cols), dtype=np.uint8)
        n = C.c_int64()
        _check(lib.isf_read_surface_image(self._h, _ptr(out, C.c_uint8), C.byref(n)), "read_surface_image")
        return out

    def stats(self) -> dict:
        """Concentration p, mean coordination zbar and critical concentration p_c = 2/zbar (Eq. 2)."""
        p, z, pc = C.c_double(), C.c_double(), C.c_double()
        _check(lib.isf_lattice_stats(self._h, C.byref(p), C.byref(z), C.byref(pc)), "lattice_stats")
        return {"p": p.value, "zbar": z.value, "p_c": pc.value}

    def write_spins(self, s, sweep):
        s = np.ascontiguousarray(s, dtype=np.int8)
        _check(lib.isf_write_spins(self._h, _ptr(s, C.c_int8), int(sweep)), "write_spins")

    def info(self) -> dict:
        n, b, sw = C.c_int64(), C.c_int64(), C.c_int64()
        z = C.c_double()
        _check(lib.isf_lattice_info(self._h, C.byref(n), C.byref(b), C.byref(z), C.byref(sw)), "lattice_info")
        return {"n_occ": n.value, "n_bonds": b.value, "zbar": z.value, "sweep": sw.value}

    def state(self, recompute=False) -> dict:
        M, B, Mf, Bf = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib.isf_read_state(self._h, C.byref(M), C.byref(B), 1 if recompute else 0, C.byref(Mf), C.byref(Bf)),
               "read_state")
        d = {"M": M.value, "B": B.value}
        if recompute:
            d.update(M_full=Mf.value, B_full=Bf.value)
        return d

    def enable_trace(self, max_sweeps):
        _check(lib.isf_enable_trace(self._h, int(max_sweeps)), "enable_trace")
        self._trace_cap = int(max_sweeps)

    def trace(self) -> np.ndarray:
        """(M, B) after each sweep since enable_trace, as an (n, 2) int64 array."""
        buf = np.zeros((max(getattr(self, "_trace_cap", 0), 1), 2), dtype=np.int64)
        n = C.c_int64()
        _check(lib.isf_read_trace(self._h, _ptr(buf, C.c_int64), getattr(self, "_trace_cap", 0), C.byref(n)),
               "read_trace")
        return buf[: n.value]

    def set_launch(self, ctas=0, threads=0):
        _check(lib.isf_set_launch(self._h, int(ctas), int(threads)), "set_launch")

    def set_item_sites(self, sites=0):
        """Sites per work item of the resident kernel: 16, 8 or 0 (automatic)."""
        _check(lib.isf_set_item_sites(self._h, int(sites)), "set_item_sites")

    def launch_info(self) -> dict:
        p, c, t, w = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib.isf_launch_info(self._h, C.byref(p), C.byref(c), C.byref(t)), "launch_info")
        _check(lib.isf_launch_item_sites(self._h, C.byref(w)), "launch_item_sites")
        return {"path": {0: None, 1: "global", 2: "resident", 3: "slabs"}[p.value], "ctas": c.value, "threads": t.value,
                "item_sites": w.value}

    def set_path(self, path="auto"):
        """'resident' (int8 film in one cluster's shared memory), 'global' (film in device memory,
        all SMs), 'slabs' (packed film in row bands, one per CTA, in shared memory) or 'auto'."""
        _check(lib.isf_set_path(self._h, PATHS[path]), "set_path")

    def save(self, path):
        _check(lib.isf_save(self._h, str(path).encode()), "save")

    @classmethod
    def load(cls, path, stream=None):
        h = C.c_void_p()
        _check(lib.isf_load(str(path).encode(), _stream_handle(stream), C.byref(h)), "load")
        with open(path, "rb") as fp:
            fp.read(8)
            hdr = np.frombuffer(fp.read(20), dtype=np.int32)
            fp.read(16)
            rows, cols, layers, flags = (int(v) for v in hdr[:4])
            heights = np.frombuffer(fp.read(rows * cols), dtype=np.uint8).reshape(rows, cols).copy()
        return cls._wrap(h, rows, cols, layers, flags, heights)


class Batch:
    """Many films advanced together (isf_batch_*); it references, not owns, its lattices."""

    def __init__(self, films=(), graph=False):
        h = C.c_void_p()
        _check(lib.isf_batch_create(C.byref(h)), "batch_create")
        self._h = h
        self.films = []
        if graph:
            self.set_graph(True)
        for f in films:
            self.add(f)

    def add(self, lat: Lattice):
        _check(lib.isf_batch_add(self._h, lat._h), "batch_add")
        self.films.append(lat)

    def clear(self):
        _check(lib.isf_batch_clear(self._h), "batch_clear")
        self.films = []

    def set_launch(self, threads_single=0, cluster_K=0, threads_cluster=0):
        _check(lib.isf_batch_set_launch(self._h, threads_single, cluster_K, threads_cluster), "batch_set_launch")

    def set_graph(self, on=True):
        _check(lib.isf_batch_set_graph(self._h, 1 if on else 0), "batch_set_graph")

    def tune(self, stream=None):
        _check(lib.isf_batch_tune(self._h, _stream_handle(stream)), "batch_tune")

    def run(self, stream=None, max_sweeps=-1):
        _check(lib.isf_batch_run_sweeps(self._h, int(max_sweeps), _stream_handle(stream)), "batch_run")

    def info(self) -> dict:
        v = (C.c_int32 * 12)()
        _check(lib.isf_batch_info(self._h, v), "batch_info")
        keys = ("single_cta_films", "cluster_films", "global_films", "ctas", "clusters", "cluster_K",
                "threads_single", "threads_cluster", "global_cta_films", "global_ctas",
                "global_cluster_films", "global_clusters")
        return dict(zip(keys, list(v)))

    def taken(self) -> dict:
        """Films of the last run that a global-memory queue kernel took from the single-CTA and
        from the cluster resident queue (waits for the run)."""
        v = (C.c_int32 * 2)()
        _check(lib.isf_batch_taken(self._h, v), "batch_taken")
        return {"single_cta": int(v[0]), "cluster": int(v[1])}

    def close(self):
        if getattr(self, "_h", None):
            lib.isf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dicts_to_obs(records):
    """Step records (dicts, as obs_to_dicts makes them) back into an isf_step_obs array."""
    out = (StepObs * max(len(records), 1))()
    for i, d in enumerate(records):
        for f, _ in StepObs._fields_:
            v = d[f]
            if f in ("sumM2", "sumB2", "sumMB"):
                v = int(v) & ((1 << 128) - 1)
                getattr(out[i], f)[0] = v & ((1 << 64) - 1)
                getattr(out[i], f)[1] = v >> 64
            else:
                setattr(out[i], f, v)
    return out


def estimate_tc(records, with_index=False):
    """Curie-temperature estimate of a temperature scan (isf_estimate_tc): the T of the largest
    susceptibility chi' among the scan's records."""
    arr = dicts_to_obs(records)
    t, k = C.c_double(), C.c_int32()
    _check(lib.isf_estimate_tc(arr, len(records), C.byref(t), C.byref(k)), "estimate_tc")
    return (t.value, k.value) if with_index else t.value


PEAK_LOP3, PEAK_MIX, PEAK_PHILOX, PEAK_ATTEMPT = 0, 1, 2, 3


def peak_probe(mode, ctas=0, threads=0, iters=1024, stream=None) -> float:
    """Launch one integer-issue probe (isf_peak_probe) on `stream`; returns its work units
    (lane-ops, Philox blocks or attempts).  Asynchronous: time it with events on that stream."""
    units = C.c_double()
    _check(lib.isf_peak_probe(int(mode), int(ctas), int(threads), int(iters), _stream_handle(stream),
                              C.byref(units)), "peak_probe")
    return units.value


def debug_wait_timeout(ctas=2) -> tuple:
    """Run the grid barrier's bounded wait against an arrival nothing makes
    (isf_debug_wait_timeout); returns (status the kernel recorded, wait site)."""
    st, wh = C.c_int32(), C.c_int32()
    _check(lib.isf_debug_wait_timeout(int(ctas), C.byref(st), C.byref(wh)), "debug_wait_timeout")
    return st.value, wh.value


JOB_STATES = {0: "queued", 1: "running", 2: "done", 3: "failed"}


class Server:
    """Continuous-batching job server (isf_server_*) on the current CUDA device."""

    def __init__(self, budget_bytes, sweeps_per_tick=50):
        h = C.c_void_p()
        _check(lib.isf_server_create(int(budget_bytes), int(sweeps_per_tick), C.byref(h)), "server_create")
        self._h = h
        self._nsteps = {}

    def submit(self, heights, layers, T, h, sweeps_eq, sweeps_meas, *, seed=1, init="random", packed=False,
               periodic_x=False, periodic_y=False, J=1.0, h_s=0.0) -> int:
        H = np.ascontiguousarray(heights, dtype=np.uint8)
        Ta = np.ascontiguousarray(T, dtype=np.float64)
        ha = np.ascontiguousarray(h, dtype=np.float64)
        eq = np.ascontiguousarray(sweeps_eq, dtype=np.int32)
        me = np.ascontiguousarray(sweeps_meas, dtype=np.int32)
        job = IsfJob(_ptr(H, C.c_uint8), H.shape[0], H.shape[1], int(layers),
                     flags_of(periodic_x, periodic_y, False, packed), int(seed),
                     INIT[init] if isinstance(init, str) else int(init), len(Ta),
                     _ptr(Ta, C.c_double), _ptr(ha, C.c_double), _ptr(eq, C.c_int32), _ptr(me, C.c_int32),
                     float(J), float(h_s))
        jid = C.c_int64()
        _check(lib.isf_server_submit(self._h, C.byref(job), C.byref(jid)), "server_submit")
        self._nsteps[jid.value] = len(Ta)
        return jid.value

    def wait(self, jid, timeout=60.0) -> str:
        st = C.c_int32()
        _check(lib.isf_server_wait(self._h, int(jid), float(timeout), C.byref(st)), "server_wait")
        return JOB_STATES[st.value]

    def result(self, jid):
        """(state, records as dicts, latency seconds); raises IsfError for a failed job."""
        n = self._nsteps.get(jid, 0)
        recs = (StepObs * max(n, 1))()
        st, got, lat = C.c_int32(), C.c_int32(), C.c_double()
        _check(lib.isf_server_poll(self._h, int(jid), C.byref(st), recs, n, C.byref(got), C.byref(lat)),
               "server_poll")
        return JOB_STATES[st.value], obs_to_dicts(recs[:got.value]), lat.value

    def job_ticks(self, jid) -> dict:
        """The batched launches (ticks) a job ran in: first, last, and how many."""
        v = (C.c_int64 * 3)()
        _check(lib.isf_server_job_ticks(self._h, int(jid), v), "server_job_ticks")
        return {"first": v[0], "last": v[1], "count": v[2]}

    def release(self, jid):
        _check(lib.isf_server_release(self._h, int(jid)), "server_release")
        self._nsteps.pop(jid, None)

    def stats(self) -> dict:
        v8 = (C.c_int64 * 8)()
        v4 = (C.c_double * 4)()
        _check(lib.isf_server_stats(self._h, v8, v4), "server_stats")
        k8 = ("submitted", "completed", "failed", "active", "queued", "ticks", "attempts_done", "peak_bytes")
        k4 = ("busy_s", "uptime_s", "bytes_in_use", "budget_bytes")
        d = dict(zip(k8, list(v8)))
        d.update(zip(k4, list(v4)))
        return d

    def close(self):
        if getattr(self, "_h", None):
            lib.isf_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def philox_blocks(seed, stream, sweep, q0, n) -> np.ndarray:
    out = np.zeros((n, 4), dtype=np.uint32)
    _check(lib.isf_philox_blocks(int(seed), int(stream), int(sweep), int(q0), int(n), _ptr(out, C.c_uint32)),
           "philox_blocks")
    return out
