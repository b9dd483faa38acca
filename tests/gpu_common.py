"""Helpers of the GPU parity tests: run one film through the CUDA path (C ABI, via the binding)
and through the CPU oracle on the same seeded inputs, and compare."""
import numpy as np
import pytest

INT_FIELDS = ("M_last", "B_last", "n_meas", "sumM", "sumAbsM", "sumB", "sumM2", "sumB2", "sumMB")
FP_FIELDS = ("m", "abs_m", "e", "chi", "chi_abs", "C")
# fp64 values derived from identical exact integer sums; the only freedom is rounding order
FP_REL = 1e-12


def gpu_lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1205_5588_gb300 import build
    build.build()
    from paper_1205_5588_gb300 import isingfilm
    return isingfilm


def spec_flags(spec):
    return dict(periodic_x=spec.get("periodic_x", False), periodic_y=spec.get("periodic_y", False),
                periodic_z=spec.get("periodic_z", False))


def oracle_flags(spec):
    return (1 if spec.get("periodic_x") else 0) | (2 if spec.get("periodic_y") else 0) | \
           (4 if spec.get("periodic_z") else 0)


def run_gpu(I, spec, sched, *, packed=None, launch=None, chunks=None, trace=True, h_s=0.0, path="auto",
            sites=0):
    packed = spec.get("packed", False) if packed is None else packed
    lat = I.Lattice(spec["heights"], spec["layers"], packed=packed, seed=spec["seed"], init=spec["init"],
                    **spec_flags(spec))
    if path != "auto":
        lat.set_path(path)
    if launch:
        lat.set_launch(*launch)
    if sites:
        lat.set_item_sites(sites)
    total = int(sched["eq"].sum() + sched["meas"].sum())
    if trace:
        lat.enable_trace(total)
    lat.set_schedule(sched["T"], sched["h"], sched["eq"], sched["meas"], J=spec.get("J", 1.0), h_s=h_s)
    if chunks:
        done = 0
        for n in chunks:
            lat.run(n)
            done += n
        if done < total:
            lat.run(total - done)
    else:
        lat.run(-1)
    out = {"recs": lat.observables(), "spins": lat.spins(), "info": lat.info(), "launch": lat.launch_info(),
           "trace": lat.trace() if trace else None, "state": lat.state(recompute=True)}
    lat.close()
    return out


def run_oracle(spec, sched, h_s=0.0):
    from oracle import oracle
    init = {"random": oracle.INIT_RANDOM, "up": oracle.INIT_UP, "down": oracle.INIT_DOWN}[spec["init"]]
    f = oracle.Film(spec["heights"], spec["layers"], flags=oracle_flags(spec), seed=spec["seed"], init=init)
    recs, ser = f.run(sched["T"], sched["h"], sched["eq"], sched["meas"], J=spec.get("J", 1.0), h_s=h_s,
                      series=True)
    out = {"recs": recs, "spins": f.spins(), "info": f.info(), "trace": ser}
    f.close()
    return out


def assert_records_equal(got, want):
    assert len(got) == len(want)
    for k, (g, w) in enumerate(zip(got, want)):
        for f in INT_FIELDS:
            assert g[f] == w[f], (k, f, g[f], w[f])
        assert g["T"] == w["T"] and g["h"] == w["h"]
        for f in FP_FIELDS:
            a, b = g[f], w[f]
            if np.isnan(b):
                assert np.isnan(a), (k, f)
            else:
                assert a == pytest.approx(b, rel=FP_REL, abs=1e-300), (k, f, a, b)


def assert_same_run(g, o):
    assert g["info"]["n_occ"] == o["info"]["n_occ"]
    assert g["info"]["n_bonds"] == o["info"]["n_bonds"]
    if g["trace"] is not None:
        assert np.array_equal(g["trace"], o["trace"]), first_diff(g["trace"], o["trace"])
    assert_records_equal(g["recs"], o["recs"])
    assert np.array_equal(g["spins"], o["spins"])
    assert g["state"]["M"] == g["state"]["M_full"] and g["state"]["B"] == g["state"]["B_full"]


def first_diff(a, b):
    if a.shape != b.shape:
        return f"shapes {a.shape} vs {b.shape}"
    idx = np.argwhere(a != b)
    return f"first difference at sweep {idx[0][0] + 1}: {a[idx[0][0]]} vs {b[idx[0][0]]}" if len(idx) else "equal"
