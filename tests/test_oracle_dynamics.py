"""Oracle pins: the Markov chain of Eq. 8 (and the Eq. 9 gate) and the observables.

- Exact enumeration of all 2^N states (Eqs. 4-5) against long oracle runs, within 5 binned
  standard errors, on periodic, open and masked films, with and without a field.
- The Eq. 9 gate multiplies both directions of a flip by the same probability, so it must
  leave those equilibrium averages unchanged; with h_s = 0 it must change nothing at all.
  Its own probability is pinned where Eq. 8 always accepts (J = 0, h = 0): a site flips
  exactly when its gate word passes exp(-|h_s| / T), site by site; and at T = h_s = 1000 the
  flip rate per attempt is e^-1 times an Eq. 8 acceptance in [exp(-0.024), 1].
- T = inf: every attempt flips, so M alternates in sign and B never changes.
- T = 0 from all up with h >= 0 (Sec. 5, the T = 0 argument): nothing flips; E = -J bonds - h N.
- High T: <M^2>/N -> 1 and T^2 C / N -> J^2 bonds / N.
- The fp64 estimators from the exact integer sums equal those computed from the per-sweep
  series with exact rational arithmetic.
- FCC Ising bulk: Binder cumulants of two periodic cubes cross between T = 8.8 and 10.8
  (literature T_c/J = 9.79 for the FCC lattice).
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle


def binned(x, nbins=50):
    x = np.asarray(x, dtype=np.float64)
    n = (len(x) // nbins) * nbins
    b = x[:n].reshape(nbins, -1).mean(axis=1)
    return float(x.mean()), float(b.std(ddof=1) / np.sqrt(nbins))


ENUM_FILMS = {
    "periodic4x4x1": (np.full((4, 4), 1, dtype=np.uint8), 1, 3),
    "open3x2x2": (np.full((2, 3), 2, dtype=np.uint8), 2, 0),
    "masked4x4x2": (np.array([[2, 1, 0, 2], [1, 2, 2, 0], [0, 2, 1, 1], [2, 0, 1, 2]], dtype=np.uint8), 2, 0),
}


@pytest.mark.parametrize("film", list(ENUM_FILMS))
# Temperatures where a 16-spin film mixes in a few sweeps; below the 2-D triangular T_c (3.64)
# the periodic film sits in one ordered state for long stretches and binned errors mislead.
@pytest.mark.parametrize("T,h,h_s", [(4.0, 0.3, 0.0), (5.0, -0.5, 0.0), (6.0, 0.0, 0.0), (4.5, 0.4, 2.0)])
def test_exact_enumeration(olib, film, T, h, h_s):
    H, L, flags = ENUM_FILMS[film]
    f = oracle.Film(H, L, flags=flags, seed=5, lib=olib)
    N = f.info()["n_occ"]
    assert N <= 20
    ex = f.exact(T, h)
    nsw = 200000
    _, ser = f.run([T], [h], [0], [nsw], h_s=h_s, series=True)
    M = ser[2000:, 0].astype(np.float64)
    B = ser[2000:, 1].astype(np.float64)
    E = -B - h * M
    for name, series, exact in (("M", M, ex["M"]), ("absM", np.abs(M), ex["absM"]),
                                ("M2", M * M, ex["M2"]), ("E", E, ex["E"]), ("E2", E * E, ex["E2"])):
        mean, err = binned(series)
        assert abs(mean - exact) <= 5 * err + 1e-9, (name, mean, exact, err)


def test_gate_off_changes_nothing(olib):
    H = np.full((6, 6), 3, dtype=np.uint8)
    a = oracle.Film(H, 3, flags=3, seed=9, lib=olib)
    b = oracle.Film(H, 3, flags=3, seed=9, lib=olib)
    ra, sa = a.run([2.5, 3.0], [0.2, -0.2], [10, 0], [20, 30], h_s=0.0, series=True)
    rb, sb = b.run([2.5, 3.0], [0.2, -0.2], [10, 0], [20, 30], series=True)
    assert np.array_equal(sa, sb) and ra == rb
    assert np.array_equal(a.spins(), b.spins())


def test_gate_slows_flips(olib):
    """With h_s > 0 fewer flips happen at the same T (items 4-5 of Sec. 5)."""
    H = np.full((8, 8), 2, dtype=np.uint8)
    flips = []
    for h_s in (0.0, 8.0):         # gate passes with probability exp(-8/8) = 0.37
        f = oracle.Film(H, 2, flags=3, seed=2, init=oracle.INIT_UP, lib=olib)
        _, ser = f.run([8.0], [0.0], [0], [400], h_s=h_s, series=True)
        flips.append(np.abs(np.diff(ser[:, 0])).sum())
    assert flips[1] < 0.5 * flips[0]


def _gate_count(p):
    """#{g in [0, 2^32): (g + 1/2) 2^-32 < p} in exact rationals (the Eq. 8/9 encoding)."""
    from tests.test_oracle_rng_table import _count_exact
    return _count_exact(p)


@pytest.mark.parametrize("T,h_s", [(2.0, 1.0), (3.0, -4.5), (0.7, 0.35), (1e3, 1e3)])
def test_gate_decides_every_flip_when_eq8_always_accepts(olib, T, h_s):
    """With J = 0 and h = 0 every Eq. 8 step has dE = 0 and is accepted, so a site flips in a
    sweep exactly when its Eq. 9 gate word (stream 1) passes: g < #{g : (g + 1/2) 2^-32 <
    exp(-|h_s| / T)}.  Checked site by site over several sweeps, against that count formed here
    in exact rationals."""
    H = np.array([[3, 2, 0, 3, 1], [1, 3, 3, 2, 0], [2, 0, 1, 3, 3], [3, 3, 2, 1, 2]], dtype=np.uint8)
    L = 3
    f = oracle.Film(H, L, seed=0xFEED, lib=olib)
    cnt = _gate_count(np.exp(-abs(h_s) / T))
    occ = [(x, y, z) for z in range(L) for y in range(H.shape[0]) for x in range(H.shape[1]) if z < H[y, x]]
    flips = 0
    for sweep in range(1, 9):
        before = f.spins()
        f.run([T], [0.0], [0], [1], J=0.0, h_s=h_s)
        after = f.spins()
        for (x, y, z) in occ:
            g = f.site_word(oracle.STREAM_GATE, sweep, x, y, z)
            passed = g < cnt
            assert (after[z, y, x] != before[z, y, x]) == passed, (sweep, x, y, z, g, cnt)
            flips += passed
    assert 0 < flips < 8 * len(occ)


def test_gate_flip_rate(olib):
    """At T = 1000 with h_s = 1000 the gate passes with probability e^-1, and Eq. 8 accepts with
    probability between exp(-24/1000) and 1 (|dE| <= 2 (12 J + |h|) with h = 0): the flip fraction
    per attempt lies in [0.976 e^-1, e^-1] up to 5 binomial standard deviations."""
    H = np.full((12, 12), 3, dtype=np.uint8)
    f = oracle.Film(H, 3, flags=3, seed=11, lib=olib)
    N = f.info()["n_occ"]
    nsw = 300
    prev = f.spins()
    flips = 0
    for _ in range(nsw):
        f.run([1e3], [0.0], [0], [1], h_s=1e3)
        cur = f.spins()
        flips += int((cur != prev).sum())
        prev = cur
    n = N * nsw
    frac = flips / n
    p = np.exp(-1.0)
    sd = np.sqrt(p * (1 - p) / n)
    assert np.exp(-24.0 / 1e3) * p - 5 * sd <= frac <= p + 5 * sd, (frac, p, sd)


@pytest.mark.parametrize("flags,init", [(3, oracle.INIT_RANDOM), (0, oracle.INIT_UP)])
def test_infinite_temperature_alternates(olib, flags, init):
    rng = np.random.Generator(np.random.PCG64(3))
    H = rng.integers(1, 4, size=(6, 8)).astype(np.uint8) if flags == 0 else np.full((6, 8), 3, np.uint8)
    f = oracle.Film(H, 3, flags=flags, seed=4, init=init, lib=olib)
    M0, B0 = f.recompute()
    s0 = f.spins()
    _, ser = f.run([float("inf")] * 3, [0.0, 1.5, -2.0], [0, 2, 1], [5, 3, 4], series=True)
    for k, (M, B) in enumerate(ser, start=1):
        assert M == (-1) ** k * M0 and B == B0
    assert np.array_equal(f.spins(), (-1) ** len(ser) * s0)


@pytest.mark.parametrize("h", [0.0, 0.5, 3.0])
def test_zero_temperature_ground_state_stays(olib, h):
    rng = np.random.Generator(np.random.PCG64(8))
    H = rng.integers(0, 5, size=(9, 7)).astype(np.uint8)
    f = oracle.Film(H, 4, seed=1, init=oracle.INIT_UP, lib=olib)
    info = f.info()
    recs, ser = f.run([0.0, 0.0], [h, h], [3, 0], [5, 4], series=True)
    assert np.all(ser[:, 0] == info["n_occ"]) and np.all(ser[:, 1] == info["n_bonds"])
    e_ground = (-1.0 * info["n_bonds"] - h * info["n_occ"]) / info["n_occ"]
    assert recs[-1]["e"] == pytest.approx(e_ground, rel=1e-15)


def test_zero_temperature_field_reversal_aligns_isolated_spins(olib):
    """Sites with no occupied neighbour follow the field at T = 0 (dE = 2 s h < 0 for s = -sign h)."""
    H = np.zeros((6, 6), dtype=np.uint8)
    H[0, 0] = H[3, 3] = H[0, 4] = 1
    f = oracle.Film(H, 1, seed=1, init=oracle.INIT_UP, lib=olib)
    _, ser = f.run([0.0], [-1.0], [0], [1], series=True)
    assert ser[0, 0] == -3 and ser[0, 1] == 0


def test_high_temperature_limits(olib):
    H = np.full((8, 8), 3, dtype=np.uint8)
    f = oracle.Film(H, 3, flags=3, seed=6, lib=olib)
    info = f.info()
    N, nb = info["n_occ"], info["n_bonds"]
    T = 400.0
    recs, ser = f.run([T], [0.0], [200], [20000], series=True)
    M = ser[200:, 0].astype(np.float64)
    m2, err = binned(M * M / N)
    assert abs(m2 - 1.0) < 5 * err + 0.02
    TC = T * T * recs[0]["C"]
    assert TC == pytest.approx(nb / N, rel=0.05)


def _exact_estimators(M, B, T, h, N, J=1.0):
    n = len(M)
    M = [int(v) for v in M]
    B = [int(v) for v in B]
    sM, sA, sB = sum(M), sum(abs(v) for v in M), sum(B)
    sM2, sB2, sMB = sum(v * v for v in M), sum(v * v for v in B), sum(a * b for a, b in zip(M, B))
    F = Fraction
    varM = F(n * sM2 - sM * sM, n * n)
    varA = F(n * sM2 - sA * sA, n * n)
    varB = F(n * sB2 - sB * sB, n * n)
    cov = F(n * sMB - sM * sB, n * n)
    Tq, hq, Jq = F(T), F(h), F(J)
    varE = Jq * Jq * varB + hq * hq * varM + 2 * Jq * hq * cov
    return {
        "m": float(F(sM, n) / N), "abs_m": float(F(sA, n) / N),
        "e": float((-Jq * F(sB, n) - hq * F(sM, n)) / N),
        "chi": float(varM / (N * Tq)), "chi_abs": float(varA / (N * Tq)), "C": float(varE / (N * Tq * Tq)),
    }


def test_estimators_from_exact_sums(olib):
    H = np.full((8, 10), 2, dtype=np.uint8)
    f = oracle.Film(H, 2, seed=12, lib=olib)
    N = f.info()["n_occ"]
    T = [1.5, 2.5, 4.0]
    h = [0.7, -0.3, 0.0]
    eq, me = [5, 3, 0], [40, 25, 33]
    recs, ser = f.run(T, h, eq, me, series=True)
    start = 0
    for k, r in enumerate(recs):
        block = ser[start + eq[k]: start + eq[k] + me[k]]
        start += eq[k] + me[k]
        assert r["n_meas"] == me[k]
        assert r["M_last"] == ser[start - 1, 0] and r["B_last"] == ser[start - 1, 1]
        assert r["sumM"] == int(block[:, 0].sum()) and r["sumB"] == int(block[:, 1].sum())
        assert r["sumM2"] == sum(int(v) ** 2 for v in block[:, 0])
        assert r["sumMB"] == sum(int(a) * int(b) for a, b in block)
        ref = _exact_estimators(block[:, 0], block[:, 1], T[k], h[k], N)
        for key, v in ref.items():
            assert r[key] == pytest.approx(v, rel=1e-12, abs=1e-300), key


def test_incremental_bookkeeping_matches_recompute(olib):
    rng = np.random.Generator(np.random.PCG64(21))
    H = rng.integers(0, 6, size=(11, 9)).astype(np.uint8)
    f = oracle.Film(H, 5, seed=77, lib=olib)
    f.run([2.0, 5.0, 9.0], [1.0, -1.0, 0.0], [2, 2, 2], [3, 3, 3])   # raises on mismatch
    info = f.info()
    assert (info["M"], info["B"]) == f.recompute()
    assert info["sweep"] == 15


def test_set_spins_and_resume_is_the_same_chain(olib):
    H = np.full((6, 8), 3, dtype=np.uint8)
    a = oracle.Film(H, 3, flags=1, seed=31, lib=olib)
    ra, _ = a.run([3.0, 2.0], [0.0, 0.5], [0, 0], [7, 6])
    b = oracle.Film(H, 3, flags=1, seed=31, lib=olib)
    b.run([3.0], [0.0], [0], [7])
    s, sw = b.spins(), b.info()["sweep"]
    c = oracle.Film(H, 3, flags=1, seed=31, init=oracle.INIT_UP, lib=olib)
    c.set_spins(s)
    c.set_sweep(sw)
    rc, _ = c.run([2.0], [0.5], [0], [6])
    assert rc[0] == ra[1]
    assert np.array_equal(c.spins(), a.spins())


def binder(M):
    M = np.asarray(M, dtype=np.float64)
    return 1.0 - np.mean(M ** 4) / (3.0 * np.mean(M ** 2) ** 2)


def test_fcc_bulk_curie_point_bracket(olib):
    U = {}
    for Lc in (6, 10):
        for T in (8.8, 10.8):
            f = oracle.Film(np.full((Lc, Lc), Lc, dtype=np.uint8), Lc, flags=7, seed=100 + Lc,
                            init=oracle.INIT_UP, lib=olib)
            _, ser = f.run([T], [0.0], [2000], [25000], series=True)
            U[(Lc, T)] = binder(ser[2000:, 0])
    # ordered side: the larger cube is closer to 2/3; disordered side: closer to 0
    assert U[(10, 8.8)] > U[(6, 8.8)]
    assert U[(10, 10.8)] < U[(6, 10.8)]
