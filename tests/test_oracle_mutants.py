"""The oracle's pins must catch plausible mistakes.

Each case copies isf_oracle.c, plants one mistake (a dropped or wrong term, a flipped sign, a
wrong index, an off-by-one), builds it on the CPU and checks that one of the pins of
test_oracle_* now fails.  The mistakes live only in temporary copies.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle
from tests.conftest import torch_philox_blocks

SRC = open(oracle.SRC).read()


def _enum_fails(lib):
    H = np.full((2, 3), 2, dtype=np.uint8)
    try:
        f = oracle.Film(H, 2, seed=5, lib=lib)
        ex = f.exact(4.0, 0.3)
        _, ser = f.run([4.0], [0.3], [0], [100000], series=True)
    except oracle.OracleError:
        return True
    M = ser[2000:, 0].astype(float)
    B = ser[2000:, 1].astype(float)
    E = -B - 0.3 * M
    for x, e in ((M, ex["M"]), (E, ex["E"]), (M * M, ex["M2"])):
        b = x[: (len(x) // 50) * 50].reshape(50, -1).mean(axis=1)
        if abs(x.mean() - e) > 5 * b.std(ddof=1) / math.sqrt(50) + 1e-9:
            return True
    return False


def _stencil_fails(lib):
    from tests.test_oracle_lattice import cartesian_neighbours
    try:
        f = oracle.Film(np.full((4, 5, ), 3, dtype=np.uint8), 3, lib=lib)
    except oracle.OracleError:
        return True
    ref = cartesian_neighbours(4, 5, 3, 0)
    return any(set(f.neighbours(*s)) != want for s, want in ref.items())


def _colouring_fails(lib):
    try:
        f = oracle.Film(np.full((6, 6), 3, dtype=np.uint8), 3, flags=3, lib=lib)
    except oracle.OracleError as e:
        return e.code == -4
    return f.check_colouring() != 0


def _bookkeeping_fails(lib):
    f = oracle.Film(np.full((6, 6), 3, dtype=np.uint8), 3, flags=3, seed=2, lib=lib)
    try:
        f.run([3.0], [0.2], [0], [20])
    except oracle.OracleError as e:
        return e.code == -7
    return False


def _threshold_fails(lib):
    from tests.test_oracle_rng_table import _count_exact
    for T in (0.5, 2.0, 7.0):
        for n in range(-12, 13):
            for s in (-1, 1):
                dE = 2.0 * s * (n + 0.1)
                thr = oracle.threshold(T, 0.1, 1.0, n, s, lib=lib)
                want = oracle.ALWAYS if dE <= 0 else _count_exact(math.exp(-dE / T))
                if want >= (1 << 32) - 1:
                    want = oracle.ALWAYS
                if thr != want:
                    return True
    return False


def _measurement_fails(lib):
    f = oracle.Film(np.full((6, 6), 2, dtype=np.uint8), 2, seed=2, lib=lib)
    recs, ser = f.run([2.0], [0.0], [4], [10], series=True)
    return recs[0]["n_meas"] != 10 or recs[0]["sumM"] != int(ser[4:, 0].sum())


def _gate_fails(lib):
    from tests.test_oracle_dynamics import _gate_count
    H = np.full((3, 4), 2, dtype=np.uint8)
    f = oracle.Film(H, 2, seed=3, lib=lib)
    for T, h_s in ((2.0, 1.0), (0.7, -0.35)):
        cnt = _gate_count(math.exp(-abs(h_s) / T))
        before = f.spins()
        f.run([T], [0.0], [0], [1], J=0.0, h_s=h_s)
        after = f.spins()
        sweep = f.info()["sweep"]
        for z in range(2):
            for y in range(3):
                for x in range(4):
                    passed = f.site_word(oracle.STREAM_GATE, sweep, x, y, z) < cnt
                    if (after[z, y, x] != before[z, y, x]) != passed:
                        return True
    return False


MUTANTS = [
    ("field sign in dE", "(J * (double)n + h)", "(J * (double)n - h)", _enum_fails),
    ("temperature dropped", "exp(-dE / T)", "exp(-dE)", _enum_fails),
    ("acceptance inverted", "accept = u < a;", "accept = u > a;", _enum_fails),
    ("neighbour sum counts sites", "n += f->spin[site_of(f, a, b, c)];", "n += 1;", _enum_fails),
    ("wrong down offset", "{ 1, 0,-1},", "{ 1, 0, 1},", _stencil_fails),
    ("transposed in-plane offset", "{ 1,-1, 0}, {-1, 1, 0},", "{ 1, 1, 0}, {-1,-1, 0},", _stencil_fails),
    ("colour ignores z", "return ((x + z) & 1) | (((y + z) & 1) << 1);", "return (x & 1) | ((y & 1) << 1);", _colouring_fails),
    ("bond update sign", "f->B += -2 * (int64_t)s * n;", "f->B += 2 * (int64_t)s * n;", _bookkeeping_fails),
    ("threshold rounding", "p * 4294967296.0 - 0.5", "p * 4294967296.0 + 0.5", _threshold_fails),
    ("measured window off by one", "if (t >= sweeps_eq[k])", "if (t > sweeps_eq[k])", _measurement_fails),
    ("temperature dropped from the gate", "exp(-a / T)", "exp(-a)", _gate_fails),
    ("gate exponent doubled", "exp(-a / T)", "exp(-2.0 * a / T)", _gate_fails),
    ("gate word compared the wrong way", "if (!(g < gate)) continue;", "if (!(g > gate)) continue;", _gate_fails),
]


@pytest.mark.parametrize("name,old,new,detect", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, name, old, new, detect):
    assert SRC.count(old) == 1, f"mutation anchor for '{name}' not found exactly once"
    src = tmp_path / "mutant.c"
    src.write_text(SRC.replace(old, new))
    # the mutant includes the oracle's own header from its directory
    (tmp_path / "isf_oracle.h").write_text(open(oracle.HDR).read())
    so = oracle.build(str(src), str(tmp_path / "libmutant.so"))
    lib = oracle.load(so)
    assert detect(lib), f"planted mistake '{name}' was not caught"


def test_planted_philox_constant_is_caught(tmp_path, torch_philox_bin):
    old = "const uint32_t M0 = 0xD2511F53u"
    assert SRC.count(old) == 1
    src = tmp_path / "mutant.c"
    src.write_text(SRC.replace(old, "const uint32_t M0 = 0xD2511F55u"))
    (tmp_path / "isf_oracle.h").write_text(open(oracle.HDR).read())
    lib = oracle.load(oracle.build(str(src), str(tmp_path / "libmutant.so")))
    rows = [(1, 2, 3, 4, 5, 6), (0, 0, 0, 0, 0, 0)]
    ref = torch_philox_blocks(torch_philox_bin, rows)
    assert any(not np.array_equal(oracle.philox(r[2:], r[:2], lib=lib), e) for r, e in zip(rows, ref))
