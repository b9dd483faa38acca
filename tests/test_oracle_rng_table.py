"""Oracle pins: the Philox4x32-10 generator and the Eq. 8 threshold table.

- Philox is checked against PyTorch's own header-only Philox4x32-10 engine (an independent
  implementation of the SC'11 generator), on edge and random counters/keys.
- The threshold is checked against its defining inequality with exact rational arithmetic,
  and against the limits Eq. 8 fixes (dE <= 0 always accepted, T = inf always, T = 0 never).
- The Eq. 9 gate threshold is checked the same way against exp(-|h_s| / T), with its limits
  (h_s = 0 and T = inf always pass, T = 0 never) and closed-form values e^-1, e^-1/2.
"""
from fractions import Fraction
import math

import numpy as np
import pytest

from oracle import oracle
from tests.conftest import torch_philox_blocks

ALWAYS = oracle.ALWAYS


def test_philox_matches_pytorch_engine(olib, torch_philox_bin):
    rng = np.random.Generator(np.random.PCG64(7))
    rows = [(0, 0, 0, 0, 0, 0), (2**32 - 1,) * 6, (1, 0, 0, 0, 0, 0), (0, 0, 0, 0, 0, 1)]
    rows += [tuple(int(v) for v in rng.integers(0, 2**32, size=6, dtype=np.uint64)) for _ in range(300)]
    ref = torch_philox_blocks(torch_philox_bin, rows)
    for r, exp in zip(rows, ref):
        got = oracle.philox(r[2:], r[:2], lib=olib)
        assert np.array_equal(got, exp), (r, got, exp)


def test_site_word_keying(olib):
    """The site -> (counter, word) map is the convention the whole build shares:
    q = ((c*L + z)*ceil(R/2) + y//2)*ceil(ceil(C/2)/4) + (x//2)//4, word (x//2) % 4."""
    H = np.full((7, 9), 5, dtype=np.uint8)
    f = oracle.Film(H, 5, seed=0x1234_5678_9ABC_DEF0, lib=olib)
    R, Cc, L = 7, 9, 5
    Rh, Ch = (R + 1) // 2, (Cc + 1) // 2
    Qw = (Ch + 3) // 4
    for (x, y, z, sweep, stream) in [(0, 0, 0, 1, 0), (8, 6, 4, 2**33 + 5, 0), (3, 2, 1, 0, 2), (5, 1, 3, 77, 1)]:
        c = ((x + z) & 1) | (((y + z) & 1) << 1)
        q = ((c * L + z) * Rh + y // 2) * Qw + (x // 2) // 4
        blk = oracle.philox([q, sweep & 0xFFFFFFFF, sweep >> 32, stream],
                            [0x9ABCDEF0, 0x12345678], lib=olib)
        assert f.site_word(stream, sweep, x, y, z) == int(blk[(x // 2) % 4])


def _count_exact(p: float) -> int:
    """#{u in [0, 2^32): (u + 1/2) / 2^32 < p}, by exact rational arithmetic."""
    P = Fraction(p) * (1 << 32) - Fraction(1, 2)
    if P <= 0:
        return 0
    n = math.ceil(P)
    return min(n, 1 << 32)


@pytest.mark.parametrize("T", [0.25, 0.5, 1.0, 2.0, 3.0, 7.3, 12.0, 1e3])
@pytest.mark.parametrize("h", [0.0, 0.1, -0.35, 2.0, -8.0])
def test_threshold_definition(olib, T, h):
    J = 1.0
    for n in range(-12, 13):
        for s in (-1, 1):
            thr = oracle.threshold(T, h, J, n, s, lib=olib)
            dE = 2.0 * s * (J * n + h)
            if dE <= 0:
                assert thr == ALWAYS
                continue
            cnt = _count_exact(math.exp(-dE / T))
            if cnt >= (1 << 32) - 1:
                assert thr == ALWAYS
            else:
                assert thr == cnt
                # the defining inequality at the boundary words
                p = Fraction(math.exp(-dE / T))
                if thr > 0:
                    assert (Fraction(thr - 1) + Fraction(1, 2)) / (1 << 32) < p
                assert (Fraction(thr) + Fraction(1, 2)) / (1 << 32) >= p


def test_threshold_limits(olib):
    inf = float("inf")
    for n in range(-12, 13):
        for s in (-1, 1):
            assert oracle.threshold(inf, 0.7, 1.0, n, s, lib=olib) == ALWAYS      # T = inf: p = 1
            dE = 2.0 * s * (n + 0.7)
            want = ALWAYS if dE <= 0 else 0                                      # T = 0: exp(-inf) = 0
            assert oracle.threshold(0.0, 0.7, 1.0, n, s, lib=olib) == want
    # monotone: a larger energy cost is never accepted more often
    T = 2.5
    costs = sorted({2.0 * s * (n + 0.3) for n in range(-12, 13) for s in (-1, 1)})
    vals = [oracle.threshold(T, 0.3, 1.0, *_ns_for(dE)) for dE in costs]
    pos = [v for d, v in zip(costs, vals) if d > 0]
    assert all(a >= b for a, b in zip(pos, pos[1:]))


def _ns_for(dE):
    for n in range(-12, 13):
        for s in (-1, 1):
            if 2.0 * s * (n + 0.3) == dE:
                return n, s
    raise AssertionError


def test_threshold_table_matches_probability(olib):
    """thr / 2^32 is the Metropolis probability to within 2^-32."""
    T, h = 3.0, -0.4
    tab = oracle.threshold_table(T, h, lib=olib)
    for n in range(-12, 13):
        for sp, s in ((0, -1), (1, 1)):
            dE = 2.0 * s * (n + h)
            p = 1.0 if dE <= 0 else math.exp(-dE / T)
            t = int(tab[n + 12, sp])
            approx = 1.0 if t == ALWAYS else t / 2.0**32
            assert abs(approx - p) <= 2.0**-32 + 1e-15


@pytest.mark.parametrize("T", [0.3, 1.0, 2.0, 4.5, 8.0, 1e3])
@pytest.mark.parametrize("h_s", [0.0, 0.25, -1.0, 2.0, 4.0, -8.0, 1e3])
def test_gate_threshold_definition(olib, T, h_s):
    """Eq. 9 gate (items 4-5 of Sec. 5): it passes with probability exp(-|S_i h_s| / T), |S_i| = 1,
    encoded like Eq. 8: g passes iff g < thr, thr = #{g : (g + 1/2) 2^-32 < p}, counts of 2^32 - 1
    or more stored as ALWAYS; h_s = 0 means no gate (p = 1)."""
    thr = oracle.gate_threshold(T, h_s, lib=olib)
    cnt = _count_exact(math.exp(-abs(h_s) / T))
    if cnt >= (1 << 32) - 1:
        assert thr == ALWAYS
    else:
        assert thr == cnt
        p = Fraction(math.exp(-abs(h_s) / T))
        if thr > 0:
            assert (Fraction(thr - 1) + Fraction(1, 2)) / (1 << 32) < p
        assert (Fraction(thr) + Fraction(1, 2)) / (1 << 32) >= p
    # the sign of the switching field does not matter (|S_i h_s|)
    assert oracle.gate_threshold(T, -h_s, lib=olib) == thr


def test_gate_threshold_limits(olib):
    inf = float("inf")
    for h_s in (0.5, 3.0, -7.0):
        assert oracle.gate_threshold(inf, h_s, lib=olib) == ALWAYS      # T = inf: p = 1
        assert oracle.gate_threshold(0.0, h_s, lib=olib) == 0           # T = 0: p = exp(-inf) = 0
    assert oracle.gate_threshold(0.0, 0.0, lib=olib) == ALWAYS          # h_s = 0: no gate at any T
    assert oracle.gate_threshold(2.0, 0.0, lib=olib) == ALWAYS
    # e^-1 and e^-1/2 as fractions of 2^32 (closed forms, independent of the oracle's rounding)
    assert abs(oracle.gate_threshold(2.0, 2.0, lib=olib) / 2.0**32 - math.exp(-1.0)) <= 2.0**-32
    assert abs(oracle.gate_threshold(4.0, -2.0, lib=olib) / 2.0**32 - math.exp(-0.5)) <= 2.0**-32
    # a larger switching field never lets the gate pass more often
    vals = [oracle.gate_threshold(3.0, a, lib=olib) for a in (0.1, 0.5, 1.0, 2.0, 5.0, 20.0)]
    assert all(a >= b for a, b in zip(vals, vals[1:]))
