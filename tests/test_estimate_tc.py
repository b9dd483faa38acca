"""T_c estimate of a temperature scan (Sec. 4, Table 1; reading: the temperature of the largest
susceptibility chi' = (<M^2> - <|M|>^2) / (N T)).  The library's isf_estimate_tc is host only,
so it runs here on CPU: against hand-built records whose answer is known, and against the
oracle's or_estimate_tc on the oracle's own records of a scan."""
import numpy as np
import pytest

from oracle import oracle
from paper_1205_5588_gb300 import workloads as W


@pytest.fixture(scope="module")
def I():
    from paper_1205_5588_gb300 import build
    build.build()
    from paper_1205_5588_gb300 import isingfilm
    return isingfilm


def record(T, n, sumAbsM, sumM2, N=100):
    """One step record from its integer sums (the other fields do not enter the estimate)."""
    if n == 0:
        return {"T": T, "h": 0.0, "M_last": 0, "B_last": 0, "n_meas": 0, "sumM": 0, "sumAbsM": 0, "sumM2": 0,
                "sumB2": 0, "sumMB": 0, "sumB": 0, "m": float("nan"), "abs_m": float("nan"), "e": float("nan"),
                "chi": float("nan"), "chi_abs": float("nan"), "C": float("nan")}
    varA = (n * sumM2 - sumAbsM * sumAbsM) / (n * n)
    chi_abs = varA / (N * T) if T > 0 else float("inf")
    return {"T": T, "h": 0.0, "M_last": 0, "B_last": 0, "n_meas": n, "sumM": 0, "sumAbsM": sumAbsM,
            "sumM2": sumM2, "sumB2": 0, "sumMB": 0, "sumB": 0, "m": 0.0, "abs_m": sumAbsM / n / N, "e": 0.0,
            "chi": 0.0, "chi_abs": chi_abs, "C": 0.0}


def test_known_peak(I):
    # Var|M| = 0, 4, 9, 1 over temperatures 1, 2, 3, 4: chi' ~ 0, 2, 3, 0.25 -> peak at T = 3
    recs = [record(1.0, 4, 40, 400), record(2.0, 4, 40, 416), record(3.0, 4, 40, 436), record(4.0, 4, 40, 404)]
    assert I.estimate_tc(recs, with_index=True) == (3.0, 2)
    assert oracle.estimate_tc(recs) == (3.0, 2)


def test_skips_unmeasured_and_degenerate_steps(I):
    recs = [record(2.0, 0, 0, 0), record(0.0, 4, 40, 500), record(float("inf"), 4, 40, 500),
            record(5.0, 4, 40, 404), record(6.0, 4, 40, 404)]
    # steps without measured sweeps, at T = 0 or T = inf take no part; equal maxima: the first
    assert I.estimate_tc(recs, with_index=True) == (5.0, 3)
    assert oracle.estimate_tc(recs) == (5.0, 3)
    with pytest.raises(I.IsfError) as e:
        I.estimate_tc(recs[:3])
    assert e.value.code == -7
    assert oracle.estimate_tc(recs[:3]) == (None, -1)


def test_library_estimate_equals_oracle_on_a_scan(I):
    """A short temperature scan of a small fractal film in the oracle; both estimators pick the
    same step from the same records."""
    H = W.fractal_heights(12, 14, 0.7, 1, 3, seed=21)
    f = oracle.Film(H, 3, seed=4)
    T = np.linspace(2.0, 12.0, 11)
    recs, _ = f.run(T, np.zeros_like(T), [40] * len(T), [200] * len(T))
    got = I.estimate_tc(recs, with_index=True)
    want = oracle.estimate_tc(recs)
    assert got == want
    assert 2.0 <= got[0] <= 12.0
    # the chosen step is the chi' maximum by the records' own derived values
    assert got[1] == int(np.argmax([r["chi_abs"] for r in recs]))
