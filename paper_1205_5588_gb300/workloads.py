"""Seeded synthetic inputs: height maps and schedules.

Holds none of the method's arithmetic (no lattice, no Metropolis, no thresholds): it only
makes the inputs that the CUDA path and the CPU oracle are both fed.  The paper builds its
films from STM/AFM images that are not available; a seeded fractal Gaussian random field,
quantised to a range of Co layer counts, stands in for them (Sec. 2: "the image pixels were
used to construct a magnet with a given number of atomic layers").
"""
from __future__ import annotations

import math

import numpy as np


def fractal_heights(rows: int, cols: int, hurst: float, lo: int, hi: int, seed: int) -> np.ndarray:
    """Spectral synthesis of a fractal Gaussian field (amplitude ~ |k|^-(H+1), numpy PCG64(seed)),
    quantised in equal-width bins to integer layer counts lo..hi.  Returns uint8 (rows, cols)."""
    if rows < 1 or cols < 1 or not (0 <= lo <= hi <= 255):
        raise ValueError("bad height-map shape or layer range")
    rng = np.random.Generator(np.random.PCG64(seed))
    ky = np.fft.fftfreq(rows)[:, None]
    kx = np.fft.fftfreq(cols)[None, :]
    k = np.sqrt(kx * kx + ky * ky)
    with np.errstate(divide="ignore"):
        amp = np.where(k > 0, k ** (-(hurst + 1.0)), 0.0)
    noise = rng.standard_normal((rows, cols)) + 1j * rng.standard_normal((rows, cols))
    f = np.fft.ifft2(noise * amp).real
    fmin, fmax = float(f.min()), float(f.max())
    if fmax <= fmin:
        return np.full((rows, cols), lo, dtype=np.uint8)
    span = hi - lo
    q = np.floor((f - fmin) / (fmax - fmin) * (span + 1)).astype(np.int64)
    q = lo + np.minimum(span, q)
    return q.astype(np.uint8)


def flat_heights(rows: int, cols: int, layers: int) -> np.ndarray:
    return np.full((rows, cols), layers, dtype=np.uint8)


def loop_fields(h_max_num: int, denom: int) -> np.ndarray:
    """Hysteresis loop +h_max -> -h_max -> +h_max in steps of 1/denom, from integer step
    indices (never accumulated): h_max = h_max_num / denom."""
    down = [(h_max_num - k) / denom for k in range(0, 2 * h_max_num + 1)]
    up = [(-h_max_num + k) / denom for k in range(1, 2 * h_max_num + 1)]
    return np.array(down + up, dtype=np.float64)


def schedule(T, h, sweeps_eq, sweeps_meas) -> dict:
    n = max(np.size(T), np.size(h), np.size(sweeps_eq), np.size(sweeps_meas))
    T = np.broadcast_to(np.asarray(T, dtype=np.float64), (n,)).copy()
    h = np.broadcast_to(np.asarray(h, dtype=np.float64), (n,)).copy()
    eq = np.broadcast_to(np.asarray(sweeps_eq, dtype=np.int32), (n,)).copy()
    me = np.broadcast_to(np.asarray(sweeps_meas, dtype=np.int32), (n,)).copy()
    return {"T": T, "h": h, "eq": eq, "meas": me}


# --------------------------------------------------------------------------- workloads ----
# Flat 16x16 x 3 film, periodic in-plane, int8 spins from seed 1, T = 3:
# hysteresis h = +4 -> -4 -> +4 in steps of 0.1 (161 steps), 100 sweeps per step.
def flat16_hysteresis() -> dict:
    h = loop_fields(40, 10)
    return {
        "name": "flat16x16x3_hysteresis",
        "heights": flat_heights(16, 16, 3), "layers": 3,
        "periodic_x": True, "periodic_y": True, "packed": False, "seed": 1, "init": "random",
        "schedule": schedule(3.0, h, 0, 100), "J": 1.0,
    }


# 256x256 fractal map (Hurst 0.7, generator seed 2) quantised to 1..6 layers, open edges, int8
# spins from seed 1; T = 0.5 .. 12 in 48 linear steps at h = 0, 2000 + 2000 sweeps per step.
def fractal256_tscan(eq: int = 2000, meas: int = 2000, nsteps: int = 48) -> dict:
    T = np.array([0.5 + k * 11.5 / 47.0 for k in range(48)], dtype=np.float64)[:nsteps]
    return {
        "name": "fractal256x256x6_tscan",
        "heights": fractal_heights(256, 256, 0.7, 1, 6, seed=2), "layers": 6,
        "periodic_x": False, "periodic_y": False, "packed": False, "seed": 1, "init": "random",
        "schedule": schedule(T, 0.0, eq, meas), "J": 1.0,
    }


# 2048x2048 fractal map (Hurst 0.8, seed 3) quantised to 2..6 layers, bit-packed spins,
# all up at the start; T = 2, h = +8 -> -8 -> +8 in steps of 0.05 (641 steps), 200 sweeps each.
def fractal2048_hysteresis(sweeps: int = 200) -> dict:
    h = loop_fields(160, 20)
    return {
        "name": "fractal2048x2048x6_hysteresis",
        "heights": fractal_heights(2048, 2048, 0.8, 2, 6, seed=3), "layers": 6,
        "periodic_x": False, "periodic_y": False, "packed": True, "seed": 1, "init": "up",
        "schedule": schedule(2.0, h, 0, sweeps), "J": 1.0,
    }


def periodic_cube(L: int) -> dict:
    """Full L x L x L cube, periodic on all three axes (bulk FCC, for the Curie-point check)."""
    return {"heights": flat_heights(L, L, L), "layers": L, "flags_xyz": (True, True, True)}


# Batched films: widths and heights uniform in 64..1024, layers 1..8, Hurst 0.5..0.9, each
# film with its own T in 1..10 and a loop +h_max -> -h_max -> +h_max (h_max in 2..8) of
# 40..200 steps, 100 sweeps per step (film i: seed 1000 + i).
def batch_films(n: int = 512, seed: int = 4, sweeps_per_step: int = 100, side=(64, 1024),
                steps=(40, 200)) -> list[dict]:
    rng = np.random.Generator(np.random.PCG64(seed))
    films = []
    for i in range(n):
        R = int(rng.integers(side[0], side[1] + 1))
        Cc = int(rng.integers(side[0], side[1] + 1))
        L = int(rng.integers(1, 9))
        hurst = float(rng.uniform(0.5, 0.9))
        T = float(rng.uniform(1.0, 10.0))
        h_max = float(rng.uniform(2.0, 8.0))
        nst = int(rng.integers(steps[0], steps[1] + 1))
        half = nst // 2
        ks = np.arange(nst)
        # triangular loop sampled at nst points from integer indices
        h = np.where(ks <= half, h_max * (1.0 - 2.0 * ks / max(half, 1)),
                     -h_max + 2.0 * h_max * (ks - half) / max(nst - 1 - half, 1))
        films.append({
            "name": f"batch{i}", "heights": fractal_heights(R, Cc, hurst, 1, L, seed=1000 + i),
            "layers": L, "periodic_x": False, "periodic_y": False, "seed": 1000 + i,
            "init": "random", "schedule": schedule(T, h, 0, sweeps_per_step), "J": 1.0,
        })
    return films


def poisson_arrivals(rate: float, duration: float, seed: int = 5) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    t, out = 0.0, []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration:
            break
        out.append(t)
    return np.array(out, dtype=np.float64)


def lognormal_side(rng: np.random.Generator, median: float = 256, sigma: float = 0.7,
                   lo: int = 64, hi: int = 2048) -> int:
    v = math.exp(math.log(median) + sigma * float(rng.standard_normal()))
    return int(min(hi, max(lo, round(v))))
