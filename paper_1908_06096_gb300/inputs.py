"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module holds no arithmetic of the transform itself: it only draws random
numbers in a fixed order and lays them out.  Both the CUDA path and the oracle
receive the arrays it returns.

Spectra: real and imaginary parts i.i.d. N(0, 1), scaled by (n + 1)^-p,
imaginary part of every m = 0 coefficient set to zero; draws come from
``numpy.random.default_rng(seed)`` in the order field -> m -> n -> (re, im),
which is the C order of the m-major triangular layout.
"""
from __future__ import annotations

import numpy as np


def nspec(T: int) -> int:
    return (T + 1) * (T + 2) // 2


def degree_of_index(T: int) -> np.ndarray:
    """n for every complex slot of the m-major triangular layout."""
    out = np.empty(nspec(T), dtype=np.int64)
    q = 0
    for m in range(T + 1):
        k = T - m + 1
        out[q:q + k] = np.arange(m, T + 1)
        q += k
    return out


def order_of_index(T: int) -> np.ndarray:
    """m for every complex slot of the m-major triangular layout."""
    out = np.empty(nspec(T), dtype=np.int64)
    q = 0
    for m in range(T + 1):
        k = T - m + 1
        out[q:q + k] = m
        q += k
    return out


def spectra(T: int, nfields: int, seed: int, p: float = 1.0, field0: int = 0) -> np.ndarray:
    """Random spectra as float64 [nfields, nspec(T), 2] (re, im interleaved).

    ``field0`` skips that many fields of the same seeded stream, so a subset of
    fields of a large batch can be regenerated without drawing the whole batch
    (each field consumes exactly nspec(T) * 2 normals).
    """
    rng = np.random.default_rng(seed)
    ns = nspec(T)
    if field0:
        rng.standard_normal(field0 * ns * 2)
    a = rng.standard_normal((nfields, ns, 2))
    n = degree_of_index(T)
    a *= ((n + 1.0) ** (-p))[None, :, None]
    m0 = order_of_index(T) == 0
    a[:, m0, 1] = 0.0
    return a


def grid_noise(npoints: int, nfields: int, seed: int) -> np.ndarray:
    """Unstructured N(0, 1) grid values [nfields, npoints] (not band-limited)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nfields, npoints))


MIXED_T = (79, 159, 255, 319, 511, 639)
SERVE_T = (63, 127, 255, 511, 1279)


def mixed_requests(n: int = 48, seed: int = 1003, max_fields: int = 256):
    """The mixed-truncation batch: T uniform over MIXED_T, grid regular
    ((T+1) x (2T+2)) or octahedral O(T+1), nfields uniform in [1, max_fields]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        T = int(rng.choice(MIXED_T))
        grid = "octahedral" if rng.integers(0, 2) else "regular"
        nf = int(rng.integers(1, max_fields + 1))
        out.append({"T": T, "grid": grid, "nfields": nf, "seed": seed * 1000 + i})
    return out


def serve_requests(n: int = 10000, seed: int = 1004, rate_hz: float = 1000.0, max_fields: int = 137,
                   choices=SERVE_T):
    """Poisson arrivals: T uniform over ``choices`` on regular grids, nfields
    uniform in [1, max_fields], direction inverse or direct with equal odds."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=n)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for i in range(n):
        out.append({
            "t": float(t[i]),
            "T": int(rng.choice(choices)),
            "nfields": int(rng.integers(1, max_fields + 1)),
            "direction": "inv" if rng.integers(0, 2) == 0 else "dir",
            "seed": seed * 100000 + i,
        })
    return out
