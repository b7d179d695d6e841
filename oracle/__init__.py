"""Plain FP64 CPU oracle for the spherical-harmonic transform (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only users.  The library under
``paper_1908_06096_gb300`` never imports this package, and this package never
imports the library: the two share nothing but the seeded input generators.

Every function follows the plain definitions stated in ``sht_oracle.c``:
the synthesis equation of ESCAPE D3.3 section 4.4.1 (repeated in 4.4.2), and
the forward direction as inner products with the basis functions (section
4.4.2), with Gaussian quadrature in latitude.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sht_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no fast-math, no FMA contraction
    so that x86 and Arm hosts round the same way)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
            "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm",
        ])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.or_nspec.restype = ctypes.c_long
            lib.or_nspec.argtypes = [ctypes.c_int]
            lib.or_grid_rows.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _I]
            lib.or_gauss.argtypes = [ctypes.c_int, _D, _D]
            lib.or_legendre.argtypes = [ctypes.c_int, ctypes.c_double, _D]
            lib.or_max_threads.restype = ctypes.c_int
            lib.or_inv_fourier.argtypes = [ctypes.c_int, ctypes.c_int, _I, _D, _D,
                                           ctypes.c_int, _D, ctypes.c_int]
            lib.or_inv_grid_from_fourier.argtypes = [ctypes.c_int, ctypes.c_int, _I, _D,
                                                     ctypes.c_int, _D, ctypes.c_int]
            lib.or_inv_trans.argtypes = [ctypes.c_int, ctypes.c_int, _I, _D, _D,
                                         ctypes.c_int, _D, ctypes.c_int]
            lib.or_dir_fourier.argtypes = [ctypes.c_int, ctypes.c_int, _I, _D,
                                           ctypes.c_int, _D, ctypes.c_int]
            lib.or_dir_spec_from_fourier.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D,
                                                     ctypes.c_int, _D, ctypes.c_int]
            lib.or_dir_trans.argtypes = [ctypes.c_int, ctypes.c_int, _I, _D, _D, _D,
                                         ctypes.c_int, _D, ctypes.c_int]
            lib.or_legendre_deriv.argtypes = [ctypes.c_int, ctypes.c_double, _D]
            lib.or_inv_trans_deriv.argtypes = [ctypes.c_int, ctypes.c_int, _I, _D, _D, ctypes.c_int,
                                               _D, _D, ctypes.c_int]
            lib.or_inv_trans_uv.argtypes = [ctypes.c_int, ctypes.c_int, _I, _D, _D, _D, ctypes.c_int,
                                            _D, _D, ctypes.c_int]
            lib.or_dir_trans_vordiv.argtypes = [ctypes.c_int, ctypes.c_int, _I, _D, _D, _D, _D,
                                                ctypes.c_int, _D, _D, ctypes.c_int]
            _lib = lib
    return _lib


class use_library:
    """Context manager that points the wrappers at another build of the
    oracle source (used by the tests that plant a mistake in a copy of the
    oracle and check that a pin catches it)."""

    def __init__(self, path: str):
        self.path = path
        self.saved = None

    def __enter__(self):
        global _lib
        _load()
        self.saved = _lib
        lib = ctypes.CDLL(self.path)
        for fn in ("or_nspec", "or_grid_rows", "or_gauss", "or_legendre", "or_max_threads",
                   "or_inv_fourier", "or_inv_grid_from_fourier", "or_inv_trans",
                   "or_dir_fourier", "or_dir_spec_from_fourier", "or_dir_trans",
                   "or_legendre_deriv", "or_inv_trans_deriv", "or_inv_trans_uv", "or_dir_trans_vordiv"):
            src = getattr(self.saved, fn)
            dst = getattr(lib, fn)
            dst.argtypes = src.argtypes
            dst.restype = src.restype
        with _lock:
            _lib = lib
        return self

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self.saved
        return False


def build_variant(source_text: str, out_path: str) -> str:
    """Compile a modified copy of the oracle source (tests only)."""
    src = out_path + ".c"
    with open(src, "w") as fh:
        fh.write(source_text)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                           "-ffp-contract=off", src, "-o", out_path, "-lm"])
    return out_path


def source_text() -> str:
    with open(_SRC) as fh:
        return fh.read()


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _ip(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(_I)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def nspec(T: int) -> int:
    """Number of complex coefficients for triangular truncation T."""
    return int(_load().or_nspec(T))


def spec_index(T: int, m: int, n: int) -> int:
    """Complex index of (m, n) in the m-major triangular layout."""
    return m * (T + 1) - m * (m - 1) // 2 + (n - m)


def max_threads() -> int:
    return int(_load().or_max_threads())


def grid_rows(kind: str, nlat: int, nlon: int = 0) -> np.ndarray:
    """Row lengths north to south; kind 'regular' or 'octahedral'."""
    rows = np.zeros(nlat, dtype=np.int32)
    _check(_load().or_grid_rows(0 if kind == "regular" else 1, nlat, nlon, _ip(rows)), "grid_rows")
    return rows


def gauss(nlat: int):
    """Gauss-Legendre nodes mu (north to south) and weights w."""
    mu = np.zeros(nlat)
    w = np.zeros(nlat)
    _check(_load().or_gauss(nlat, _dp(mu), _dp(w)), "gauss")
    return mu, w


def legendre(T: int, mu: float) -> np.ndarray:
    """All Pbar_n^m(mu), n <= T, in the triangular spectral order."""
    P = np.zeros(nspec(T))
    _check(_load().or_legendre(T, float(mu), _dp(P)), "legendre")
    return P


def _spec_arr(spec: np.ndarray, T: int) -> np.ndarray:
    """Accept complex [nf, nspec] or real [nf, nspec, 2]; return float64 [nf, nspec, 2]."""
    if np.iscomplexobj(spec):
        spec = np.stack([spec.real, spec.imag], axis=-1)
    spec = np.ascontiguousarray(spec, dtype=np.float64)
    assert spec.shape[-2:] == (nspec(T), 2), spec.shape
    return spec.reshape(-1, nspec(T), 2)


def inv_fourier(T, rows, mu, spec, nthreads=0):
    """F_m(mu_j) for every row: [nf, nlat, T+1] complex (zero for m > M_j)."""
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    s = _spec_arr(spec, T)
    nf, nlat = s.shape[0], len(rows)
    out = np.zeros((nf, nlat, T + 1, 2))
    _check(_load().or_inv_fourier(T, nlat, _ip(rows), _dp(mu), _dp(s), nf, _dp(out), nthreads),
           "inv_fourier")
    return out[..., 0] + 1j * out[..., 1]


def inv_grid_from_fourier(T, rows, four, nthreads=0):
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    four = np.ascontiguousarray(np.stack([four.real, four.imag], -1), dtype=np.float64)
    nf, nlat = four.shape[0], len(rows)
    out = np.zeros((nf, int(rows.sum())))
    _check(_load().or_inv_grid_from_fourier(T, nlat, _ip(rows), _dp(four), nf, _dp(out), nthreads),
           "inv_grid_from_fourier")
    return out


def inv_trans(T, rows, mu, spec, nthreads=0):
    """Grid [nf, sum(rows)] from spectra ([nf, nspec] complex or [nf, nspec, 2])."""
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    s = _spec_arr(spec, T)
    nf, nlat = s.shape[0], len(rows)
    out = np.zeros((nf, int(rows.sum())))
    _check(_load().or_inv_trans(T, nlat, _ip(rows), _dp(mu), _dp(s), nf, _dp(out), nthreads),
           "inv_trans")
    return out


def dir_fourier(T, rows, grid, nthreads=0):
    """F_m(mu_j) of every row by the direct DFT: [nf, nlat, T+1] complex."""
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    g = np.ascontiguousarray(grid, dtype=np.float64).reshape(-1, int(rows.sum()))
    nf, nlat = g.shape[0], len(rows)
    out = np.zeros((nf, nlat, T + 1, 2))
    _check(_load().or_dir_fourier(T, nlat, _ip(rows), _dp(g), nf, _dp(out), nthreads), "dir_fourier")
    return out[..., 0] + 1j * out[..., 1]


def dir_spec_from_fourier(T, mu, w, four, nthreads=0):
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    four = np.ascontiguousarray(np.stack([four.real, four.imag], -1), dtype=np.float64)
    nf, nlat = four.shape[0], four.shape[1]
    out = np.zeros((nf, nspec(T), 2))
    _check(_load().or_dir_spec_from_fourier(T, nlat, _dp(mu), _dp(w), _dp(four), nf, _dp(out),
                                            nthreads), "dir_spec_from_fourier")
    return out[..., 0] + 1j * out[..., 1]


def dir_trans(T, rows, mu, w, grid, nthreads=0):
    """Spectra [nf, nspec] complex from a grid [nf, sum(rows)]."""
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    g = np.ascontiguousarray(grid, dtype=np.float64).reshape(-1, int(rows.sum()))
    nf, nlat = g.shape[0], len(rows)
    out = np.zeros((nf, nspec(T), 2))
    _check(_load().or_dir_trans(T, nlat, _ip(rows), _dp(mu), _dp(w), _dp(g), nf, _dp(out), nthreads),
           "dir_trans")
    return out[..., 0] + 1j * out[..., 1]


# ---------------------------------------------------------------- derivatives
# Readings: unit sphere, phi the latitude (mu = sin phi); H_n^m = (1 - mu^2)
# dPbar_n^m/dmu; wind images U = u cos(phi), V = v cos(phi).

def legendre_deriv(T: int, mu: float) -> np.ndarray:
    """All H_n^m(mu) = (1 - mu^2) dPbar_n^m/dmu, n <= T, triangular order."""
    H = np.zeros(nspec(T))
    _check(_load().or_legendre_deriv(T, float(mu), _dp(H)), "legendre_deriv")
    return H


def inv_trans_deriv(T, rows, mu, spec, nthreads=0):
    """(dF/dlambda, (1 - mu^2) dF/dmu) on the grid, each [nf, sum(rows)]."""
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    s = _spec_arr(spec, T)
    nf, nlat = s.shape[0], len(rows)
    a = np.zeros((nf, int(rows.sum())))
    b = np.zeros((nf, int(rows.sum())))
    _check(_load().or_inv_trans_deriv(T, nlat, _ip(rows), _dp(mu), _dp(s), nf, _dp(a), _dp(b), nthreads),
           "inv_trans_deriv")
    return a, b


def inv_trans_uv(T, rows, mu, vor, div, nthreads=0):
    """Wind images (U, V) = (u cos phi, v cos phi) from vorticity and divergence spectra."""
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    z = _spec_arr(vor, T)
    d = _spec_arr(div, T)
    nf, nlat = z.shape[0], len(rows)
    U = np.zeros((nf, int(rows.sum())))
    V = np.zeros((nf, int(rows.sum())))
    _check(_load().or_inv_trans_uv(T, nlat, _ip(rows), _dp(mu), _dp(z), _dp(d), nf, _dp(U), _dp(V), nthreads),
           "inv_trans_uv")
    return U, V


def dir_trans_vordiv(T, rows, mu, w, U, V, nthreads=0):
    """Vorticity and divergence spectra ([nf, nspec] complex each) from wind images U, V."""
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    npts = int(rows.sum())
    U = np.ascontiguousarray(U, dtype=np.float64).reshape(-1, npts)
    V = np.ascontiguousarray(V, dtype=np.float64).reshape(-1, npts)
    nf, nlat = U.shape[0], len(rows)
    z = np.zeros((nf, nspec(T), 2))
    d = np.zeros((nf, nspec(T), 2))
    _check(_load().or_dir_trans_vordiv(T, nlat, _ip(rows), _dp(mu), _dp(w), _dp(U), _dp(V), nf, _dp(z), _dp(d),
                                       nthreads), "dir_trans_vordiv")
    return z[..., 0] + 1j * z[..., 1], d[..., 0] + 1j * d[..., 1]
