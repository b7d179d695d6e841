"""Pins of the FP64 oracle against what the mathematics fixes (no GPU).

The paper (ESCAPE D3.3, section 4.4.1, synthesis equation) prints no worked
example, so every pin here is a closed form, an invariant, a library special
case or a brute force on tiny inputs.  Each is chosen so that a plausible slip
in the oracle (a dropped term, a wrong sign, a swapped index, a wrong
normalisation) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

from paper_1908_06096_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLD, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([c.strip() for c in line.split("|")])
    return rows


def _ev(expr, **kw):
    env = {"sqrt": math.sqrt}
    env.update(kw)
    return float(eval(expr, {"__builtins__": {}}, env))


# ---------------------------------------------------------------- nodes, weights

@pytest.mark.parametrize("nlat", [2, 3, 4, 5, 8, 32, 160, 640, 1280, 2560])
def test_weights_sum_to_two(oracle_mod, nlat):
    mu, w = oracle_mod.gauss(nlat)
    assert abs(w.sum() - 2.0) <= 1e-14 * nlat
    assert np.all(w > 0)
    assert np.all(np.diff(mu) < 0), "nodes must run north to south"
    assert np.allclose(mu, -mu[::-1], atol=0, rtol=0)


@pytest.mark.parametrize("nlat", [4, 7, 32, 160])
def test_quadrature_exact_for_even_powers(oracle_mod, nlat):
    mu, w = oracle_mod.gauss(nlat)
    for k in range(0, nlat):          # degree 2k <= 2 nlat - 2
        got = float(np.sum(w * mu ** (2 * k)))
        assert abs(got - 2.0 / (2 * k + 1)) < 1e-13, (nlat, k)
    # odd moments vanish by symmetry
    assert abs(float(np.sum(w * mu ** 3))) < 1e-15


def test_gauss_closed_forms(oracle_mod):
    rows = _golden("gauss_legendre_closed_forms.txt")
    for nlat in sorted({int(r[0]) for r in rows}):
        mu, w = oracle_mod.gauss(nlat)
        for r in rows:
            if int(r[0]) != nlat:
                continue
            x, wx = _ev(r[1]), _ev(r[2])
            j = int(np.argmin(np.abs(mu - x)))
            assert abs(mu[j] - x) < 1e-15, (nlat, x, mu[j])
            assert abs(w[j] - wx) < 1e-15, (nlat, wx, w[j])


# ---------------------------------------------------------------- Legendre values

def test_low_degree_closed_forms(oracle_mod):
    T = 3
    for x in (0.93, 0.31, -0.57, 0.0, 0.999):
        P = oracle_mod.legendre(T, x)
        s = math.sqrt(1 - x * x)
        for n, m, expr in _golden("legendre_low_degree.txt"):
            n, m = int(n), int(m)
            want = _ev(expr, mu=x, s=s)
            got = P[oracle_mod.spec_index(T, m, n)]
            assert abs(got - want) < 1e-15, (n, m, x, got, want)


def test_rodrigues_brute_force(oracle_mod):
    """Exact Rodrigues formula (sympy), evaluated at 50 digits, for n, m <= 8."""
    sympy = pytest.importorskip("sympy")
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    xs = sympy.symbols("x")
    T = 8
    pts = [mp.mpf("0.8"), mp.mpf("-0.35"), mp.mpf("0.0625"), mp.mpf("0.999")]
    for n in range(T + 1):
        Pn = sympy.legendre(n, xs)
        for m in range(n + 1):
            dm = sympy.diff(Pn, xs, m) if m else Pn
            f = sympy.lambdify(xs, dm, modules="mpmath")
            norm = mp.sqrt(mp.mpf(2 * n + 1) / 2 * mp.factorial(n - m) / mp.factorial(n + m))
            for x in pts:
                exact = norm * (1 - x * x) ** (mp.mpf(m) / 2) * f(x)
                got = oracle_mod.legendre(T, float(x))[oracle_mod.spec_index(T, m, n)]
                assert abs(got - float(exact)) < 2e-14, (n, m, float(x), got, float(exact))


@pytest.mark.parametrize("T,nlat", [(31, 32), (159, 160)])
def test_discrete_orthonormality(oracle_mod, T, nlat):
    mu, w = oracle_mod.gauss(nlat)
    P = np.stack([oracle_mod.legendre(T, x) for x in mu])     # [nlat, nspec]
    for m in sorted({0, 1, 2, T // 3, T // 2, T - 1, T}):
        cols = [oracle_mod.spec_index(T, m, n) for n in range(m, T + 1)]
        Pm = P[:, cols]
        G = Pm.T @ (w[:, None] * Pm)
        assert np.max(np.abs(G - np.eye(len(cols)))) < 1e-13, m


@pytest.mark.parametrize("x", [0.99, 0.5, 0.0, -0.73])
def test_addition_theorem(oracle_mod, x):
    """(Pbar_n^0)^2 + 2 sum_{m>=1} (Pbar_n^m)^2 = (2n+1)/2 at every mu."""
    T = 200
    P = oracle_mod.legendre(T, x)
    for n in (0, 1, 5, 50, 137, 200):
        tot = P[oracle_mod.spec_index(T, 0, n)] ** 2
        tot += 2 * sum(P[oracle_mod.spec_index(T, m, n)] ** 2 for m in range(1, n + 1))
        assert abs(tot - (2 * n + 1) / 2) < 1e-12 * (2 * n + 1), (n, tot)


def test_high_order_polar_values_extended_range(oracle_mod):
    """At T1279 next to the pole, the FP64 recurrence agrees with the same
    values carried in 40-digit arithmetic with unbounded exponent range wherever
    they are above 1e-290, and is tiny wherever the exact value is.  The
    relative bound 1e-10 allows for the forward recurrence's rounding growth
    over ~1300 steps (about n * eps times a small cancellation factor)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    T = 1279
    mu, _ = oracle_mod.gauss(2 * (T + 1))
    x = mp.mpf(float(mu[0]))
    P = oracle_mod.legendre(T, float(mu[0]))
    s = mp.sqrt((1 - x) * (1 + x))
    pmm = 1 / mp.sqrt(2)
    for m in range(0, T + 1):
        if m:
            pmm = mp.sqrt(mp.mpf(2 * m + 1) / (2 * m)) * s * pmm
        if m % 97:
            continue
        p0, p1 = pmm, mp.sqrt(2 * m + 3) * x * pmm
        vals = {m: p0, m + 1: p1}
        for n in range(m + 2, T + 1):
            a = mp.sqrt(mp.mpf(4 * n * n - 1) / (n * n - m * m))
            b = mp.sqrt(mp.mpf((n - 1) ** 2 - m * m) / (4 * (n - 1) ** 2 - 1))
            p0, p1 = p1, a * (x * p1 - b * p0)
            vals[n] = p1
        for n in range(m, T + 1, 61):
            exact = vals[n]
            got = P[oracle_mod.spec_index(T, m, n)]
            if abs(exact) > mp.mpf("1e-290"):
                assert abs(got - float(exact)) <= 1e-10 * float(abs(exact)), (m, n)
            else:
                assert abs(got) < 1e-280, (m, n, got)


# ---------------------------------------------------------------- transforms

def _regular(oracle_mod, T):
    nlat = T + 1
    rows = oracle_mod.grid_rows("regular", nlat, 2 * nlat)
    mu, w = oracle_mod.gauss(nlat)
    return rows, mu, w


def test_dft_stage_matches_numpy_rfft(oracle_mod):
    """The longitude stage is numpy.fft.rfft(row) / N_j truncated to m <= M_j."""
    T = 31
    rows = oracle_mod.grid_rows("octahedral", 32)
    g = inputs.grid_noise(int(rows.sum()), 2, seed=5)
    F = oracle_mod.dir_fourier(T, rows, g)
    off = np.concatenate([[0], np.cumsum(rows)])
    for f in range(2):
        for j in range(len(rows)):
            nj = rows[j]
            mj = min(T, (nj - 1) // 2)
            ref = np.fft.rfft(g[f, off[j]:off[j + 1]]) / nj
            ref = ref[:mj + 1].copy()
            ref[0] = ref[0].real
            assert np.max(np.abs(F[f, j, :mj + 1] - ref)) < 1e-14
            assert np.all(F[f, j, mj + 1:] == 0)


def test_synthesis_stage_matches_numpy_irfft(oracle_mod):
    T = 31
    rows = oracle_mod.grid_rows("octahedral", 32)
    rng = np.random.default_rng(3)
    four = rng.standard_normal((2, 32, T + 1)) + 1j * rng.standard_normal((2, 32, T + 1))
    for j in range(32):
        four[:, j, min(T, (rows[j] - 1) // 2) + 1:] = 0
    g = oracle_mod.inv_grid_from_fourier(T, rows, four)
    off = np.concatenate([[0], np.cumsum(rows)])
    for f in range(2):
        for j in range(32):
            nj = rows[j]
            spec = np.zeros(nj // 2 + 1, complex)
            mj = min(T, (nj - 1) // 2)
            spec[:mj + 1] = four[f, j, :mj + 1]
            spec[0] = spec[0].real
            ref = np.fft.irfft(spec * nj, n=nj)
            assert np.max(np.abs(g[f, off[j]:off[j + 1]] - ref)) < 1e-13


@pytest.mark.parametrize("m,n,val", [(0, 0, 1.0), (3, 7, 1.0), (3, 7, 1j), (12, 20, 1j), (31, 31, 1.0)])
def test_single_mode(oracle_mod, m, n, val):
    T = 31
    rows, mu, w = _regular(oracle_mod, T)
    a = np.zeros((1, oracle_mod.nspec(T)), complex)
    a[0, oracle_mod.spec_index(T, m, n)] = val
    g = oracle_mod.inv_trans(T, rows, mu, a)
    lam = 2 * np.pi * np.arange(rows[0]) / rows[0]
    for j in (0, 5, 16, 31):
        P = oracle_mod.legendre(T, mu[j])[oracle_mod.spec_index(T, m, n)]
        row = g[0, j * rows[0]:(j + 1) * rows[0]]
        if m == 0:
            ref = P * np.ones_like(lam) * val.real
        elif val == 1.0:
            ref = 2 * P * np.cos(m * lam)
        else:
            ref = -2 * P * np.sin(m * lam)
        assert np.max(np.abs(row - ref)) < 1e-13
    back = oracle_mod.dir_trans(T, rows, mu, w, g)
    assert np.max(np.abs(back - a)) < 1e-13


@pytest.mark.parametrize("T", [15, 31])
def test_round_trip_regular(oracle_mod, T):
    rows, mu, w = _regular(oracle_mod, T)
    a = inputs.spectra(T, 3, seed=1000)
    g = oracle_mod.inv_trans(T, rows, mu, a)
    b = oracle_mod.dir_trans(T, rows, mu, w, g)
    ac = a[..., 0] + 1j * a[..., 1]
    assert np.max(np.abs(b - ac)) < 1e-13
    g2 = oracle_mod.inv_trans(T, rows, mu, b)
    assert np.max(np.abs(g2 - g)) < 1e-13 * np.max(np.abs(g))


def test_round_trip_octahedral_band_limited(oracle_mod):
    """O32 with T = 11: every row has N_j >= 24 > 2T, so nothing aliases."""
    T, nlat = 11, 64
    rows = oracle_mod.grid_rows("octahedral", nlat)
    mu, w = oracle_mod.gauss(nlat)
    a = inputs.spectra(T, 2, seed=7)
    g = oracle_mod.inv_trans(T, rows, mu, a)
    b = oracle_mod.dir_trans(T, rows, mu, w, g)
    assert np.max(np.abs(b - (a[..., 0] + 1j * a[..., 1]))) < 1e-13


def test_parseval_regular(oracle_mod):
    T = 31
    rows, mu, w = _regular(oracle_mod, T)
    a = inputs.spectra(T, 2, seed=11)
    g = oracle_mod.inv_trans(T, rows, mu, a)
    N = rows[0]
    ac = a[..., 0] + 1j * a[..., 1]
    m_of = inputs.order_of_index(T)
    for f in range(2):
        lhs = float(np.sum(w * (g[f].reshape(len(rows), N) ** 2).sum(axis=1) / N))
        mult = np.where(m_of == 0, 1.0, 2.0)
        rhs = float(np.sum(mult * np.abs(ac[f]) ** 2))
        assert abs(lhs - rhs) < 1e-13 * rhs


def test_inverse_is_linear_and_fields_are_independent(oracle_mod):
    T = 15
    rows, mu, w = _regular(oracle_mod, T)
    a = inputs.spectra(T, 3, seed=2)
    g = oracle_mod.inv_trans(T, rows, mu, a)
    g1 = oracle_mod.inv_trans(T, rows, mu, a[1:2])
    assert np.array_equal(g[1:2], g1)
    g_sum = oracle_mod.inv_trans(T, rows, mu, a[0:1] + 2 * a[2:3])
    assert np.max(np.abs(g_sum - (g[0:1] + 2 * g[2:3]))) < 1e-13


# ---------------------------------------------------------------- grid geometry

def test_octahedral_grid_rule(oracle_mod):
    """Row i from either pole (i = 1 .. nlat/2) of the octahedral grid has
    20 + 4 i points (the configuration's O640 grid: 1280 latitudes, 24 points
    on the polar rows, 2580 on the two equatorial rows, 1 666 560 in all),
    mirrored about the equator."""
    rows = oracle_mod.grid_rows("octahedral", 1280)
    assert rows.shape == (1280,)
    assert rows[0] == rows[-1] == 24
    assert rows[639] == rows[640] == 2580
    assert int(rows.sum()) == 1_666_560
    for j in range(640):
        assert rows[j] == 20 + 4 * (j + 1) == rows[1279 - j], j
    # O1280 (2560 latitudes): 20 + 4 i up to 5140 points at the equator
    big = oracle_mod.grid_rows("octahedral", 2560)
    assert big[0] == 24 and big[1279] == big[1280] == 5140
    assert int(big.sum()) == 2 * sum(20 + 4 * i for i in range(1, 1281))


def test_regular_grid_rule(oracle_mod):
    rows = oracle_mod.grid_rows("regular", 160, 320)
    assert rows.shape == (160,) and np.all(rows == 320)
    with pytest.raises(RuntimeError):
        oracle_mod.grid_rows("regular", 31, 64)      # odd number of latitudes


# ---------------------------------------------------------------- derivatives
# Readings (the paper names the derivative and wind transforms of the time
# step but prints no formula): unit sphere, phi the latitude (mu = sin phi),
# H_n^m = (1 - mu^2) dPbar_n^m/dmu, wind images U = u cos(phi), V = v cos(phi),
# psi = -zeta / (n (n+1)), chi = -D / (n (n+1)).

@pytest.mark.parametrize("x", [-0.93, -0.2, 0.0, 0.41, 0.97])
def test_derivative_closed_forms(oracle_mod, x):
    q = oracle_mod.spec_index
    H = oracle_mod.legendre_deriv(3, x)
    s = math.sqrt(1 - x * x)
    assert abs(H[q(3, 0, 0)]) < 1e-15                                      # constant
    assert abs(H[q(3, 0, 1)] - math.sqrt(1.5) * (1 - x * x)) < 1e-14        # sqrt(3/2) mu
    assert abs(H[q(3, 1, 1)] + math.sqrt(3) / 2 * x * s) < 1e-14           # (sqrt 3 / 2) sin theta
    assert abs(H[q(3, 0, 2)] - math.sqrt(2.5) * 3 * x * (1 - x * x)) < 1e-14  # sqrt(5/2) (3 mu^2 - 1)/2


@pytest.mark.parametrize("x", [-0.7, 0.05, 0.6])
def test_derivative_values_match_finite_differences(oracle_mod, x):
    """H from the recurrence relation against a central difference of the
    oracle's own Pbar (fourth order), every (m, n) up to T = 12."""
    T, h = 12, 3e-4               # truncation error ~ h^4, about 1e-10 here
    P = [oracle_mod.legendre(T, x + k * h) for k in (-2, -1, 1, 2)]
    dP = (P[0] - 8 * P[1] + 8 * P[2] - P[3]) / (12 * h)
    H = oracle_mod.legendre_deriv(T, x)
    assert np.max(np.abs(H - (1 - x * x) * dP)) < 1e-9


def test_derivative_synthesis_matches_finite_differences(oracle_mod):
    """d/dlambda against a centred difference of the synthesis of the spectra
    rotated by +-delta (a_n^m e^{+-i m delta}); (1 - mu^2) d/dmu against a
    centred difference of the synthesis at mu +- delta.  Neither reference
    touches the derivative code."""
    T, nlat = 15, 16
    rows = oracle_mod.grid_rows("regular", nlat, 32)
    mu, _ = oracle_mod.gauss(nlat)
    a = inputs.spectra(T, 2, seed=41)
    ac = a[..., 0] + 1j * a[..., 1]
    m_of = inputs.order_of_index(T)
    dl, dm = oracle_mod.inv_trans_deriv(T, rows, mu, a)
    d = 1e-4                      # fourth-order differences: truncation error ~ 1e-10 here

    def diff4(f):
        return (f(-2) - 8 * f(-1) + 8 * f(1) - f(2)) / (12 * d)

    ref = diff4(lambda k: oracle_mod.inv_trans(T, rows, mu, ac * np.exp(1j * m_of * k * d)))
    assert np.max(np.abs(dl - ref)) / np.max(np.abs(ref)) < 1e-8
    w1 = np.repeat(1 - mu * mu, rows)
    ref = w1 * diff4(lambda k: oracle_mod.inv_trans(T, rows, mu + k * d, a))
    assert np.max(np.abs(dm - ref)) / np.max(np.abs(ref)) < 1e-8


def test_solid_body_rotation(oracle_mod):
    """Vorticity 2 Omega mu (zeta_1^0 = 2 Omega sqrt(2/3)) is the rotation
    u = Omega cos(phi), v = 0: U = Omega (1 - mu^2), V = 0."""
    T, nlat, om = 10, 12, 0.7
    rows = oracle_mod.grid_rows("regular", nlat, 24)
    mu, _ = oracle_mod.gauss(nlat)
    z = np.zeros((1, oracle_mod.nspec(T)), complex)
    z[0, oracle_mod.spec_index(T, 0, 1)] = 2 * om * math.sqrt(2.0 / 3.0)
    U, V = oracle_mod.inv_trans_uv(T, rows, mu, z, np.zeros_like(z))
    assert np.max(np.abs(U[0] - om * np.repeat(1 - mu * mu, rows))) < 1e-14
    assert np.max(np.abs(V)) < 1e-14


@pytest.mark.parametrize("T,nlat", [(15, 16), (31, 48)])
def test_wind_round_trip(oracle_mod, T, nlat):
    """Vorticity and divergence -> wind images -> vorticity and divergence is
    the identity on regular Gaussian grids (n = 0 terms zero)."""
    rows = oracle_mod.grid_rows("regular", nlat, 2 * nlat)
    mu, w = oracle_mod.gauss(nlat)
    z = inputs.spectra(T, 3, seed=51)
    dv = inputs.spectra(T, 3, seed=52)
    zc, dc = z[..., 0] + 1j * z[..., 1], dv[..., 0] + 1j * dv[..., 1]
    zc[:, 0] = 0
    dc[:, 0] = 0
    U, V = oracle_mod.inv_trans_uv(T, rows, mu, zc, dc)
    z2, d2 = oracle_mod.dir_trans_vordiv(T, rows, mu, w, U, V)
    assert np.max(np.abs(z2 - zc)) / np.max(np.abs(zc)) < 1e-13
    assert np.max(np.abs(d2 - dc)) / np.max(np.abs(dc)) < 1e-13
