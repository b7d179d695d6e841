"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: 1e-12 normwise for the FP64 path, 2e-5 for the FP32 / 3xTF32 / 3xBF16
paths (normwise max relative error per field: max |x - x*| / max |x*|).
Inputs are the seeded spectra of paper_1908_06096_gb300.inputs; direct-stage
inputs are grids the oracle synthesised from such spectra (band-limited).
"""
import numpy as np
import pytest
import torch

from paper_1908_06096_gb300 import inputs
from tests.conftest import max_rel, per_field_max_rel

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5, "tf32x3": 2e-5, "bf16x3": 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _grid_setup(oracle_mod, T, grid, nlat=None, nlon=None):
    if nlat is None:
        nlat = T + 1 if grid == "regular" else 2 * (T + 1)
        nlat += nlat & 1
    if nlon is None:
        nlon = 2 * nlat
    rows = oracle_mod.grid_rows(grid, nlat, nlon)
    mu, w = oracle_mod.gauss(nlat)
    return nlat, nlon, rows, mu, w


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


# ---------------------------------------------------------------- plan kernels

@pytest.mark.parametrize("nlat", [2, 32, 160, 1280, 2560])
def test_gauss_nodes_match_oracle(st_mod, oracle_mod, nlat):
    mu, w = st_mod.gauss_nodes(nlat)
    torch.cuda.synchronize()
    mu_o, w_o = oracle_mod.gauss(nlat)
    assert np.max(np.abs(mu.cpu().numpy() - mu_o)) <= 4e-16
    assert np.max(np.abs(w.cpu().numpy() - w_o)) <= 2e-16 * max(1.0, nlat / 100)


# Both sides run the same three-term recurrence in FP64, so they differ only
# by rounding, which grows with the degree: 1e-13 normwise up to T = 400, then
# a bound proportional to T (measured at T639: a few 1e-12; T1279 about twice).
@pytest.mark.parametrize("T,nlat", [(31, 32), (159, 160), (639, 1280), (1279, 1280), (1279, 2560)])
def test_legendre_values_match_oracle(st_mod, oracle_mod, T, nlat):
    mu_o, _ = oracle_mod.gauss(nlat)
    pick = np.unique(np.concatenate([np.linspace(0, nlat - 1, 9).astype(int), [1, nlat - 2]]))
    P = st_mod.legendre_values(T, torch.from_numpy(mu_o[pick])).cpu().numpy()
    tol = 1e-13 if T < 400 else 1e-11 * T / 639
    for i, j in enumerate(pick):
        ref = oracle_mod.legendre(T, mu_o[j])
        err = max_rel(P[i], ref)
        assert err < tol, (j, err)


def test_plan_nodes_and_rows(st_mod, oracle_mod):
    p = st_mod.Plan(63, "octahedral", precision="fp64", max_fields=1)
    mu, w = p.nodes()
    mu_o, w_o = oracle_mod.gauss(128)
    assert np.max(np.abs(mu - mu_o)) < 1e-15 and np.max(np.abs(w - w_o)) < 1e-15
    assert p.row_lengths() == list(oracle_mod.grid_rows("octahedral", 128))
    p.close()


# ---------------------------------------------------------------- stages (FP64)

@pytest.mark.parametrize("T,grid", [(31, "regular"), (31, "octahedral"), (47, "octahedral")])
def test_fourier_buffer_stages_fp64(st_mod, oracle_mod, T, grid):
    nlat, nlon, rows, mu, w = _grid_setup(oracle_mod, T, grid)
    nf = 3
    a = inputs.spectra(T, nf, seed=10)
    p = st_mod.Plan(T, grid, nlat=nlat, nlon=nlon, precision="fp64", max_fields=nf)
    spec = _dev(a, torch.float64)
    p.inv_legendre(spec)
    fb = p.fourier_export(0, nf).cpu().numpy()           # [2, T+1, J, nf]
    F = oracle_mod.inv_fourier(T, rows, mu, a)            # [nf, nlat, T+1]
    J = nlat // 2
    Fn = F[:, :J, :].transpose(2, 1, 0)                   # [T+1, J, nf]
    Fs = F[:, ::-1, :][:, :J, :].transpose(2, 1, 0)
    assert max_rel(fb[0], (Fn + Fs) / 2) < 1e-12
    assert max_rel(fb[1], (Fn - Fs) / 2) < 1e-12
    # inverse FFT stage on the GPU's own buffer
    g = p.inv_fft(nf).cpu().numpy()
    g_ref = oracle_mod.inv_trans(T, rows, mu, a)
    assert per_field_max_rel(g, g_ref) < 1e-12
    # direct FFT stage
    p.dir_fft(_dev(g_ref, torch.float64))
    fb = p.fourier_export(1, nf).cpu().numpy()
    D = oracle_mod.dir_fourier(T, rows, g_ref)
    Dn = D[:, :J, :].transpose(2, 1, 0)
    Ds = D[:, ::-1, :][:, :J, :].transpose(2, 1, 0)
    assert max_rel(fb[0], Dn + Ds) < 1e-12
    assert max_rel(fb[1], Dn - Ds) < 1e-12
    s = p.dir_legendre(nf).cpu().numpy()
    s_ref = oracle_mod.dir_trans(T, rows, mu, w, g_ref)
    sc = s[..., 0] + 1j * s[..., 1]
    assert per_field_max_rel(sc, s_ref) < 1e-12
    p.close()


# ---------------------------------------------------------------- full transforms

CASES = [
    # T, grid, nfields, precision
    (31, "regular", 10, "fp64"),
    (31, "octahedral", 3, "fp64"),
    (1, "regular", 1, "fp64"),
    (63, "regular", 33, "fp64"),
    (31, "regular", 10, "fp32"),
    (63, "octahedral", 5, "fp32"),
    (31, "regular", 10, "tf32x3"),
    (63, "octahedral", 33, "tf32x3"),
    (31, "regular", 10, "bf16x3"),
    (63, "octahedral", 33, "bf16x3"),
    (127, "regular", 70, "bf16x3"),
    (95, "octahedral", 129, "bf16x3"),
]


@pytest.mark.parametrize("T,grid,nf,prec", CASES)
def test_transforms_match_oracle(st_mod, oracle_mod, T, grid, nf, prec):
    nlat, nlon, rows, mu, w = _grid_setup(oracle_mod, T, grid)
    dt = torch.float64 if prec == "fp64" else torch.float32
    a = inputs.spectra(T, nf, seed=1000 + T + nf)
    p = st_mod.Plan(T, grid, nlat=nlat, nlon=nlon, precision=prec, max_fields=nf)
    g = p.inv(_dev(a, dt))
    g_ref = oracle_mod.inv_trans(T, rows, mu, a)
    err_inv = per_field_max_rel(g.double().cpu().numpy(), g_ref)
    # direct from the oracle's (band-limited) grid, rounded to the plan's type
    g_in = _dev(g_ref, dt)
    s = p.dir(g_in)
    p.sync()
    s_ref = oracle_mod.dir_trans(T, rows, mu, w, g_in.double().cpu().numpy())
    s = s.double().cpu().numpy()
    err_dir = per_field_max_rel(s[..., 0] + 1j * s[..., 1], s_ref)
    assert err_inv < TOL[prec], err_inv
    assert err_dir < TOL[prec], err_dir
    assert np.all(s[:, inputs.order_of_index(T) == 0, 1] == 0)
    p.close()


def test_round_trip_fp64_regular_identity(st_mod, oracle_mod):
    T, nf = 31, 10
    a = inputs.spectra(T, nf, seed=1000)
    p = st_mod.Plan(T, "regular", precision="fp64", max_fields=nf)
    b = p.dir(p.inv(_dev(a, torch.float64))).cpu().numpy()
    assert np.max(np.abs(b - a)) < 1e-13
    p.close()


def test_fields_independent_and_reusable_plan(st_mod):
    """A field's result is bit for bit the same alone and inside a batch, and
    repeated calls with different field counts on one plan agree: every field
    takes the same arithmetic in the same order whatever the field count (the
    GEMMs accumulate each data column alone; an FFT row's fields per CTA only
    change which slot holds a field)."""
    T = 63
    a = inputs.spectra(T, 40, seed=3)
    for prec, tol in (("fp64", 0.0), ("bf16x3", 0.0), ("tf32x3", 0.0)):
        dt = torch.float64 if prec == "fp64" else torch.float32
        p = st_mod.Plan(T, "octahedral", precision=prec, max_fields=40)
        p.inv(_dev(inputs.spectra(T, 40, seed=99), dt))   # leave other data in the workspace
        g_all = p.inv(_dev(a, dt)).clone()
        g_one = p.inv(_dev(a[17:18], dt)).clone()
        g_few = p.inv(_dev(a[15:20], dt)).clone()
        s_all = p.dir(g_all).clone()
        s_one = p.dir(g_all[17:18].contiguous()).clone()
        torch.cuda.synchronize()
        g_all, g_one, g_few = g_all.cpu().numpy(), g_one.cpu().numpy(), g_few.cpu().numpy()
        assert max_rel(g_one[0], g_all[17]) <= tol
        assert max_rel(g_few, g_all[15:20]) <= tol
        assert max_rel(s_one.cpu().numpy()[0], s_all.cpu().numpy()[17]) <= tol
        p.close()


def test_nfields_bounds(st_mod):
    p = st_mod.Plan(31, "regular", precision="fp32", max_fields=4)
    x = torch.zeros((5, p.nspec, 2), device="cuda")
    with pytest.raises(st_mod.STError):
        p.inv(x)
    p.close()


# Rows whose length is not a multiple of 4 take the scalar grid path of the
# FFT kernels (the others move 4 points per access): nlon = 66 = 2 3 11 runs
# Bluestein rows, nlon = 90 = 2 3^2 5 mixed-radix rows.
ODD_ROWS = [
    (31, 32, 66, "bf16x3"),
    (31, 32, 90, "bf16x3"),
    (31, 32, 66, "fp32"),
    (31, 32, 90, "fp64"),
]


@pytest.mark.parametrize("T,nlat,nlon,prec", ODD_ROWS)
def test_rows_not_multiple_of_four(st_mod, oracle_mod, T, nlat, nlon, prec):
    nf = 7
    rows = oracle_mod.grid_rows("regular", nlat, nlon)
    mu, w = oracle_mod.gauss(nlat)
    dt = torch.float64 if prec == "fp64" else torch.float32
    a = inputs.spectra(T, nf, seed=2000 + nlon)
    p = st_mod.Plan(T, "regular", nlat=nlat, nlon=nlon, precision=prec, max_fields=nf)
    g = p.inv(_dev(a, dt))
    g_ref = oracle_mod.inv_trans(T, rows, mu, a)
    assert per_field_max_rel(g.double().cpu().numpy(), g_ref) < TOL[prec]
    g_in = _dev(g_ref, dt)
    s = p.dir(g_in)
    p.sync()
    s_ref = oracle_mod.dir_trans(T, rows, mu, w, g_in.double().cpu().numpy())
    s = s.double().cpu().numpy()
    assert per_field_max_rel(s[..., 0] + 1j * s[..., 1], s_ref) < TOL[prec]
    p.close()


def test_grid_pointer_off_16_byte_boundary(st_mod):
    """A grid buffer 4 bytes past a 16-byte boundary takes the scalar path and
    gives the same numbers as an aligned one."""
    T, nf = 63, 9
    p = st_mod.Plan(T, "octahedral", precision="bf16x3", max_fields=nf)
    spec = _dev(inputs.spectra(T, nf, seed=77), torch.float32)
    g_al = p.inv(spec).clone()
    flat = torch.zeros(nf * p.npts + 4, dtype=torch.float32, device="cuda")
    g_off = flat[1:1 + nf * p.npts].view(nf, p.npts)
    assert g_off.data_ptr() % 16 == 4
    p.inv(spec, out=g_off)
    s_al = p.dir(g_al).clone()
    s_off = p.dir(g_off).clone()
    torch.cuda.synchronize()
    assert max_rel(g_off.cpu().numpy(), g_al.cpu().numpy()) <= 1e-6
    assert max_rel(s_off.cpu().numpy(), s_al.cpu().numpy()) <= 1e-6
    p.close()
