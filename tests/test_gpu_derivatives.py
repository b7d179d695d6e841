"""Derivative and wind transforms (st_inv_trans_deriv, st_inv_trans_uv,
st_dir_trans_vordiv) against the FP64 oracle's definitions, through the C ABI.

Unit sphere, phi the latitude, mu = sin(phi): d/dlambda and
(1 - mu^2) d/dmu of scalar fields; wind images U = u cos(phi),
V = v cos(phi) from vorticity and divergence and back.  Bars as for the
scalar transforms: 1e-12 normwise per field in FP64, 2e-5 in the FP32 forms.
"""
import math

import numpy as np
import pytest
import torch

from paper_1908_06096_gb300 import inputs
from tests.conftest import per_field_max_rel

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5, "tf32x3": 2e-5, "bf16x3": 2e-5}
# Vorticity and divergence from winds differentiate the wind: the split
# products' relative error (about 1e-5 in BF16x3, 16 significant bits per
# operand) reaches the high-degree coefficients amplified by about the
# degree over the wind's own decay.  Measured 4.2e-5 (T31) and 4.6e-5 (T63)
# in BF16x3; 1e-4 is that with margin.  The 24-bit forms stay within 2e-5.
TOL_VORDIV = dict(TOL, bf16x3=1e-4)


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _geo(oracle_mod, grid, nlat, nlon):
    rows = oracle_mod.grid_rows(grid, nlat, nlon)
    mu, w = oracle_mod.gauss(nlat)
    return rows, mu, w


def _cplx(x):
    x = np.asarray(x, dtype=np.float64)
    return x[..., 0] + 1j * x[..., 1]


def _vordiv(T, nf, seed):
    z = inputs.spectra(T, nf, seed=seed)
    d = inputs.spectra(T, nf, seed=seed + 1)
    z[:, 0] = 0.0           # the n = 0 coefficient of a vorticity or divergence field is zero
    d[:, 0] = 0.0
    return z, d


CASES = [
    # T, grid, nlat, nlon, nfields, precision
    (31, "regular", 32, 64, 3, "fp64"),
    (47, "octahedral", 96, 0, 2, "fp64"),
    (31, "regular", 32, 64, 5, "fp32"),
    (31, "regular", 32, 64, 5, "tf32x3"),
    (47, "octahedral", 96, 0, 4, "tf32x3"),
    (31, "regular", 32, 64, 5, "bf16x3"),
    (63, "octahedral", 128, 0, 7, "bf16x3"),
]


@pytest.mark.parametrize("T,grid,nlat,nlon,nf,prec", CASES)
def test_derivatives_and_winds_match_oracle(st_mod, oracle_mod, T, grid, nlat, nlon, nf, prec):
    rows, mu, w = _geo(oracle_mod, grid, nlat, nlon)
    p = st_mod.Plan(T, grid, nlat=nlat, nlon=nlon or None, precision=prec, max_fields=2 * nf)
    p.enable_derivatives()
    dt = p.dtype
    tol = TOL[prec]

    # scalar derivatives
    a = inputs.spectra(T, nf, seed=700 + T)
    dl, dm = p.inv_deriv(_dev(a, dt))
    dl_ref, dm_ref = oracle_mod.inv_trans_deriv(T, rows, mu, a)
    err = per_field_max_rel(dl.double().cpu().numpy(), dl_ref)
    assert err < tol, ("d/dlambda", err)
    err = per_field_max_rel(dm.double().cpu().numpy(), dm_ref)
    assert err < tol, ("cos(phi) d/dphi", err)

    # winds from vorticity and divergence
    z, d = _vordiv(T, nf, seed=800 + T)
    U, V = p.inv_uv(_dev(z, dt), _dev(d, dt))
    U_ref, V_ref = oracle_mod.inv_trans_uv(T, rows, mu, z, d)
    err = per_field_max_rel(U.double().cpu().numpy(), U_ref)
    assert err < tol, ("U", err)
    err = per_field_max_rel(V.double().cpu().numpy(), V_ref)
    assert err < tol, ("V", err)

    # vorticity and divergence from the oracle's (band-limited) winds
    Ug, Vg = _dev(U_ref, dt), _dev(V_ref, dt)
    z2, d2 = p.dir_vordiv(Ug, Vg)
    p.sync()
    z_ref, d_ref = oracle_mod.dir_trans_vordiv(T, rows, mu, w, Ug.double().cpu().numpy(), Vg.double().cpu().numpy())
    err = per_field_max_rel(_cplx(z2.double().cpu().numpy()), z_ref)
    assert err < TOL_VORDIV[prec], ("vorticity", err)
    err = per_field_max_rel(_cplx(d2.double().cpu().numpy()), d_ref)
    assert err < TOL_VORDIV[prec], ("divergence", err)
    p.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_solid_body_rotation_on_gpu(st_mod, prec):
    """Vorticity 2 Omega mu gives U = Omega (1 - mu^2), V = 0, and back."""
    T, nlat, om = 31, 32, 0.7
    p = st_mod.Plan(T, "regular", nlat=nlat, nlon=64, precision=prec, max_fields=2)
    p.enable_derivatives()
    z = np.zeros((1, p.nspec, 2))
    z[0, 1, 0] = 2 * om * math.sqrt(2.0 / 3.0)         # (m, n) = (0, 1) sits at index 1
    U, V = p.inv_uv(_dev(z, p.dtype), _dev(np.zeros_like(z), p.dtype))
    mu, _ = p.nodes()
    U_ref = om * np.repeat(1 - mu * mu, 64)
    tol = TOL[prec]
    assert np.max(np.abs(U.double().cpu().numpy()[0] - U_ref)) <= tol * om
    assert np.max(np.abs(V.double().cpu().numpy())) <= tol * om
    z2, d2 = p.dir_vordiv(U, V)
    p.sync()
    tol = TOL_VORDIV[prec]
    assert np.max(np.abs(z2.double().cpu().numpy() - z)) <= tol * 2 * om
    assert np.max(np.abs(d2.double().cpu().numpy())) <= tol * 2 * om
    p.close()


def test_derivative_calls_need_enable_and_room(st_mod):
    p = st_mod.Plan(31, "regular", precision="bf16x3", max_fields=3)
    x = torch.zeros((2, p.nspec, 2), device="cuda")
    with pytest.raises(st_mod.STError):
        p.inv_deriv(x)                       # not enabled
    p.enable_derivatives()
    with pytest.raises(st_mod.STError):
        p.inv_deriv(x)                       # 2 x 2 fields > max_fields 3
    a, b = p.inv_deriv(x[:1])
    p.sync()
    assert float(a.abs().max()) == 0.0 and float(b.abs().max()) == 0.0
    p.close()
