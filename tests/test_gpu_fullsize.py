"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (all fields in one call), on fields the oracle computes one by one:

  T639 on O640 (1280 latitudes, rows 20 + 4i), 548 fields, spectra
  N(0,1) (n+1)^-1.5, in every form the benchmark times: BF16x3 and 3xTF32
  (fields 0, 273 and 547; bar 2e-5) and FP64 (fields 0 and 547; bar 1e-12);
  T159 on the regular 160 x 320 grid, 411 fields, FP64 and 3xTF32 — fields
  0 and 410;
  T1279 on the regular 1280 x 2560 grid (the largest truncation the serving
  mix uses), 16 fields, BF16x3 and FP64 — fields 0 and 15;
  T1279 on O1280 (2560 latitudes, rows 20 + 4i up to 5140 points, FFT lengths
  up to 8192), 24 fields in BF16x3 and 4 in FP64 — the first and last field.

Inverse: GPU grid of the sampled fields vs the oracle's synthesis of the same
spectra.  Direct: the sampled fields' grids are replaced by the oracle's
(band-limited) grids before the GPU direct transform of the whole batch; GPU
spectra of those fields vs the oracle's analysis of the same grids.
"""
import numpy as np
import pytest
import torch

from paper_1908_06096_gb300 import inputs
from tests.conftest import per_field_max_rel

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "tf32x3": 2e-5, "bf16x3": 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


CASES = [
    (639, "octahedral", 1280, 0, 548, 1.5, 1002, "bf16x3", (0, 273, 547)),
    (639, "octahedral", 1280, 0, 548, 1.5, 1002, "tf32x3", (0, 273, 547)),
    (639, "octahedral", 1280, 0, 548, 1.5, 1002, "fp64", (0, 547)),
    (159, "regular", 160, 320, 411, 1.0, 1001, "fp64", (0, 410)),
    (159, "regular", 160, 320, 411, 1.0, 1001, "tf32x3", (0, 410)),
    (1279, "regular", 1280, 2560, 16, 1.0, 1004, "bf16x3", (0, 15)),
    (1279, "regular", 1280, 2560, 16, 1.0, 1004, "fp64", (0, 15)),
    (1279, "octahedral", 2560, 0, 24, 1.5, 1005, "bf16x3", (0, 23)),
    (1279, "octahedral", 2560, 0, 4, 1.5, 1005, "fp64", (0, 3)),
]


@pytest.mark.parametrize("T,grid,nlat,nlon,F,pdec,seed,prec,sample", CASES)
def test_full_size_sampled_fields(st_mod, oracle_mod, T, grid, nlat, nlon, F, pdec, seed, prec, sample):
    a = inputs.spectra(T, F, seed=seed, p=pdec)
    plan = st_mod.Plan(T, grid, nlat=nlat, nlon=nlon or None, precision=prec, max_fields=F)
    dt = plan.dtype
    g = plan.inv(torch.from_numpy(a).to("cuda", dt))
    rows = oracle_mod.grid_rows(grid, nlat, nlon)
    mu, w = oracle_mod.gauss(nlat)
    idx = list(sample)
    g_ref = oracle_mod.inv_trans(T, rows, mu, a[idx])
    g_gpu = g[idx].double().cpu().numpy()
    err = per_field_max_rel(g_gpu, g_ref)
    assert err < TOL[prec], err
    # direct: put the oracle's grids into the sampled slots of the batch
    g_in = g.clone()
    g_in[idx] = torch.from_numpy(g_ref).to("cuda", dt)
    s = plan.dir(g_in)
    plan.sync()
    s_ref = oracle_mod.dir_trans(T, rows, mu, w, g_in[idx].double().cpu().numpy())
    s_gpu = s[idx].double().cpu().numpy()
    err = per_field_max_rel(s_gpu[..., 0] + 1j * s_gpu[..., 1], s_ref)
    assert err < TOL[prec], err
    plan.close()
