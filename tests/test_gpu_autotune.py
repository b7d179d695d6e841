"""Autotuner: the tuned plan still matches the oracle, the choice lands in the
cache file, and a new plan with the same key picks it up at creation."""
import os

import numpy as np
import pytest
import torch

from paper_1908_06096_gb300 import inputs
from tests.conftest import per_field_max_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_autotune_keeps_results_and_caches(st_mod, oracle_mod, tmp_path, monkeypatch):
    T, nf = 95, 24
    cache = str(tmp_path / "tune.txt")
    p = st_mod.Plan(T, "octahedral", precision="bf16x3", max_fields=nf)
    p.autotune(nf, cache_path=cache)
    shape = p.launch_shape()
    assert shape[4] in (64, 96, 128, 160, 192, 224, 256)
    assert shape[5] in (0, 64, 96, 128, 160, 192, 224, 256)
    a = inputs.spectra(T, nf, seed=31)
    g = p.inv(torch.from_numpy(a).to("cuda", torch.float32))
    nlat = 2 * (T + 1)
    rows = oracle_mod.grid_rows("octahedral", nlat)
    mu, w = oracle_mod.gauss(nlat)
    g_ref = oracle_mod.inv_trans(T, rows, mu, a)
    assert per_field_max_rel(g.double().cpu().numpy(), g_ref) < 2e-5
    s = p.dir(torch.from_numpy(g_ref).to("cuda", torch.float32))
    p.sync()
    s_ref = oracle_mod.dir_trans(T, rows, mu, w, torch.from_numpy(g_ref).float().double().numpy())
    s = s.double().cpu().numpy()
    assert per_field_max_rel(s[..., 0] + 1j * s[..., 1], s_ref) < 2e-5
    p.close()
    assert os.path.exists(cache) and open(cache).read().strip()
    monkeypatch.setenv("ST_TUNE_CACHE", cache)
    q = st_mod.Plan(T, "octahedral", precision="bf16x3", max_fields=nf)
    assert q.launch_shape() == shape
    q.close()


def test_split_tile_widths_match_oracle(st_mod, oracle_mod, tmp_path, monkeypatch):
    """Different inverse column-tile widths below and above the middle
    wavenumber (set through a cache entry) lay the tables out per group and
    still give the oracle's grid."""
    T, nf = 127, 6
    cache = str(tmp_path / "tune.txt")
    # the entry the autotuner writes for this plan, with its tile widths replaced
    p1 = st_mod.Plan(T, "octahedral", precision="bf16x3", max_fields=nf)
    p1.autotune(nf, cache_path=cache)
    p1.close()
    head, vals = open(cache).read().strip().splitlines()[-1].split("|")
    v = vals.split()
    v[4], v[5] = "64", "128"
    open(cache, "w").write(head + "| " + " ".join(v) + "\n")
    monkeypatch.setenv("ST_TUNE_CACHE", cache)
    p = st_mod.Plan(T, "octahedral", precision="bf16x3", max_fields=nf)
    assert p.launch_shape()[4:6] == [64, 128]
    a = inputs.spectra(T, nf, seed=37)
    g = p.inv(torch.from_numpy(a).to("cuda", torch.float32))
    p.sync()
    nlat = 2 * (T + 1)
    rows = oracle_mod.grid_rows("octahedral", nlat)
    mu, _ = oracle_mod.gauss(nlat)
    assert per_field_max_rel(g.double().cpu().numpy(), oracle_mod.inv_trans(T, rows, mu, a)) < 2e-5
    p.close()
